// Internal interface between the translation units of the operator apply: the stencil registry
// (central rows of every registered level, host copy), the device helpers every apply kernel's
// fused epilogue uses, and the launchers that live in their own translation units.
#pragma once
#include <cuda_runtime.h>

#include "cd_internal.h"

namespace cd {

struct StencilHost {
  int m, P, lo, hi;
  double c[3][13];
  float2* ffT;  // device: the level's k-major bands [3][2P+1][m] split into (hi, lo) FP32 pairs
};
// the registered level whose band device pointer is bands_dev (false: none)
bool find_level(const void* bands_dev, StencilHost& out);

// M and S palindromes and A skew with a zero centre: the folded interior forms need that exactly
inline bool stencil_folds(const StencilHost& sh) {
  const int P = sh.P;
  for (int t = 1; t <= P; ++t) {
    if (sh.c[0][P - t] != sh.c[0][P + t] || sh.c[2][P - t] != sh.c[2][P + t]) return false;
    if (sh.c[1][P - t] != -sh.c[1][P + t]) return false;
  }
  return sh.c[1][P] == 0.0;
}

// ---- device helpers
static __device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a double (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
static __device__ inline double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Chebyshev step coefficients of one solve: d = c1 dprev + c2 D^{-1} r (c1 = 0 for step 0).
static __device__ __forceinline__ void cheb_coef(double lmax, int step, double& c1, double& c2) {
  const double hi = kChebHi * lmax, lo = hi / kChebRatio;
  const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sigma = th / de;
  if (step == 0) {
    c1 = 0.0;
    c2 = 1.0 / th;
    return;
  }
  double rho_prev = 1.0 / sigma, rho = rho_prev;
  for (int j = 1; j <= step; ++j) {
    rho_prev = rho;
    rho = 1.0 / (2.0 * sigma - rho_prev);
  }
  c1 = rho * rho_prev;
  c2 = 2.0 * rho / de;
}

// The same coefficients computed once per CTA (thread 0, FP64) and shared.  GB300's FP64 pipe
// runs at 1/64 of the FP32 rate, so a per-thread FP64 recurrence with divisions costs more than
// a whole FP32 stencil.  Every thread of the CTA must reach this call.
static __device__ __forceinline__ void cheb_coef_cta(double lmax, int step, double& c1, double& c2) {
  __shared__ double s_cc[2];
  if (threadIdx.x == 0) {
    double a, b;
    cheb_coef(lmax, step, a, b);
    s_cc[0] = a;
    s_cc[1] = b;
  }
  __syncthreads();
  c1 = s_cc[0];
  c2 = s_cc[1];
}

// fused Chebyshev smoother step of one grid point: x = x_prev + d, d = c2 D^{-1} r + c1 d_prev
template <typename T>
static __device__ __forceinline__ void cheb_epi(const Epi<T>& e, long long o, T r, T dinv, T c1, T c2) {
  T d = c2 * dinv * r;
  if (e.step > 0) d += c1 * e.dprev[o];
  e.xout[o] = e.xprev[o] + d;
  if (e.dout) e.dout[o] = d;
  if (e.rout) e.rout[o] = r;
}

// ---- launchers in other translation units
// double-FP32 2D apply (apply2d_ff.cu): kernel 2 = packed folded kernel, 1 = plain kernel; false
// when the level or the arguments do not fit (the caller then takes an FP64 kernel)
bool try_apply2d_ff(int m, int P, const double* bands, const double* w, double* y, const double* rhs,
                    int mode, int B, Coef c, double* dotp, int* nblk, const int* active,
                    cudaStream_t s, const Epi<double>& epi, int kernel);
void prepare_ff_kernels();
// 3D tuned passes (apply3d_pass.cu), y = A w; false when the level is not registered or P > 6.
// scratch: 18 m^3 B elements (the double-FP32 form: 18 m^3 B float2 pairs)
bool launch_pass3d_f32(int m, int P, const float* bands, const float* w, float* y, int B, Coef c,
                       const int* active, float* scratch, cudaStream_t s);
bool launch_pass3d_f64(int m, int P, const double* bands, const double* w, double* y, int B, Coef c,
                       const int* active, double* scratch, cudaStream_t s);
bool launch_pass3d_ff(int m, int P, const double* bands, const double* w, double* y, int B, Coef c,
                      const int* active, float2* scratch, cudaStream_t s);

}  // namespace cd
