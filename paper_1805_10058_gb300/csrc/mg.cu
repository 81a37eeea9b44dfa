// Multigrid kernels and the V-cycle (Section 6.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <thread>

#include "krylov.h"
#include "mg.h"
#include "ffmath.h"

namespace cd {

static constexpr int kPowerIts = 14;

MgData::~MgData() {
  for (void* p : owned) cudaFree(p);
}

// ------------------------------------------------------------------ transfer kernels
// coarse(J) = sum over taps a in {0,1,2}^d of prod_l w_{a_l} fine(2 J_l + a_l), w = (1/2, 1, 1/2).
// The tap weights (1, 1/2, 1/4, 1/8) are exact in every precision; the index arithmetic is 32-bit
// (one solve's vector has fewer than 2^31 entries on every level this library builds: the
// set-up rejects larger problems).
// Accumulation type A: T itself, or float for FP64 vectors whose transfers run on the FP32 pipe
// (the FP64 inner solves with double-FP32 applies): the taps' FP32 truncations (integer
// operations) are summed in FP32 and the sum is widened exactly, leaving one FP64 operation per
// output (the prolongation's add) instead of several on GB300's narrow FP64 pipe.  A multigrid
// correction, like a smoother step, needs no more than FP32 accuracy inside a flexible Krylov
// solve whose residuals stay FP64.
template <typename A, typename T>
__device__ __forceinline__ A tap_load(T v) {
  if constexpr (sizeof(A) == 4 && sizeof(T) == 8) return ff_split_bits(v).x;
  else return (A)v;
}
template <typename T, typename A>
__device__ __forceinline__ T tap_widen(A v) {
  if constexpr (sizeof(A) == 4 && sizeof(T) == 8) return f2d_bits(v);
  else return (T)v;
}

template <typename T, typename A>
__global__ void __launch_bounds__(256) restrict_kernel(int d, int mf, int mc, const T* __restrict__ fine,
                                                       T* __restrict__ coarse,
                                                       const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nfc = d == 2 ? mf * mf : mf * mf * mf, ncc = d == 2 ? mc * mc : mc * mc * mc;
  const int total = d * ncc;
  const T* fb = fine + (long long)b * d * nfc;
  T* cb = coarse + (long long)b * total;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int comp = idx / ncc;
    int rem = idx - comp * ncc;
    int J[3] = {0, 0, 0};
    for (int l = d - 1; l >= 0; --l) {
      const int q = rem / mc;
      J[l] = rem - q * mc;
      rem = q;
    }
    const T* src = fb + (long long)comp * nfc;
    A acc = 0;
    if (d == 2) {
#pragma unroll
      for (int a0 = 0; a0 < 3; ++a0) {
        const int i0 = 2 * J[0] + a0;
        if (i0 >= mf) break;
        A row = 0;
#pragma unroll
        for (int a1 = 0; a1 < 3; ++a1) {
          const int i1 = 2 * J[1] + a1;
          if (i1 >= mf) break;
          const A v = tap_load<A>(src[i0 * mf + i1]);
          row += a1 == 1 ? v : A(0.5) * v;
        }
        acc += a0 == 1 ? row : A(0.5) * row;
      }
    } else {
#pragma unroll 1
      for (int a0 = 0; a0 < 3; ++a0) {
        const int i0 = 2 * J[0] + a0;
        if (i0 >= mf) break;
        A pl = 0;
        for (int a1 = 0; a1 < 3; ++a1) {
          const int i1 = 2 * J[1] + a1;
          if (i1 >= mf) break;
          A row = 0;
#pragma unroll
          for (int a2 = 0; a2 < 3; ++a2) {
            const int i2 = 2 * J[2] + a2;
            if (i2 >= mf) break;
            const A v = tap_load<A>(src[((long long)i0 * mf + i1) * mf + i2]);
            row += a2 == 1 ? v : A(0.5) * v;
          }
          pl += a1 == 1 ? row : A(0.5) * row;
        }
        acc += a0 == 1 ? pl : A(0.5) * pl;
      }
    }
    cb[idx] = tap_widen<T>(acc);
  }
}

// fine(i) += sum_J prod_l P(i_l, J_l) coarse(J); P(i, J) = 1 if i = 2J+1, 1/2 if i = 2J or 2J+2
template <typename T, typename A>
__global__ void __launch_bounds__(256) prolong_kernel(int d, int mf, int mc, const T* __restrict__ coarse,
                                                      T* __restrict__ fine,
                                                      const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nfc = d == 2 ? mf * mf : mf * mf * mf, ncc = d == 2 ? mc * mc : mc * mc * mc;
  const int total = d * nfc;
  const T* cb = coarse + (long long)b * d * ncc;
  T* fb = fine + (long long)b * total;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int comp = idx / nfc;
    int rem = idx - comp * nfc;
    int I[3] = {0, 0, 0};
    for (int l = d - 1; l >= 0; --l) {
      const int q = rem / mf;
      I[l] = rem - q * mf;
      rem = q;
    }
    // per axis: one coarse index with weight 1 (odd i) or up to two with weight 1/2 (even i)
    int j0[3], j1[3];  // j1 = -1: no second index
    bool half[3];
    for (int l = 0; l < d; ++l) {
      const int i = I[l];
      if (i & 1) {
        j0[l] = (i - 1) / 2;
        j1[l] = -1;
        half[l] = false;
      } else {
        j0[l] = i / 2 < mc ? i / 2 : -1;
        j1[l] = i / 2 - 1;
        half[l] = true;
      }
    }
    const T* src = cb + (long long)comp * ncc;
    A acc = 0;
    if (d == 2) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int ja = a == 0 ? j0[0] : j1[0];
        if (ja < 0 || ja >= mc) continue;
        A row = 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int jc = c == 0 ? j0[1] : j1[1];
          if (jc < 0 || jc >= mc) continue;
          row += tap_load<A>(src[ja * mc + jc]);
        }
        acc += half[1] ? A(0.5) * row : row;
      }
      if (half[0]) acc = A(0.5) * acc;
    } else {
      for (int a = 0; a < 2; ++a) {
        const int ja = a == 0 ? j0[0] : j1[0];
        if (ja < 0 || ja >= mc) continue;
        A pl = 0;
        for (int c = 0; c < 2; ++c) {
          const int jc = c == 0 ? j0[1] : j1[1];
          if (jc < 0 || jc >= mc) continue;
          A row = 0;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int je = e == 0 ? j0[2] : j1[2];
            if (je < 0 || je >= mc) continue;
            row += tap_load<A>(src[((long long)ja * mc + jc) * mc + je]);
          }
          pl += half[2] ? A(0.5) * row : row;
        }
        acc += half[1] ? A(0.5) * pl : pl;
      }
      if (half[0]) acc = A(0.5) * acc;
    }
    fb[idx] += tap_widen<T>(acc);
  }
}

static inline dim3 grid_for(long long n, int B) {
  long long nb = (n + 255) / 256;
  nb = std::max<long long>(1, std::min<long long>(nb, 4096));
  return dim3((unsigned)nb, B);
}

template <typename T>
void mg_restrict(int d, int mf, int mc, int B, const T* fine, T* coarse, const int* active,
                 cudaStream_t s) {
  long long nc = d;
  for (int l = 0; l < d; ++l) nc *= mc;
  if (sizeof(T) == 8 && fp64_emulated())
    restrict_kernel<T, float><<<grid_for(nc, B), 256, 0, s>>>(d, mf, mc, fine, coarse, active);
  else
    restrict_kernel<T, T><<<grid_for(nc, B), 256, 0, s>>>(d, mf, mc, fine, coarse, active);
  count_launch();
}
template <typename T>
void mg_prolong_add(int d, int mf, int mc, int B, const T* coarse, T* fine, const int* active,
                    cudaStream_t s) {
  long long nf = d;
  for (int l = 0; l < d; ++l) nf *= mf;
  if (sizeof(T) == 8 && fp64_emulated())
    prolong_kernel<T, float><<<grid_for(nf, B), 256, 0, s>>>(d, mf, mc, coarse, fine, active);
  else
    prolong_kernel<T, T><<<grid_for(nf, B), 256, 0, s>>>(d, mf, mc, coarse, fine, active);
  count_launch();
}
template void mg_restrict<double>(int, int, int, int, const double*, double*, const int*, cudaStream_t);
template void mg_restrict<float>(int, int, int, int, const float*, float*, const int*, cudaStream_t);
template void mg_prolong_add<double>(int, int, int, int, const double*, double*, const int*, cudaStream_t);
template void mg_prolong_add<float>(int, int, int, int, const float*, float*, const int*, cudaStream_t);

// ------------------------------------------------------------------ Jacobi / Chebyshev
// 1 / diag of the block operator at (comp, multi-index): the diagonal of block c is
// sum_l c_{c,l} prod_k X_k(i_k, i_k) with X_k = S on axis l and M elsewhere, c = beta on the
// component's own axis and alpha on the others.
template <typename T>
__device__ __forceinline__ T dinv_at(int d, int m, int P, const T* bands, int comp,
                                     const int* I, double al, double be) {
  const int W = 2 * P + 1;
  const T* Mb = bands;
  const T* Sb = bands + 2 * (size_t)m * W;
  double diag = 0.0;
  for (int l = 0; l < d; ++l) {
    double t = (l == comp) ? be : al;
    for (int k = 0; k < d; ++k) t *= (double)((k == l) ? Sb[I[k] * W + P] : Mb[I[k] * W + P]);
    diag += t;
  }
  return T(1.0 / diag);
}

__device__ __forceinline__ void decode(int d, int m, long long nper, long long idx, int& comp,
                                       int* I) {
  comp = (int)(idx / nper);
  long long rem = idx - comp * nper;
  for (int l = d - 1; l >= 0; --l) {
    I[l] = (int)(rem % m);
    rem /= m;
  }
}

__device__ __forceinline__ void cheb_params(double lmax, double& theta, double& delta) {
  const double hi = kChebHi * lmax, lo = hi / kChebRatio;
  theta = 0.5 * (hi + lo);
  delta = 0.5 * (hi - lo);
}

// d = D^{-1} r / theta; x = (xzero ? 0 : x) + d   (dinv: precomputed 1 / diag per solve).
// The per-solve scalar is formed once per CTA (FP64 divisions per thread are expensive on
// GB300).  lowp (FP64 vectors only): d in FP32 arithmetic from the FP32 truncations of dinv and
// r, exactly widened (a smoother step needs no more; x and the residuals stay FP64).
template <typename T>
__global__ void __launch_bounds__(256) cheb_first_kernel(long long N, const T* __restrict__ dinv,
                                                         const double* __restrict__ lmax,
                                                         const T* __restrict__ r, T* __restrict__ x,
                                                         T* __restrict__ dv, int xzero,
                                                         const int* __restrict__ active, int lowp) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ double s_ith;
  __shared__ float s_ithf;
  if (threadIdx.x == 0) {
    double th, de;
    cheb_params(lmax[b], th, de);
    s_ith = 1.0 / th;
    s_ithf = (float)s_ith;
  }
  __syncthreads();
  const long long base = (long long)b * N;
  if (sizeof(T) == 8 && lowp) {
    const float ith = s_ithf;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
      const float vf = ff_split_bits((double)dinv[base + idx]).x *
                       ff_split_bits((double)r[base + idx]).x * ith;
      const T v = (T)f2d_bits(vf);
      dv[base + idx] = v;
      x[base + idx] = xzero ? v : x[base + idx] + v;
    }
    return;
  }
  const T ith = T(s_ith);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const T v = dinv[base + idx] * r[base + idx] * ith;
    dv[base + idx] = v;
    x[base + idx] = (xzero ? T(0) : x[base + idx]) + v;
  }
}

// step k >= 1: rho_k = 1/(2 sigma - rho_{k-1}); d = rho_k rho_{k-1} d + (2 rho_k / delta) D^{-1} r; x += d
template <typename T>
__global__ void __launch_bounds__(256) cheb_next_kernel(long long N, const T* __restrict__ dinv,
                                                        const double* __restrict__ lmax,
                                                        const T* __restrict__ r, T* __restrict__ x,
                                                        T* __restrict__ dv, int k,
                                                        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ double s_c[2];
  if (threadIdx.x == 0) {
    double th, de;
    cheb_params(lmax[b], th, de);
    const double sigma = th / de;
    double rho_prev = 1.0 / sigma, rho = rho_prev;
    for (int j = 1; j <= k; ++j) {
      rho_prev = rho;
      rho = 1.0 / (2.0 * sigma - rho_prev);
    }
    s_c[0] = rho * rho_prev;
    s_c[1] = 2.0 * rho / de;
  }
  __syncthreads();
  const T c1 = T(s_c[0]), c2 = T(s_c[1]);
  const long long base = (long long)b * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const T v = c1 * dv[base + idx] + c2 * dinv[base + idx] * r[base + idx];
    dv[base + idx] = v;
    x[base + idx] += v;
  }
}

// 1 / diag(A_l) for every solve, written in FP64 and FP32
__global__ void __launch_bounds__(256) dinv_fill_kernel(int d, int m, int P, const double* __restrict__ bands,
                                                        const double* __restrict__ alpha,
                                                        const double* __restrict__ beta,
                                                        double* __restrict__ d64, float* __restrict__ d32) {
  const int b = blockIdx.y;
  long long nper = 1;
  for (int l = 0; l < d; ++l) nper *= m;
  const long long N = d * nper;
  const long long base = (long long)b * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    int comp, I[3];
    decode(d, m, nper, idx, comp, I);
    const double v = dinv_at<double>(d, m, P, bands, comp, I, alpha[b], beta[b]);
    d64[base + idx] = v;
    d32[base + idx] = (float)v;
  }
}

// ------------------------------------------------------------------ power iteration (FP64)
__global__ void hash_init_kernel(long long N, double* v, int level) {
  const int b = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + (unsigned long long)(level + 1) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 31;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 29;
    v[(long long)b * N + i] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0 + 0.05;
  }
}

__global__ void __launch_bounds__(256) jacobi_scale_kernel(long long N, const double* __restrict__ dinv,
                                                           const double* __restrict__ y,
                                                           double* __restrict__ v) {
  const int b = blockIdx.y;
  const long long base = (long long)b * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x)
    v[base + idx] = dinv[base + idx] * y[base + idx];
}

__global__ void norm_step_kernel(int B, const double* part, int nblk, double* lam_out,
                                 double* inv_norm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[(size_t)b * nblk + i];
  const double nrm = sqrt(s);
  if (lam_out) lam_out[b] = nrm;
  inv_norm[b] = nrm > 0 ? 1.0 / nrm : 0.0;
}

__global__ void scale_kernel(long long N, double* v, const double* sc) {
  const int b = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    v[(long long)b * N + i] *= sc[b];
}

// ------------------------------------------------------------------ coarsest solve
template <typename T>
__global__ void __launch_bounds__(256) coarse_solve_kernel(int nc, const T* __restrict__ inv,
                                                           const T* __restrict__ rhs,
                                                           T* __restrict__ x,
                                                           const int* __restrict__ active) {
  // one warp per row of the dense inverse (coalesced row reads), 8 rows per CTA
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int lane = threadIdx.x & 31, i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nc) return;
  const T* Ai = inv + ((size_t)b * nc + i) * nc;
  const T* rb = rhs + (size_t)b * nc;
  T s = 0;
  for (int j = lane; j < nc; j += 32) s += Ai[j] * rb[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[(size_t)b * nc + i] = s;
}

// In-place inverses of SPD matrices by blocked Gauss-Jordan elimination without pivoting (the
// pivots of an SPD matrix, and of its Schur complements, are positive), FP64.  With the index
// set split into the current panel P (kGJW columns) and the rest R, one block step maps
//   A_PP -> A_PP^{-1},  A_PR -> A_PP^{-1} A_PR,  A_RP -> -A_RP A_PP^{-1},
//   A_RR -> A_RR - A_RP A_PP^{-1} A_PR,
// and the steps over all panels in order leave A^{-1}.  The rank-kGJW update of A_RR, all but a
// vanishing part of the n^3 multiply-adds, is spread over 64 x 64 tiles of every matrix, so the
// inverse runs on the whole GPU (on GB300 an SM issues about two FP64 FMAs per clock: one CTA
// per matrix would take tens of milliseconds at n ~ 600).
static constexpr int kGJW = 32;  // panel width
static constexpr int kGJT = 64;  // tile of the update (rows and columns)
static __host__ __device__ size_t gj_ws_per_matrix(int n) { return (size_t)kGJW * kGJW + 2 * (size_t)kGJW * n; }

// Block step, part 1; CTA (slice, matrix): D^{-1} of the panel's diagonal block by Gauss-Jordan
// in shared memory, U = D^{-1} A[P, slice] and the old column panel L = A[slice, P] into the
// side buffer [D^{-1}: W x W | U: W x n | L: n x W] of the matrix.  A pivot that is not
// positive sets *bad (the host then fails the call).
__global__ void __launch_bounds__(256) gj_panel_kernel(int n, int k0, int w,
                                                       const double* __restrict__ mats,
                                                       double* __restrict__ ws,
                                                       int* __restrict__ bad) {
  __shared__ double sD[kGJW][kGJW + 1];
  __shared__ double sA[kGJW][kGJT + 1];
  __shared__ double sCol[kGJW];
  __shared__ double sPiv;
  const int b = blockIdx.y, c0 = blockIdx.x * kGJT;
  const double* a = mats + (size_t)b * n * n;
  double* inv = ws + (size_t)b * gj_ws_per_matrix(n);
  double* U = inv + kGJW * kGJW;
  double* L = U + (size_t)kGJW * n;
  for (int e = threadIdx.x; e < kGJW * kGJW; e += blockDim.x) {
    const int i = e / kGJW, j = e % kGJW;
    sD[i][j] = (i < w && j < w) ? a[(size_t)(k0 + i) * n + k0 + j] : 0.0;
  }
  for (int e = threadIdx.x; e < kGJW * kGJT; e += blockDim.x) {
    const int t = e / kGJT, jj = e % kGJT;
    sA[t][jj] = (t < w && c0 + jj < n) ? a[(size_t)(k0 + t) * n + c0 + jj] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    if (threadIdx.x == 0) {
      double p = sD[k][k];
      if (!(p > 0.0)) {
        atomicExch(bad, 1);
        p = 1.0;
      }
      sPiv = 1.0 / p;
    }
    if (threadIdx.x < kGJW) sCol[threadIdx.x] = sD[threadIdx.x][k];
    __syncthreads();
    const double piv = sPiv;
    if (threadIdx.x < w) sD[k][threadIdx.x] = threadIdx.x == k ? piv : sD[k][threadIdx.x] * piv;
    __syncthreads();
    for (int e = threadIdx.x; e < kGJW * kGJW; e += blockDim.x) {
      const int i = e / kGJW, j = e % kGJW;
      if (i == k || i >= w || j >= w) continue;
      sD[i][j] = j == k ? -sCol[i] * piv : sD[i][j] - sCol[i] * sD[k][j];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0)
    for (int e = threadIdx.x; e < kGJW * kGJW; e += blockDim.x) inv[e] = sD[e / kGJW][e % kGJW];
  for (int e = threadIdx.x; e < kGJW * kGJT; e += blockDim.x) {
    const int t = e / kGJT, jj = e % kGJT;
    if (t >= w || c0 + jj >= n) continue;
    double acc = 0.0;
    for (int q = 0; q < w; ++q) acc = fma(sD[t][q], sA[q][jj], acc);
    U[(size_t)t * n + c0 + jj] = acc;
  }
  for (int e = threadIdx.x; e < kGJT * kGJW; e += blockDim.x) {
    const int ii = e / kGJW, t = e % kGJW;
    if (c0 + ii < n && t < w) L[(size_t)(c0 + ii) * kGJW + t] = a[(size_t)(c0 + ii) * n + k0 + t];
  }
}

// Block step, part 2; CTA (column tile, row tile, matrix): the new values of a 64 x 64 tile,
// a 4 x 4 block of outputs per thread.
__global__ void __launch_bounds__(256) gj_update_kernel(int n, int k0, int w, double* __restrict__ mats,
                                                        const double* __restrict__ ws) {
  __shared__ double sL[kGJT][kGJW + 1];
  __shared__ double sX[kGJW][kGJT + 1];
  const int b = blockIdx.z, I = blockIdx.y * kGJT, J = blockIdx.x * kGJT;
  double* a = mats + (size_t)b * n * n;
  const double* inv = ws + (size_t)b * gj_ws_per_matrix(n);
  const double* U = inv + kGJW * kGJW;
  const double* L = U + (size_t)kGJW * n;
  for (int e = threadIdx.x; e < kGJT * kGJW; e += blockDim.x) {
    const int ii = e / kGJW, t = e % kGJW;
    sL[ii][t] = (I + ii < n && t < w) ? L[(size_t)(I + ii) * kGJW + t] : 0.0;
  }
  for (int e = threadIdx.x; e < kGJW * kGJT; e += blockDim.x) {
    const int t = e / kGJT, jj = e % kGJT, j = J + jj;
    double v = 0.0;
    if (t < w && j < n) v = (j >= k0 && j < k0 + w) ? inv[t * kGJW + (j - k0)] : U[(size_t)t * n + j];
    sX[t][jj] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int t = 0; t < w; ++t) {
    double l[4], x[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) l[r] = sL[ty + 16 * r][t];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = sX[t][tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fma(l[r], x[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = I + ty + 16 * r;
    if (i >= n) continue;
    const bool ip = i >= k0 && i < k0 + w;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = J + tx + 16 * c;
      if (j >= n) continue;
      const bool jp = j >= k0 && j < k0 + w;
      double& y = a[(size_t)i * n + j];
      if (ip)
        y = sX[i - k0][tx + 16 * c];  // D^{-1} or U
      else
        y = jp ? -acc[r][c] : y - acc[r][c];
    }
  }
}

__global__ void __launch_bounds__(256) to_f32_kernel(long long n, const double* __restrict__ src,
                                                     float* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// nmat SPD matrices of order n (contiguous, row-major) inverted in place, the FP32 copies
// written to mats32; *bad (device) is set for a matrix that is not SPD.  ws: nmat *
// gj_ws_per_matrix(n) doubles.
static void gpu_spd_invert(int n, int nmat, double* mats, float* mats32, int* bad, double* ws,
                           cudaStream_t s) {
  const unsigned tiles = (unsigned)((n + kGJT - 1) / kGJT);
  for (int k0 = 0; k0 < n; k0 += kGJW) {
    const int w = std::min(kGJW, n - k0);
    gj_panel_kernel<<<dim3(tiles, nmat), 256, 0, s>>>(n, k0, w, mats, ws, bad);
    gj_update_kernel<<<dim3(tiles, tiles, nmat), 256, 0, s>>>(n, k0, w, mats, ws);
    count_launch(2);
  }
  const long long tot = (long long)nmat * n * n;
  to_f32_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, s>>>(tot, mats, mats32);
  count_launch();
}

// ------------------------------------------------------------------ host side
std::vector<double> dense_operator(int d, const Band& M, const Band& A, const Band& S,
                                   double alpha, double beta) {
  const int m = M.m;
  long long nper = 1;
  for (int l = 0; l < d; ++l) nper *= m;
  const long long n = d * nper;
  std::vector<double> D((size_t)(n * n), 0.0);
  const double gamma = alpha - beta;
  std::vector<int> I(d), J(d);
  for (long long r = 0; r < n; ++r) {
    const int c = (int)(r / nper);
    long long rem = r % nper;
    for (int l = d - 1; l >= 0; --l) {
      I[l] = (int)(rem % m);
      rem /= m;
    }
    for (long long q = 0; q < n; ++q) {
      const int c2 = (int)(q / nper);
      long long rem2 = q % nper;
      for (int l = d - 1; l >= 0; --l) {
        J[l] = (int)(rem2 % m);
        rem2 /= m;
      }
      double v = 0.0;
      if (c == c2) {
        for (int l = 0; l < d; ++l) {
          double t = (l == c) ? beta : alpha;
          for (int k = 0; k < d; ++k) t *= (k == l) ? S.at(I[k], J[k]) : M.at(I[k], J[k]);
          v += t;
        }
      } else {
        double t = gamma;
        for (int k = 0; k < d; ++k) t *= (k == c || k == c2) ? A.at(I[k], J[k]) : M.at(I[k], J[k]);
        v = t;
      }
      D[(size_t)(r * n + q)] = v;
    }
  }
  return D;
}

cd_status mg_build(MgData& mg, int d, int P, const std::vector<int>& ml,
                   const std::vector<Band>& hM, const std::vector<Band>& hA,
                   const std::vector<Band>& hS, int B, int deg, const double* bands64,
                   const float* bands32, const std::vector<size_t>& boff) {
  mg.d = d;
  mg.P = P;
  mg.L = (int)ml.size();
  mg.B = B;
  mg.deg = deg;
  mg.ml = ml;
  mg.boff = boff;
  mg.bands64 = bands64;
  mg.bands32 = bands32;
  mg.hM = hM;
  mg.hA = hA;
  mg.hS = hS;
  mg.Nl.clear();
  for (int m : ml) {
    long long n = d;
    for (int l = 0; l < d; ++l) n *= m;
    mg.Nl.push_back(n);
  }
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    mg.owned.push_back(p);
    return p;
  };
  mg.lv64.assign(mg.L, MgLevelBuf{});
  mg.lv32.assign(mg.L, MgLevelBuf{});
  for (int l = 0; l < mg.L; ++l) {
    const size_t n = (size_t)mg.Nl[l] * B;
    for (int prec = 0; prec < 2; ++prec) {
      const size_t es = prec == 0 ? 8 : 4;
      MgLevelBuf& lb = prec == 0 ? mg.lv64[l] : mg.lv32[l];
      lb.b = alloc(n * es);
      lb.x = alloc(n * es);
      lb.r = alloc(n * es);
      lb.dv = alloc(n * es);
      lb.dinv = alloc(n * es);
      lb.xb = alloc(n * es);
      if (!lb.b || !lb.x || !lb.r || !lb.dv || !lb.dinv || !lb.xb) return CD_ENOMEM;
    }
  }
  mg.nc = (int)mg.Nl.back();
  mg.lmax = (double*)alloc(sizeof(double) * mg.L * B);
  mg.cinv64 = (double*)alloc(sizeof(double) * (size_t)B * mg.nc * mg.nc);
  mg.cinv32 = (float*)alloc(sizeof(float) * (size_t)B * mg.nc * mg.nc);
  mg.part = (double*)alloc(sizeof(double) * (size_t)B * kMaxPartials);
  mg.tmpB = (double*)alloc(sizeof(double) * B);
  if (mg.nc >= 128) {  // side buffer of the GPU inversion of the coarsest matrices
    mg.gjws = (double*)alloc(sizeof(double) * B * gj_ws_per_matrix(mg.nc));
    if (!mg.gjws) return CD_ENOMEM;
  }
  // 3D scratch for levels >= 1 (the finest level uses the handle's scratch)
  if (d == 3 && mg.L > 1) {
    const size_t n3 = (size_t)(mg.Nl[1] / 3) * B;
    mg.scratch64 = alloc(21 * n3 * 8);
    mg.scratch32 = alloc(21 * n3 * 4);
    if (!mg.scratch64 || !mg.scratch32) return CD_ENOMEM;
  }
  if (!mg.lmax || !mg.cinv64 || !mg.cinv32 || !mg.part || !mg.tmpB) return CD_ENOMEM;
  return CD_OK;
}

template <typename T>
static const T* level_bands(const MgData& mg, int l) {
  if (sizeof(T) == 8) return reinterpret_cast<const T*>(mg.bands64 + mg.boff[l]);
  return reinterpret_cast<const T*>(mg.bands32 + mg.boff[l]);
}

template <typename T>
static T* level_scratch(MgData& mg) {
  return (T*)(sizeof(T) == 8 ? mg.scratch64 : mg.scratch32);
}

// The dense coarsest inverses of the listed solves only (a serving session's new slots); the
// others keep theirs.  Same arithmetic as mg_set_params for those solves.
cd_status mg_set_params_slots(MgData& mg, int d, int P, const std::vector<double>& alpha,
                              const std::vector<double>& beta, const std::vector<int>& slots,
                              cudaStream_t s) {
  (void)P;
  const int L = mg.L, nc = mg.nc;
  for (int b : slots) {
    std::vector<double> D = dense_operator(d, mg.hM[L - 1], mg.hA[L - 1], mg.hS[L - 1], alpha[b], beta[b]);
    if (mg.diag_only) {
      const int per = nc / d;
      for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j)
          if (i / per != j / per) D[(size_t)i * nc + j] = 0.0;
    }
    double* dst64 = mg.cinv64 + (size_t)b * nc * nc;
    float* dst32 = mg.cinv32 + (size_t)b * nc * nc;
    if (nc >= 128) {
      CD_CUDA_OK(cudaMemcpyAsync(dst64, D.data(), D.size() * 8, cudaMemcpyHostToDevice, s));
      CD_CUDA_OK(cudaMemsetAsync(mg.tmpB, 0, sizeof(double), s));
      gpu_spd_invert(nc, 1, dst64, dst32, reinterpret_cast<int*>(mg.tmpB), mg.gjws, s);
      int bad = 0;
      CD_CUDA_OK(cudaMemcpyAsync(&bad, mg.tmpB, sizeof(int), cudaMemcpyDeviceToHost, s));
      CD_CUDA_OK(cudaStreamSynchronize(s));  // D goes out of scope
      if (bad) {
        set_error("coarsest multigrid matrix is not SPD");
        return CD_BREAKDOWN;
      }
    } else {
      if (!spd_inverse(nc, D)) {
        set_error("coarsest multigrid matrix is not SPD");
        return CD_BREAKDOWN;
      }
      std::vector<float> D32(D.begin(), D.end());
      CD_CUDA_OK(cudaMemcpyAsync(dst64, D.data(), D.size() * 8, cudaMemcpyHostToDevice, s));
      CD_CUDA_OK(cudaMemcpyAsync(dst32, D32.data(), D32.size() * 4, cudaMemcpyHostToDevice, s));
      CD_CUDA_OK(cudaStreamSynchronize(s));
    }
  }
  return CD_OK;
}

cd_status mg_set_params(MgData& mg, int d, int P, int nrhs, const std::vector<double>& alpha,
                        const std::vector<double>& beta, cudaStream_t s) {
  // coarsest dense inverses (host, FP64)
  const int L = mg.L, nc = mg.nc;
  std::vector<double> inv64((size_t)nrhs * nc * nc);
  std::vector<float> inv32(inv64.size());
  std::vector<char> ok(nrhs, 1);
  if (nc >= 128) {  // large coarsest level: the matrices go up, the GPU inverts them
    for (int b = 0; b < nrhs; ++b) {
      std::vector<double> D = dense_operator(d, mg.hM[L - 1], mg.hA[L - 1], mg.hS[L - 1], alpha[b], beta[b]);
      if (mg.diag_only) {
        const int per = nc / d;
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j)
            if (i / per != j / per) D[(size_t)i * nc + j] = 0.0;
      }
      std::copy(D.begin(), D.end(), inv64.begin() + (size_t)b * nc * nc);
    }
    CD_CUDA_OK(cudaMemcpyAsync(mg.cinv64, inv64.data(), inv64.size() * 8, cudaMemcpyHostToDevice, s));
    CD_CUDA_OK(cudaMemsetAsync(mg.tmpB, 0, sizeof(double), s));
    gpu_spd_invert(nc, nrhs, mg.cinv64, mg.cinv32, reinterpret_cast<int*>(mg.tmpB), mg.gjws, s);
    int bad = 0;
    CD_CUDA_OK(cudaMemcpyAsync(&bad, mg.tmpB, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA_OK(cudaStreamSynchronize(s));  // inv64 (host) goes out of scope
    if (bad) {
      set_error("coarsest multigrid matrix is not SPD");
      return CD_BREAKDOWN;
    }
    return CD_OK;
  }
  auto one = [&](int b) {
    std::vector<double> D = dense_operator(d, mg.hM[L - 1], mg.hA[L - 1], mg.hS[L - 1], alpha[b], beta[b]);
    if (mg.diag_only) {  // keep the diagonal blocks of the component-major ordering
      const int per = nc / d;
      for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j)
          if (i / per != j / per) D[(size_t)i * nc + j] = 0.0;
    }
    if (!spd_inverse(nc, D)) {
      ok[b] = 0;
      return;
    }
    std::copy(D.begin(), D.end(), inv64.begin() + (size_t)b * nc * nc);
  };
  // one solve's inverse per host thread when the coarsest level is large (each is O(nc^3))
  const int nth = nc >= 128 ? std::min(nrhs, std::max(1, (int)std::thread::hardware_concurrency())) : 1;
  if (nth > 1) {
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t] {
        for (int b = t; b < nrhs; b += nth) one(b);
      });
    for (auto& x : th) x.join();
  } else {
    for (int b = 0; b < nrhs; ++b) one(b);
  }
  for (int b = 0; b < nrhs; ++b)
    if (!ok[b]) {
      set_error("coarsest multigrid matrix is not SPD");
      return CD_BREAKDOWN;
    }
  for (size_t i = 0; i < inv64.size(); ++i) inv32[i] = (float)inv64[i];
  CD_CUDA_OK(cudaMemcpyAsync(mg.cinv64, inv64.data(), inv64.size() * 8, cudaMemcpyHostToDevice, s));
  CD_CUDA_OK(cudaMemcpyAsync(mg.cinv32, inv32.data(), inv32.size() * 4, cudaMemcpyHostToDevice, s));
  CD_CUDA_OK(cudaStreamSynchronize(s));  // host vectors go out of scope
  return CD_OK;
}

// Power iteration for lambda_max(D^{-1} A_l) on every smoothed level (FP64), per solve.
static void mg_power(MgData& mg, int B, Coef c, double* fine_scratch64, cudaStream_t s) {
  for (int l = 0; l + 1 < mg.L; ++l) {
    const int m = mg.ml[l];
    const long long N = mg.Nl[l];
    double* v = (double*)mg.lv64[l].x;
    double* y = (double*)mg.lv64[l].r;
    const dim3 g = grid_for(N, B);
    hash_init_kernel<<<g, 256, 0, s>>>(N, v, l);
    const int nb = partial_blocks(N);
    launch_dot<double>(v, v, N, B, mg.part, nb, nullptr, s);
    norm_step_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mg.part, nb, nullptr, mg.tmpB);
    scale_kernel<<<g, 256, 0, s>>>(N, v, mg.tmpB);
    count_launch(3);
    double* scr = l == 0 ? fine_scratch64 : (double*)mg.scratch64;
    dinv_fill_kernel<<<g, 256, 0, s>>>(mg.d, m, mg.P, level_bands<double>(mg, l), c.alpha, c.beta,
                                       (double*)mg.lv64[l].dinv, (float*)mg.lv32[l].dinv);
    count_launch();
    for (int it = 0; it < kPowerIts; ++it) {
      launch_apply<double>(mg.d, m, mg.P, level_bands<double>(mg, l), v, y, nullptr, 0, B, c,
                           nullptr, nullptr, nullptr, scr, s);
      jacobi_scale_kernel<<<g, 256, 0, s>>>(N, (const double*)mg.lv64[l].dinv, y, v);
      launch_dot<double>(v, v, N, B, mg.part, nb, nullptr, s);
      norm_step_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mg.part, nb, mg.lmax + (size_t)l * mg.B,
                                                       mg.tmpB);
      scale_kernel<<<g, 256, 0, s>>>(N, v, mg.tmpB);
      count_launch(3);
    }
  }
}

cd_status mg_prepare(MgData& mg, int B, Coef c, double* fine_scratch64, cudaStream_t s) {
  if (mg.diag_only) c.gsc = mg.gsc_zero;
  mg_power(mg, B, c, fine_scratch64, s);
  CD_CUDA_OK(cudaGetLastError());
  return CD_OK;
}

template <typename T>
static void smooth(MgData& mg, int l, int B, const T* bl, T* xl, bool xzero, Coef c,
                   const int* active, T* scr, cudaStream_t s) {
  const int m = mg.ml[l];
  const long long N = mg.Nl[l];
  MgLevelBuf& lb = sizeof(T) == 8 ? mg.lv64[l] : mg.lv32[l];
  T* r = (T*)lb.r;
  T* dv = (T*)lb.dv;
  const T* bands = level_bands<T>(mg, l);
  const double* lm = mg.lmax + (size_t)l * mg.B;
  const dim3 g = grid_for(N, B);
  const T* rsrc = bl;
  if (!xzero) {
    launch_apply<T>(mg.d, m, mg.P, bands, xl, r, bl, 1, B, c, nullptr, nullptr, active, scr, s);
    rsrc = r;
  }
  const T* dinv = (const T*)lb.dinv;
  cheb_first_kernel<T><<<g, 256, 0, s>>>(N, dinv, lm, rsrc, xl, dv, xzero ? 1 : 0, active,
                                         fp64_emulated());
  count_launch();
  for (int k = 1; k < mg.deg; ++k) {
    launch_apply<T>(mg.d, m, mg.P, bands, dv, r, rsrc, 1, B, c, nullptr, nullptr, active, scr, s);
    rsrc = r;
    cheb_next_kernel<T><<<g, 256, 0, s>>>(N, dinv, lm, r, xl, dv, k, active);
    count_launch();
  }
}

// Degree-2 Chebyshev smoothing with the second step fused into the apply (mode 2).
// Pre-smoothing from x = 0: X0 = D^{-1} b / theta (= d1), then XB = X0 + d2 with
// d2 = c1 d1 + c2 D^{-1} (b - A X0).  Post-smoothing from XB: X0 = XB + d1 with
// d1 = D^{-1} (b - A XB) / theta (d1 -> dv, r0 -> r), then X0 += c1 d1 + c2 D^{-1} (r0 - A d1).
template <typename T>
static void smooth_pre_fused(MgData& mg, int l, int B, const T* bl, T* X0, T* XB, Coef c,
                             const int* active, T* scr, cudaStream_t s) {
  const int m = mg.ml[l];
  const long long N = mg.Nl[l];
  MgLevelBuf& lb = sizeof(T) == 8 ? mg.lv64[l] : mg.lv32[l];
  const double* lm = mg.lmax + (size_t)l * mg.B;
  cheb_first_kernel<T><<<grid_for(N, B), 256, 0, s>>>(N, (const T*)lb.dinv, lm, bl, X0, (T*)lb.dv, 1,
                                                      active, fp64_emulated());
  count_launch();
  Epi<T> e{X0, X0, XB, nullptr, nullptr, lm, 1, (const T*)lb.dinv};
  launch_apply<T>(mg.d, m, mg.P, level_bands<T>(mg, l), X0, nullptr, bl, 2, B, c, nullptr, nullptr,
                  active, scr, s, &e);
}

template <typename T>
static void smooth_post_fused(MgData& mg, int l, int B, const T* bl, const T* XB, T* X0, Coef c,
                              const int* active, T* scr, cudaStream_t s) {
  const int m = mg.ml[l];
  MgLevelBuf& lb = sizeof(T) == 8 ? mg.lv64[l] : mg.lv32[l];
  const double* lm = mg.lmax + (size_t)l * mg.B;
  const T* bands = level_bands<T>(mg, l);
  Epi<T> e0{nullptr, XB, X0, (T*)lb.dv, (T*)lb.r, lm, 0, (const T*)lb.dinv};
  launch_apply<T>(mg.d, m, mg.P, bands, XB, nullptr, bl, 2, B, c, nullptr, nullptr, active, scr, s,
                  &e0);
  Epi<T> e1{(const T*)lb.dv, X0, X0, nullptr, nullptr, lm, 1, (const T*)lb.dinv};
  launch_apply<T>(mg.d, m, mg.P, bands, (const T*)lb.dv, nullptr, (const T*)lb.r, 2, B, c, nullptr,
                  nullptr, active, scr, s, &e1);
}

template <typename T>
static void vcycle_rec(MgData& mg, int l, int B, const T* bl, T* xl, Coef c, const int* active,
                       T* fine_scr, cudaStream_t s, int post) {
  T* scr = l == 0 ? fine_scr : level_scratch<T>(mg);
  if (l == mg.L - 1) {
    coarse_solve_kernel<T><<<dim3((mg.nc + 7) / 8, B), 256, 0, s>>>(
        mg.nc, sizeof(T) == 8 ? (const T*)mg.cinv64 : (const T*)mg.cinv32, bl, xl, active);
    count_launch();
    return;
  }
  MgLevelBuf& lb = sizeof(T) == 8 ? mg.lv64[l] : mg.lv32[l];
  MgLevelBuf& nb = sizeof(T) == 8 ? mg.lv64[l + 1] : mg.lv32[l + 1];
  const bool fused = mg.deg == 2 && apply_can_fuse<T>(mg.d, mg.ml[l], mg.P, level_bands<T>(mg, l), B);
  T* cur = xl;  // buffer holding the level's iterate after pre-smoothing
  if (fused) {
    smooth_pre_fused<T>(mg, l, B, bl, xl, (T*)lb.xb, c, active, scr, s);
    cur = (T*)lb.xb;
  } else {
    smooth<T>(mg, l, B, bl, xl, true, c, active, scr, s);
  }
  launch_apply<T>(mg.d, mg.ml[l], mg.P, level_bands<T>(mg, l), cur, (T*)lb.r, bl, 1, B, c, nullptr,
                  nullptr, active, scr, s);
  mg_restrict<T>(mg.d, mg.ml[l], mg.ml[l + 1], B, (const T*)lb.r, (T*)nb.b, active, s);
  vcycle_rec<T>(mg, l + 1, B, (const T*)nb.b, (T*)nb.x, c, active, fine_scr, s, kPostCheb);
  mg_prolong_add<T>(mg.d, mg.ml[l], mg.ml[l + 1], B, (const T*)nb.x, cur, active, s);
  if (l == 0 && post == kPostPgmres) {
    ks_pgmres<T>(mg, B, bl, cur, xl, c, active, scr, s);
  } else if (l == 0 && post == kPostPcg) {
    ks_pcg<T>(mg, B, bl, cur, xl, c, active, scr, s);
  } else if (fused) {
    smooth_post_fused<T>(mg, l, B, bl, cur, xl, c, active, scr, s);
  } else {
    smooth<T>(mg, l, B, bl, xl, false, c, active, scr, s);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) add_kernel(long long N, T* __restrict__ z,
                                                  const T* __restrict__ e,
                                                  const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    z[base + i] += e[base + i];
}

template <typename T>
void mg_vcycle(MgData& mg, int d, int P, int B, const T* r, T* z, Coef c, const int* active,
               cudaStream_t s, T* fine_scr, int post, int cycles) {
  (void)d;
  (void)P;
  if (mg.diag_only) c.gsc = mg.gsc_zero;
  if (post != kPostCheb && mg.ks_steps < 1) post = kPostCheb;
  vcycle_rec<T>(mg, 0, B, r, z, c, active, fine_scr, s, post);
  if (cycles < 2) return;
  const long long N = mg.Nl[0];
  T* rc = (T*)(sizeof(T) == 8 ? mg.cyc64 : mg.cyc32);
  T* e = rc + N * (long long)mg.B;
  for (int k = 1; k < cycles; ++k) {
    launch_apply<T>(mg.d, mg.ml[0], mg.P, level_bands<T>(mg, 0), z, rc, r, 1, B, c, nullptr,
                    nullptr, active, fine_scr, s);
    vcycle_rec<T>(mg, 0, B, rc, e, c, active, fine_scr, s, post);
    add_kernel<T><<<grid_for(N, B), 256, 0, s>>>(N, z, e, active);
    count_launch();
  }
}

cd_status mg_setup_ksmooth(MgData& mg, int steps, const void* Lb64, const void* dinv64,
                           const void* Lb32, const void* dinv32) {
  if (steps < 1 || steps > 7) {
    set_error("Krylov post-smoother: 1 <= steps <= 7");
    return CD_EINVAL;
  }
  mg.tLb64 = Lb64;
  mg.tdinv64 = dinv64;
  mg.tLb32 = Lb32;
  mg.tdinv32 = dinv32;
  if (mg.ks_steps >= steps) return CD_OK;
  const size_t n = (size_t)mg.Nl[0] * mg.B;
  const size_t nv = 2 * (size_t)steps + 2;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    mg.owned.push_back(p);
    return p;
  };
  mg.ks64 = alloc(nv * n * 8);
  mg.ks32 = alloc(nv * n * 4);
  if (!mg.cyc64) {
    mg.cyc64 = alloc(2 * n * 8);
    mg.cyc32 = alloc(2 * n * 4);
  }
  const size_t B = mg.B;
  mg.ks_H = (double*)alloc(8 * B * (steps + 1) * steps);
  mg.ks_hc = (double*)alloc(8 * B * 8);
  mg.ks_y = (double*)alloc(8 * B * 8);
  mg.ks_inv = (double*)alloc(8 * B);
  mg.ks_beta0 = (double*)alloc(8 * B);
  mg.ks_rz = (double*)alloc(8 * B);
  mg.ks_a = (double*)alloc(8 * B);
  mg.ks_b = (double*)alloc(8 * B);
  mg.ks_part = (double*)alloc(8 * B * 8 * 256);
  if (!mg.ks64 || !mg.ks32 || !mg.cyc64 || !mg.cyc32 || !mg.ks_H || !mg.ks_hc || !mg.ks_y ||
      !mg.ks_inv || !mg.ks_beta0 || !mg.ks_rz || !mg.ks_a || !mg.ks_b || !mg.ks_part) {
    cudaGetLastError();
    set_error("Krylov post-smoother: workspace allocation failed");
    return CD_ENOMEM;
  }
  mg.ks_steps = steps;
  return CD_OK;
}

cd_status mg_set_block_diagonal(MgData& mg) {
  if (!mg.gsc_zero) {
    void* p = nullptr;
    if (cudaMalloc(&p, 8 * (size_t)std::max(1, mg.B)) != cudaSuccess) {
      cudaGetLastError();
      return CD_ENOMEM;
    }
    mg.owned.push_back(p);
    CD_CUDA_OK(cudaMemset(p, 0, 8 * (size_t)std::max(1, mg.B)));
    mg.gsc_zero = (double*)p;
  }
  mg.diag_only = true;
  return CD_OK;
}

template void mg_vcycle<double>(MgData&, int, int, int, const double*, double*, Coef, const int*,
                                cudaStream_t, double*, int, int);
template void mg_vcycle<float>(MgData&, int, int, int, const float*, float*, Coef, const int*,
                               cudaStream_t, float*, int, int);

}  // namespace cd
