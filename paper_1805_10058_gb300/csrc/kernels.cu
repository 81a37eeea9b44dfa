// CUDA kernels (sm_103a) of the curl-div solve loop.
//
// Layout of a batch of vectors: [B][d][m]^d, x_d fastest (component-major, Kronecker
// order).  1D bands: [3][m][2P+1] = (M, A, S), row i holding X(i, i-P .. i+P).
// Per-solve operator coefficients alpha[b], beta[b] (FP64); gamma = alpha - beta.
//
// The block operator is applied in the form (A^T = -A turns every off-diagonal
// Kronecker term of eq:matr_Amu / eq:matr_Amu3D into gamma A(x)A(x)...):
//   d = 2:  y1 = alpha M(x)S w1 + beta S(x)M w1 + gamma A(x)A w2
//           y2 = gamma A(x)A w1 + alpha S(x)M w2 + beta M(x)S w2
//   d = 3:  y1 = [alpha (MMS + MSM) + beta SMM] w1 + gamma AAM w2 + gamma AMA w3
//           y2 = gamma AAM w1 + [alpha (SMM + MMS) + beta MSM] w2 + gamma MAA w3
//           y3 = gamma AMA w1 + gamma MAA w2 + [alpha (SMM + MSM) + beta MMS] w3
// (X1 X2 X3 = X1 (x) X2 (x) X3, X1 acting along x_1.)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <unordered_map>

#include "cd_internal.h"
#include "apply_shared.h"
#include "ffmath.h"

namespace cd {

static std::atomic<int> g_use_stream3d{1};  // 3D: 1 = streaming fused kernel, 0 = three banded passes

// ------------------------------------------------------------------ helpers


// 1 / (x * y * z + u * v * t) rounded step by step (no contraction), shared by every 2D kernel's
// fused smoother epilogue so that all of them produce the same bits.
__device__ __forceinline__ float inv_diag2(float x, float y, float z, float u, float v, float t) {
  return __fdiv_rn(1.0f, __fadd_rn(__fmul_rn(__fmul_rn(x, y), z), __fmul_rn(__fmul_rn(u, v), t)));
}
__device__ __forceinline__ double inv_diag2(double x, double y, double z, double u, double v,
                                            double t) {
  return __ddiv_rn(1.0, __dadd_rn(__dmul_rn(__dmul_rn(x, y), z), __dmul_rn(__dmul_rn(u, v), t)));
}

// 1 / (diagonal entry of block c of the 3D operator) at a grid point whose 1D mass and
// stiffness diagonals along the three axes are Md, Sd:
//   sum_l (l == c ? beta : alpha) prod_k (k == l ? Sd[k] : Md[k]),
// in the kernel's arithmetic type (FP32 kernels stay off the FP64 pipe).
template <typename T>
__device__ __forceinline__ T inv_diag3(T al, T be, int c, const T* Md, const T* Sd) {
  T diag = T(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    T t = (l == c) ? be : al;
#pragma unroll
    for (int k = 0; k < 3; ++k) t *= (k == l) ? Sd[k] : Md[k];
    diag += t;
  }
  return T(1) / diag;
}

// ------------------------------------------------------------------ 2D fused apply
// One CTA: TR output rows (axis x_1) of one solve, all m columns (axis x_2), both
// components.  Shared memory: bands [3][m][W], input rows [2][TR+2P][m] (zero outside
// the domain), intermediates [6][TR][m].
template <typename T>
__global__ void __launch_bounds__(256) apply2d_kernel(int m, int P, int TR,
                                                      const T* __restrict__ bands,
                                                      const T* __restrict__ w, T* __restrict__ y,
                                                      const T* __restrict__ rhs, int mode,
                                                      const double* __restrict__ alpha,
                                                      const double* __restrict__ beta, const double* __restrict__ gsc,
                                                      const int* __restrict__ active,
                                                      double* __restrict__ dotp) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sb = reinterpret_cast<T*>(smem_raw);
  const int W = 2 * P + 1;
  const int HR = TR + 2 * P;
  T* sw = sb + 3 * m * W;
  T* su = sw + 2 * HR * m;
  const long long N = 2LL * m * m;
  const long long base = (long long)b * N;
  const int r0 = blockIdx.x * TR;
  const int nt = blockDim.x;
  for (int idx = threadIdx.x; idx < 3 * m * W; idx += nt) sb[idx] = bands[idx];
  for (int idx = threadIdx.x; idx < 2 * HR * m; idx += nt) {
    const int c = idx / (HR * m), rem = idx - c * HR * m;
    const int rr = rem / m, j = rem - rr * m;
    const int row = r0 - P + rr;
    sw[idx] = (row >= 0 && row < m) ? w[base + (long long)c * m * m + (long long)row * m + j] : T(0);
  }
  __syncthreads();
  const T a = T(alpha[b]), be = T(beta[b]), g = T((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  const T* Mb = sb;
  const T* Ab = sb + m * W;
  const T* Sb = sb + 2 * m * W;
  const int rows = min(TR, m - r0);
  // axis x_1 (slow): u = X w along rows, six intermediates premultiplied by their weights
  for (int idx = threadIdx.x; idx < rows * m; idx += nt) {
    const int r = idx / m, j = idx - r * m;
    const int i = r0 + r;
    T uM1 = 0, uS1 = 0, uA1 = 0, uM2 = 0, uS2 = 0, uA2 = 0;
    const T* s1 = sw + (size_t)r * m + j;
    const T* s2 = sw + (size_t)(HR + r) * m + j;
    for (int k = 0; k < W; ++k) {
      const T mk = Mb[i * W + k], ak = Ab[i * W + k], sk = Sb[i * W + k];
      const T v1 = s1[(size_t)k * m], v2 = s2[(size_t)k * m];
      uM1 += mk * v1; uS1 += sk * v1; uA1 += ak * v1;
      uM2 += mk * v2; uS2 += sk * v2; uA2 += ak * v2;
    }
    const size_t o = (size_t)r * m + j, st = (size_t)TR * m;
    su[0 * st + o] = a * uM1;   // -> S along x_2 for y1
    su[1 * st + o] = be * uS1;  // -> M along x_2 for y1
    su[2 * st + o] = g * uA2;   // -> A along x_2 for y1
    su[3 * st + o] = g * uA1;   // -> A along x_2 for y2
    su[4 * st + o] = a * uS2;   // -> M along x_2 for y2
    su[5 * st + o] = be * uM2;  // -> S along x_2 for y2
  }
  __syncthreads();
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < rows * m; idx += nt) {
    const int r = idx / m, j = idx - r * m;
    const int i = r0 + r;
    T y1 = 0, y2 = 0;
    const size_t st = (size_t)TR * m;
    const T* u = su + (size_t)r * m;
    const int k0 = max(0, P - j), k1 = min(W - 1, m - 1 - j + P);
    for (int k = k0; k <= k1; ++k) {
      const int q = j + k - P;
      const T mk = Mb[j * W + k], ak = Ab[j * W + k], sk = Sb[j * W + k];
      y1 += sk * u[0 * st + q] + mk * u[1 * st + q] + ak * u[2 * st + q];
      y2 += ak * u[3 * st + q] + mk * u[4 * st + q] + sk * u[5 * st + q];
    }
    const long long o1 = base + (long long)i * m + j, o2 = o1 + (long long)m * m;
    if (mode == 1) {
      y1 = rhs[o1] - y1;
      y2 = rhs[o2] - y2;
      if (dotp) acc += (double)y1 * (double)y1 + (double)y2 * (double)y2;
    } else if (dotp) {
      acc += (double)sw[(size_t)(r + P) * m + j] * (double)y1 +
             (double)sw[(size_t)(HR + r + P) * m + j] * (double)y2;
    }
    y[o1] = y1;
    y[o2] = y2;
  }
  if (dotp) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) dotp[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------ 2D fused apply, v2
// Rows lo..hi-1 of M, A and S equal the central Toeplitz stencil (Section 3.2: the central
// entries are cardinal-spline values), which arrives as a kernel parameter (constant bank,
// read straight into the FMAs); the ~2p boundary rows read the k-major band copy
// bandT[X][k][i].  Phase A (axis x_1): each thread owns a column and keeps its TR + 2P
// input rows in registers.  Phase B (axis x_2): each thread produces 4 consecutive
// outputs from a register window over zero-padded shared-memory rows.
template <typename T>
struct Stencil {
  T c[3][13];  // M, A, S central rows (k = 0..2P)
  int lo, hi;  // rows [lo, hi) are Toeplitz
};

template <typename T, int P, int TR>
__global__ void __launch_bounds__(256, 2) apply2d_v2_kernel(
    int m, const T* __restrict__ bandT, Stencil<T> cs, const T* __restrict__ w,
    T* __restrict__ y, const T* __restrict__ rhs, int mode, const double* __restrict__ alpha,
    const double* __restrict__ beta, const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<T> epi) {
  constexpr int W = 2 * P + 1;
  constexpr int NC = sizeof(T) == 8 ? 2 : 4;  // outputs per thread along x_2
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  const int ld = m + 2 * P;
  const long long N = 2LL * m * m;
  const T* w1 = w + (long long)b * N;
  const T* w2 = w1 + (long long)m * m;
  const int r0 = blockIdx.x * TR;
  const int rows = min(TR, m - r0);
  const T a = T(alpha[b]), be = T(beta[b]), g = T((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  const T* BM = bandT;
  const T* BA = bandT + (size_t)W * m;
  const T* BS = bandT + (size_t)2 * W * m;
  const size_t plane = (size_t)TR * ld;
  // ---- phase A: axis x_1
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    T in1[TR + 2 * P], in2[TR + 2 * P];
#pragma unroll
    for (int q = 0; q < TR + 2 * P; ++q) {
      const int row = r0 - P + q;
      const bool ok = row >= 0 && row < m;
      in1[q] = ok ? w1[(long long)row * m + j] : T(0);
      in2[q] = ok ? w2[(long long)row * m + j] : T(0);
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      if (r < rows) {
        const int i = r0 + r;
        T uM1 = 0, uS1 = 0, uA1 = 0, uM2 = 0, uS2 = 0, uA2 = 0;
        if (i >= cs.lo && i < cs.hi) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const T v1 = in1[r + k], v2 = in2[r + k];
            uM1 += cs.c[0][k] * v1; uA1 += cs.c[1][k] * v1; uS1 += cs.c[2][k] * v1;
            uM2 += cs.c[0][k] * v2; uA2 += cs.c[1][k] * v2; uS2 += cs.c[2][k] * v2;
          }
        } else {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const T mk = BM[(size_t)k * m + i], ak = BA[(size_t)k * m + i], sk = BS[(size_t)k * m + i];
            const T v1 = in1[r + k], v2 = in2[r + k];
            uM1 += mk * v1; uA1 += ak * v1; uS1 += sk * v1;
            uM2 += mk * v2; uA2 += ak * v2; uS2 += sk * v2;
          }
        }
        const size_t o = (size_t)r * ld + j + P;
        su[0 * plane + o] = a * uM1;   // -> S along x_2 for y1
        su[1 * plane + o] = be * uS1;  // -> M along x_2 for y1
        su[2 * plane + o] = g * uA2;   // -> A along x_2 for y1
        su[3 * plane + o] = g * uA1;   // -> A along x_2 for y2
        su[4 * plane + o] = a * uS2;   // -> M along x_2 for y2
        su[5 * plane + o] = be * uM2;  // -> S along x_2 for y2
      }
    }
  }
  for (int idx = threadIdx.x; idx < 6 * TR * 2 * P; idx += blockDim.x) {
    const int c = idx / (TR * 2 * P), rem = idx - c * TR * 2 * P;
    const int r = rem / (2 * P), pc = rem - r * 2 * P;
    su[c * plane + (size_t)r * ld + (pc < P ? pc : m + pc)] = T(0);
  }
  __syncthreads();
  // ---- phase B: axis x_2
  const int nc4 = (m + NC - 1) / NC;
  double acc = 0.0;
  T ec1 = 0, ec2 = 0;
  if (mode == 2) {
    double c1, c2;
    cheb_coef_cta(epi.lmax[b], epi.step, c1, c2);
    ec1 = T(c1);
    ec2 = T(c2);
  }
  for (int idx = threadIdx.x; idx < rows * nc4; idx += blockDim.x) {
    const int r = idx / nc4, j0 = (idx - r * nc4) * NC;
    const int i = r0 + r;
    T s[6][NC + 2 * P];
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int t = 0; t < NC + 2 * P; ++t) s[c][t] = su[c * plane + (size_t)r * ld + j0 + t];
    const long long o1 = (long long)b * N + (long long)i * m;
    const long long o2 = o1 + (long long)m * m;
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      const int jj = j0 + u;
      if (jj >= m) break;
      T y1 = 0, y2 = 0;
      if (jj >= cs.lo && jj < cs.hi) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          y1 += cs.c[2][k] * s[0][u + k] + cs.c[0][k] * s[1][u + k] + cs.c[1][k] * s[2][u + k];
          y2 += cs.c[1][k] * s[3][u + k] + cs.c[0][k] * s[4][u + k] + cs.c[2][k] * s[5][u + k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const T mk = BM[(size_t)k * m + jj], ak = BA[(size_t)k * m + jj], sk = BS[(size_t)k * m + jj];
          y1 += sk * s[0][u + k] + mk * s[1][u + k] + ak * s[2][u + k];
          y2 += ak * s[3][u + k] + mk * s[4][u + k] + sk * s[5][u + k];
        }
      }
      if (mode == 2) {
        const T Mi = BM[(size_t)P * m + i], Si = BS[(size_t)P * m + i];
        const T Mj = BM[(size_t)P * m + jj], Sj = BS[(size_t)P * m + jj];
        cheb_epi(epi, o1 + jj, rhs[o1 + jj] - y1, inv_diag2(be, Si, Mj, a, Mi, Sj), ec1, ec2);
        cheb_epi(epi, o2 + jj, rhs[o2 + jj] - y2, inv_diag2(a, Si, Mj, be, Mi, Sj), ec1, ec2);
        continue;
      }
      if (mode == 1) {
        y1 = rhs[o1 + jj] - y1;
        y2 = rhs[o2 + jj] - y2;
        if (dotp) acc += (double)y1 * (double)y1 + (double)y2 * (double)y2;
      } else if (dotp) {
        acc += (double)w1[(long long)i * m + jj] * (double)y1 + (double)w2[(long long)i * m + jj] * (double)y2;
      }
      y[o1 + jj] = y1;
      y[o2 + jj] = y2;
    }
  }
  if (dotp) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0) dotp[(size_t)b * gridDim.x + blockIdx.x] = sum;
  }
}

// ------------------------------------------------------------------ 2D fused apply, v3
// Axis x_2 first, straight from global memory: each thread computes 4 consecutive columns of
// one input row for both components at once (packed pairs (w1, w2): one FFMA2 per tap on
// FP32).  The results, grouped by the x_1 operator they feed,
//   PM = (alpha S2 w1, beta S2 w2), PS = (beta M2 w1, alpha M2 w2), PA = gamma (A2 w2, A2 w1),
// go to shared memory; then each thread owns one column and applies M1, S1, A1 along x_1 from
// a register window, producing (y1, y2) = M1 PM + S1 PS + A1 PA with one FFMA2 per tap.
// Tile: TR rows x 64 columns, TR + 2P rows of intermediates (halo rows recomputed).
template <typename T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
__device__ __forceinline__ float2 pfma(float a, float2 x, float2 acc) {
  return __ffma2_rn(make_float2(a, a), x, acc);
}
__device__ __forceinline__ double2 pfma(double a, double2 x, double2 acc) {
  return make_double2(fma(a, x.x, acc.x), fma(a, x.y, acc.y));
}
template <typename T2, typename T>
__device__ __forceinline__ T2 mk2(T a, T b) {
  T2 r;
  r.x = a;
  r.y = b;
  return r;
}

template <typename T, int P, int TR>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) apply2d_v3_kernel(
    int m, const T* __restrict__ bandT, Stencil<T> cs, const T* __restrict__ w,
    T* __restrict__ y, const T* __restrict__ rhs, int mode, const double* __restrict__ alpha,
    const double* __restrict__ beta, const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<T> epi) {
  using T2 = typename Pair<T>::type;
  constexpr int W = 2 * P + 1;
  constexpr int NC = 4, TC = 64, CG = TC / NC;  // 128 threads: phase A 3 rounds, phase B 1
  constexpr int HR = TR + 2 * P;
  constexpr int RS = TR / 2;  // rows per thread in the x_1 pass (two row segments)
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* sp = reinterpret_cast<T2*>(smem_raw);  // [3][HR][TC]
  const long long N = 2LL * m * m;
  const T* w1 = w + (long long)b * N;
  const T* w2 = w1 + (long long)m * m;
  const int c0 = blockIdx.x * TC, r0 = blockIdx.y * TR;
  const int rows = min(TR, m - r0), cols = min(TC, m - c0);
  const T al = T(alpha[b]), be = T(beta[b]), ga = T((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  const T* BM = bandT;
  const T* BA = bandT + (size_t)W * m;
  const T* BS = bandT + (size_t)2 * W * m;
  // ---- phase A: axis x_2 for rows r0-P .. r0+TR+P-1
  for (int item = threadIdx.x; item < HR * CG; item += blockDim.x) {
    const int q = item / CG, g = item - q * CG;
    const int row = r0 - P + q;
    const int j0 = c0 + g * NC;
    T2 tM[NC], tS[NC], tA[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) tM[u] = tS[u] = tA[u] = mk2<T2>(T(0), T(0));
    if (row >= 0 && row < m && j0 < m) {
      T2 win[NC + 2 * P];
      const T* a1 = w1 + (long long)row * m;
      const T* a2 = w2 + (long long)row * m;
#pragma unroll
      for (int t = 0; t < NC + 2 * P; ++t) {
        const int jj = j0 - P + t;
        const bool ok = jj >= 0 && jj < m;
        win[t] = mk2<T2>(ok ? a1[jj] : T(0), ok ? a2[jj] : T(0));
      }
      const bool interior = j0 >= cs.lo && j0 + NC - 1 < cs.hi;
      if (interior) {
#pragma unroll
        for (int u = 0; u < NC; ++u)
#pragma unroll
          for (int k = 0; k < W; ++k) {
            tM[u] = pfma(cs.c[0][k], win[u + k], tM[u]);
            tA[u] = pfma(cs.c[1][k], win[u + k], tA[u]);
            tS[u] = pfma(cs.c[2][k], win[u + k], tS[u]);
          }
      } else {
#pragma unroll
        for (int u = 0; u < NC; ++u) {
          const int j = j0 + u;
          if (j < m) {
#pragma unroll
            for (int k = 0; k < W; ++k) {
              tM[u] = pfma(BM[(size_t)k * m + j], win[u + k], tM[u]);
              tA[u] = pfma(BA[(size_t)k * m + j], win[u + k], tA[u]);
              tS[u] = pfma(BS[(size_t)k * m + j], win[u + k], tS[u]);
            }
          }
        }
      }
    }
    T2* pM = sp + (size_t)(0 * HR + q) * TC + g * NC;
    T2* pS = sp + (size_t)(1 * HR + q) * TC + g * NC;
    T2* pA = sp + (size_t)(2 * HR + q) * TC + g * NC;
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      pM[u] = mk2<T2>(al * tS[u].x, be * tS[u].y);  // feeds M along x_1
      pS[u] = mk2<T2>(be * tM[u].x, al * tM[u].y);  // feeds S along x_1
      pA[u] = mk2<T2>(ga * tA[u].y, ga * tA[u].x);  // feeds A along x_1
    }
  }
  __syncthreads();
  // ---- phase B: axis x_1, one column and RS rows per item
  double acc = 0.0;
  T ec1 = 0, ec2 = 0;
  if (mode == 2) {
    double c1, c2;
    cheb_coef_cta(epi.lmax[b], epi.step, c1, c2);
    ec1 = T(c1);
    ec2 = T(c2);
  }
  for (int item = threadIdx.x; item < 2 * TC; item += blockDim.x) {
    const int cc = item % TC, seg = item / TC;
    if (cc >= cols) continue;
    const int j = c0 + cc;
    const int rb = seg * RS;
    if (rb >= rows) continue;
    T2 vM[RS + 2 * P], vS[RS + 2 * P], vA[RS + 2 * P];
#pragma unroll
    for (int t = 0; t < RS + 2 * P; ++t) {
      vM[t] = sp[(size_t)(0 * HR + rb + t) * TC + cc];
      vS[t] = sp[(size_t)(1 * HR + rb + t) * TC + cc];
      vA[t] = sp[(size_t)(2 * HR + rb + t) * TC + cc];
    }
#pragma unroll
    for (int r = 0; r < RS; ++r) {
      if (rb + r < rows) {
        const int i = r0 + rb + r;
        T2 yy = mk2<T2>(T(0), T(0));
        if (i >= cs.lo && i < cs.hi) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            yy = pfma(cs.c[0][k], vM[r + k], yy);
            yy = pfma(cs.c[2][k], vS[r + k], yy);
            yy = pfma(cs.c[1][k], vA[r + k], yy);
          }
        } else {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            yy = pfma(BM[(size_t)k * m + i], vM[r + k], yy);
            yy = pfma(BS[(size_t)k * m + i], vS[r + k], yy);
            yy = pfma(BA[(size_t)k * m + i], vA[r + k], yy);
          }
        }
        const long long o1 = (long long)b * N + (long long)i * m + j, o2 = o1 + (long long)m * m;
        T y1 = yy.x, y2 = yy.y;
        if (mode == 2) {
          const T Mi = BM[(size_t)P * m + i], Si = BS[(size_t)P * m + i];
          const T Mj = BM[(size_t)P * m + j], Sj = BS[(size_t)P * m + j];
          cheb_epi(epi, o1, rhs[o1] - y1, inv_diag2(be, Si, Mj, al, Mi, Sj), ec1, ec2);
          cheb_epi(epi, o2, rhs[o2] - y2, inv_diag2(al, Si, Mj, be, Mi, Sj), ec1, ec2);
          continue;
        }
        if (mode == 1) {
          y1 = rhs[o1] - y1;
          y2 = rhs[o2] - y2;
          if (dotp) acc += (double)y1 * (double)y1 + (double)y2 * (double)y2;
        } else if (dotp) {
          acc += (double)w[o1] * (double)y1 + (double)w[o2] * (double)y2;
        }
        y[o1] = y1;
        y[o2] = y2;
      }
    }
  }
  if (dotp) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0)
      dotp[(size_t)b * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

// ---- stencil registry: band device pointer -> central stencil of that level (host copy)
static std::mutex g_stencil_mu;
static std::unordered_map<const void*, StencilHost> g_stencils;

__global__ void split_bands_kernel(int n, const double* __restrict__ src, float2* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float h = __double2float_rn(src[i]);
    dst[i] = make_float2(h, __double2float_rn(src[i] - (double)h));
  }
}

void register_level(const void* bands_dev, int m, int P, int lo, int hi, const double* central) {
  StencilHost st{m, P, lo, hi, {}, nullptr};
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 2 * P + 1 && k < 13; ++k) st.c[x][k] = central[x * (2 * P + 1) + k];
  std::lock_guard<std::mutex> lk(g_stencil_mu);
  auto it = g_stencils.find(bands_dev);
  if (it != g_stencils.end() && it->second.ffT) cudaFree(it->second.ffT);
  g_stencils[bands_dev] = st;
}
// FP64 levels also get the (hi, lo) split of their k-major bands for the double-FP32 apply.
void register_level_ff(const double* bands_dev, int m, int P) {
  const int n = 3 * (2 * P + 1) * m;
  float2* ff = nullptr;
  if (cudaMalloc(&ff, sizeof(float2) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return;  // the double-FP32 apply then declines this level
  }
  split_bands_kernel<<<(n + 255) / 256, 256>>>(n, bands_dev + (size_t)3 * m * (2 * P + 1), ff);
  count_launch();
  std::lock_guard<std::mutex> lk(g_stencil_mu);
  auto it = g_stencils.find(bands_dev);
  if (it == g_stencils.end()) {
    cudaFree(ff);
    return;
  }
  if (it->second.ffT) cudaFree(it->second.ffT);
  it->second.ffT = ff;
}
void unregister_level(const void* bands_dev) {
  std::lock_guard<std::mutex> lk(g_stencil_mu);
  auto it = g_stencils.find(bands_dev);
  if (it != g_stencils.end()) {
    if (it->second.ffT) cudaFree(it->second.ffT);
    g_stencils.erase(it);
  }
}
bool find_level(const void* bands_dev, StencilHost& out) {
  std::lock_guard<std::mutex> lk(g_stencil_mu);
  auto it = g_stencils.find(bands_dev);
  if (it == g_stencils.end()) return false;
  out = it->second;
  return true;
}

template <typename T>
static thread_local Epi<T> g_epi{};  // epilogue of the launch in progress (mode 2)

template <typename T, int P, int TR>
static void launch_v2(int m, const T* bands, const StencilHost& sh, const T* w, T* y, const T* rhs,
                      int mode, int B, Coef c, double* dotp, int* nblk, const int* active,
                      cudaStream_t s) {
  Stencil<T> cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) cs.c[x][k] = k < 2 * P + 1 ? (T)sh.c[x][k] : T(0);
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  const size_t smem = sizeof(T) * ((size_t)6 * TR * (m + 2 * P) + 8);
  dim3 grid((m + TR - 1) / TR, B);
  apply2d_v2_kernel<T, P, TR><<<grid, 256, smem, s>>>(m, bands + (size_t)3 * m * (2 * P + 1), cs,
                                                     w, y, rhs, mode, c.alpha, c.beta, c.gsc, active, dotp,
                                                     g_epi<T>);
  count_launch();
  if (nblk) *nblk = grid.x;
}

template <typename T, int P, int TR>
static void launch_v3(int m, const T* bands, const StencilHost& sh, const T* w, T* y, const T* rhs,
                      int mode, int B, Coef c, double* dotp, int* nblk, const int* active,
                      cudaStream_t s) {
  Stencil<T> cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) cs.c[x][k] = k < 2 * P + 1 ? (T)sh.c[x][k] : T(0);
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  const size_t smem = (size_t)3 * (TR + 2 * P) * 64 * 2 * sizeof(T);
  dim3 grid((m + 63) / 64, (m + TR - 1) / TR, B);
  apply2d_v3_kernel<T, P, TR><<<grid, 128, smem, s>>>(m, bands + (size_t)3 * m * (2 * P + 1), cs,
                                                     w, y, rhs, mode, c.alpha, c.beta, c.gsc, active, dotp,
                                                     g_epi<T>);
  count_launch();
  if (nblk) *nblk = grid.x * grid.y;
}

template <typename T, int P>
static bool try_v3_P_tr(int TR, int m, const T* bands, const StencilHost& sh, const T* w, T* y,
                        const T* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                        const int* active, cudaStream_t s) {
  if (TR == 16)
    launch_v3<T, P, 16>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  else
    launch_v3<T, P, 8>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  return true;
}

template <typename T, int P>
static bool try_v3_P(int m, const T* bands, const StencilHost& sh, const T* w, T* y, const T* rhs,
                     int mode, int B, Coef c, double* dotp, int* nblk, const int* active,
                     cudaStream_t s) {
  // FP32: 16 rows per tile except P = 5 (fewest spills at 128 registers); FP64: 8 rows
  if (sizeof(T) == 4 && P != 5)
    launch_v3<T, P, 16>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  else
    launch_v3<T, P, 8>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  return true;
}

template <typename T>
static bool try_apply2d_v3(int m, int P, const T* bands, const T* w, T* y, const T* rhs, int mode,
                           int B, Coef c, double* dotp, int* nblk, const int* active,
                           cudaStream_t s, int TR = 0) {
  StencilHost sh;
  if (!find_level(bands, sh) || sh.P != P) return false;
  if (dotp && (long long)((m + 63) / 64) * ((m + 7) / 8) > kMaxPartials) return false;
  if (TR == 8 || TR == 16) {
    switch (P) {
      case 1: return try_v3_P_tr<T, 1>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      case 2: return try_v3_P_tr<T, 2>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      case 3: return try_v3_P_tr<T, 3>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      case 4: return try_v3_P_tr<T, 4>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      case 5: return try_v3_P_tr<T, 5>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      case 6: return try_v3_P_tr<T, 6>(TR, m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
      default: return false;
    }
  }
  switch (P) {
    case 1: return try_v3_P<T, 1>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 2: return try_v3_P<T, 2>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 3: return try_v3_P<T, 3>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 4: return try_v3_P<T, 4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 5: return try_v3_P<T, 5>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 6: return try_v3_P<T, 6>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    default: return false;
  }
}

template <typename T, int P, int TR>
static void set_v3_attr() {
  cudaFuncSetAttribute(apply2d_v3_kernel<T, P, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((size_t)3 * (TR + 2 * P) * 64 * 2 * sizeof(T)));
}
template <typename T, int P>
static void set_v3_attrs() {
  set_v3_attr<T, P, 16>();
  set_v3_attr<T, P, 8>();
}

template <typename T, int P>
static bool try_v2_P(int m, const T* bands, const StencilHost& sh, const T* w, T* y, const T* rhs,
                     int mode, int B, Coef c, double* dotp, int* nblk, const int* active,
                     cudaStream_t s) {
  const size_t cap = 110 * 1024;
  auto fits = [&](int TR) { return sizeof(T) * ((size_t)6 * TR * (m + 2 * P) + 8) <= cap; };
  if (sizeof(T) == 4 && fits(16)) {
    launch_v2<T, P, 16>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  } else if (sizeof(T) == 4 && fits(8)) {
    launch_v2<T, P, 8>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  } else if (fits(4)) {
    launch_v2<T, P, 4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
  } else {
    return false;
  }
  return true;
}

template <typename T>
static bool try_apply2d_v2(int m, int P, const T* bands, const T* w, T* y, const T* rhs, int mode,
                           int B, Coef c, double* dotp, int* nblk, const int* active,
                           cudaStream_t s) {
  StencilHost sh;
  if (!find_level(bands, sh) || sh.P != P) return false;
  switch (P) {
    case 1: return try_v2_P<T, 1>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 2: return try_v2_P<T, 2>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 3: return try_v2_P<T, 3>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 4: return try_v2_P<T, 4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 5: return try_v2_P<T, 5>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 6: return try_v2_P<T, 6>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    default: return false;
  }
}

// ------------------------------------------------------------------ 2D FP32 apply, v5
// The FP32 operator apply on the tile layout of the packed double-FP32 kernel: the input tile
// with its halo is staged once in shared memory by coalesced loads (w1, w2 interleaved as
// float2), the x_2 pass runs one halo row per lane (folded symmetric / skew interior stencils,
// FFMA2 on the component pair), the x_1 pass one column per lane; both shared-memory arrays
// have an odd row stride in 8-byte slots, so both passes are free of bank conflicts.
template <int P>
struct V5Tile {
  static constexpr int W = 2 * P + 1;
  static constexpr int TC = 32;
  static constexpr int TR = P <= 4 ? 24 : 20;
  static constexpr int HR = TR + 2 * P;           // <= 32
  static constexpr int HC = TC + 2 * P;
  static constexpr int HCP = HC | 1;              // odd row strides (8-byte slots)
  static constexpr int TCP = TC + 1;
  static constexpr int NC = 4;
  static constexpr int RS = TR / 4;
  // input tile | intermediates | band rows of the tile's columns (boundary tiles); the band rows
  // of the tile's rows reuse the input tile's space in the x_1 pass
  static constexpr size_t off_mid = sizeof(float2) * HR * HCP;
  static constexpr size_t off_col = off_mid + sizeof(float2) * 3 * HR * TCP;
  static constexpr size_t smem = off_col + sizeof(float) * 3 * W * TC;
  static_assert(sizeof(float) * 3 * W * TR <= off_mid, "row coefficients fit the input tile");
};

__device__ __forceinline__ float2 bc2(float c) { return make_float2(c, c); }

__device__ __forceinline__ void v5_emit(float2 yy, int i, int j, long long o1, long long o2, int mode,
                                        int m, int P, const float* __restrict__ BM,
                                        const float* __restrict__ BS, float al, float be,
                                        const float* __restrict__ w, float* __restrict__ y,
                                        const float* __restrict__ rhs, const Epi<float>& epi,
                                        float ec1, float ec2, const double* dotp, double& acc) {
  float y1 = yy.x, y2 = yy.y;
  if (mode == 2) {
    const float Mi = BM[(size_t)P * m + i], Si = BS[(size_t)P * m + i];
    const float Mj = BM[(size_t)P * m + j], Sj = BS[(size_t)P * m + j];
    cheb_epi(epi, o1, rhs[o1] - y1, inv_diag2(be, Si, Mj, al, Mi, Sj), ec1, ec2);
    cheb_epi(epi, o2, rhs[o2] - y2, inv_diag2(al, Si, Mj, be, Mi, Sj), ec1, ec2);
    return;
  }
  if (mode == 1) {
    y1 = rhs[o1] - y1;
    y2 = rhs[o2] - y2;
    if (dotp) acc += (double)y1 * (double)y1 + (double)y2 * (double)y2;
  } else if (dotp) {
    acc += (double)w[o1] * (double)y1 + (double)w[o2] * (double)y2;
  }
  y[o1] = y1;
  y[o2] = y2;
}

template <int P>
__global__ void __launch_bounds__(128, P <= 4 ? 4 : 3) apply2d_v5_kernel(
    int m, const float* __restrict__ bandT, Stencil<float> cs, const float* __restrict__ w,
    float* __restrict__ y, const float* __restrict__ rhs, int mode,
    const double* __restrict__ alpha, const double* __restrict__ beta,
    const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<float> epi) {
  using G = V5Tile<P>;
  constexpr int W = G::W, TC = G::TC, TR = G::TR, HR = G::HR, HC = G::HC, HCP = G::HCP;
  constexpr int TCP = G::TCP, NC = G::NC, RS = G::RS;
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sIn = reinterpret_cast<float2*>(smem_raw);                // [HR][HCP] (w1, w2)
  float2* sMid = reinterpret_cast<float2*>(smem_raw + G::off_mid);  // [3][HR][TCP] PM, PS, PA
  float* sCol = reinterpret_cast<float*>(smem_raw + G::off_col);    // [3][W][TC]
  float* sRow = reinterpret_cast<float*>(smem_raw);                 // [3][W][TR] (x_1 pass)
  const long long N = 2LL * m * m;
  const float* wb = w + (long long)b * N;
  const int c0 = blockIdx.x * TC, r0 = blockIdx.y * TR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool bcol = c0 < cs.lo || c0 + TC > cs.hi;
  const bool brow = r0 < cs.lo || r0 + TR > cs.hi;
  {  // every load of the tile in flight before the first store (one memory latency per tile)
    constexpr int NE = (HR * HC + 127) / 128;
    float2 v[NE];
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int rr = idx / HC, cc = idx - rr * HC;
      const int row = r0 - P + rr, col = c0 - P + cc;
      v[t] = make_float2(0.f, 0.f);
      if (idx < HR * HC && row >= 0 && row < m && col >= 0 && col < m) {
        const long long o = (long long)row * m + col;
        v[t] = make_float2(wb[o], wb[(long long)m * m + o]);
      }
    }
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int rr = idx / HC, cc = idx - rr * HC;
      if (idx < HR * HC) sIn[rr * HCP + cc] = v[t];
    }
  }
  if (bcol) {
    constexpr int NK = (3 * W * TC + 127) / 128;
    float v[NK];
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int xk = idx / TC, cc = idx - xk * TC;
      v[t] = idx < 3 * W * TC && c0 + cc < m ? bandT[(size_t)xk * m + c0 + cc] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < NK; ++t)
      if (threadIdx.x + 128 * t < 3 * W * TC) sCol[threadIdx.x + 128 * t] = v[t];
  }
  __shared__ float s_par[3];  // alpha, beta, gamma in FP32, converted once per CTA
  if (threadIdx.x == 0) {
    s_par[0] = float(alpha[b]);
    s_par[1] = float(beta[b]);
    s_par[2] = float((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  }
  __syncthreads();
  const float al = s_par[0], be = s_par[1], ga = s_par[2];
  // ---- axis x_2: lane = halo row
  if (lane < HR) {
    const int q = lane, row = r0 - P + q;
    const bool rowok = row >= 0 && row < m;
    for (int g = warp; g < TC / NC; g += 4) {
      const int j0 = c0 + g * NC;
      if (rowok && j0 < m && j0 >= cs.lo && j0 + NC - 1 < cs.hi) {
        float2 x[NC + 2 * P];
#pragma unroll
        for (int t = 0; t < NC + 2 * P; ++t) x[t] = sIn[q * HCP + g * NC + t];
#pragma unroll
        for (int u = 0; u < NC; ++u) {
          float2 tM = __fmul2_rn(bc2(cs.c[0][P]), x[u + P]);
          float2 tS = __fmul2_rn(bc2(cs.c[2][P]), x[u + P]);
          float2 tA = make_float2(0.f, 0.f);
#pragma unroll
          for (int t = 1; t <= P; ++t) {
            const float2 sp = __fadd2_rn(x[u + P - t], x[u + P + t]);
            const float2 dp = __ffma2_rn(x[u + P - t], bc2(-1.f), x[u + P + t]);
            tM = __ffma2_rn(bc2(cs.c[0][P + t]), sp, tM);
            tS = __ffma2_rn(bc2(cs.c[2][P + t]), sp, tS);
            tA = __ffma2_rn(bc2(cs.c[1][P + t]), dp, tA);
          }
          const int cc = g * NC + u;
          sMid[(0 * HR + q) * TCP + cc] = __fmul2_rn(make_float2(al, be), tS);  // feeds M1
          sMid[(1 * HR + q) * TCP + cc] = __fmul2_rn(make_float2(be, al), tM);  // feeds S1
          sMid[(2 * HR + q) * TCP + cc] = __fmul2_rn(bc2(ga), make_float2(tA.y, tA.x));
        }
      } else {  // boundary columns (band rows staged in shared memory) or outside the domain
#pragma unroll 1
        for (int u = 0; u < NC; ++u) {
          const int cc = g * NC + u;
          float2 tM = make_float2(0.f, 0.f), tS = tM, tA = tM;
          if (rowok && c0 + cc < m) {
#pragma unroll 1
            for (int k = 0; k < W; ++k) {
              const float2 xv = sIn[q * HCP + cc + k];
              tM = __ffma2_rn(bc2(sCol[(0 * W + k) * TC + cc]), xv, tM);
              tA = __ffma2_rn(bc2(sCol[(1 * W + k) * TC + cc]), xv, tA);
              tS = __ffma2_rn(bc2(sCol[(2 * W + k) * TC + cc]), xv, tS);
            }
          }
          sMid[(0 * HR + q) * TCP + cc] = __fmul2_rn(make_float2(al, be), tS);
          sMid[(1 * HR + q) * TCP + cc] = __fmul2_rn(make_float2(be, al), tM);
          sMid[(2 * HR + q) * TCP + cc] = __fmul2_rn(bc2(ga), make_float2(tA.y, tA.x));
        }
      }
    }
  }
  __syncthreads();
  if (brow) {
    constexpr int NK = (3 * W * TR + 127) / 128;
    float v[NK];
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int xk = idx / TR, rr = idx - xk * TR;
      v[t] = idx < 3 * W * TR && r0 + rr < m ? bandT[(size_t)xk * m + r0 + rr] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < NK; ++t)
      if (threadIdx.x + 128 * t < 3 * W * TR) sRow[threadIdx.x + 128 * t] = v[t];
    __syncthreads();
  }
  // ---- axis x_1: lane = column, RS rows per warp
  double acc = 0.0;
  float ec1 = 0.f, ec2 = 0.f;
  if (mode == 2) {
    double c1, c2;
    cheb_coef_cta(epi.lmax[b], epi.step, c1, c2);
    ec1 = float(c1);
    ec2 = float(c2);
  }
  const float* BM = bandT;
  const float* BS = bandT + (size_t)2 * W * m;
  const int cc = lane, j = c0 + cc, rb = warp * RS;
  if (j < m) {
    if (r0 + rb >= cs.lo && r0 + rb + RS - 1 < cs.hi) {
      float2 yy[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) yy[r] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int band = 0; band < 2; ++band) {  // M on PM, S on PS (symmetric)
        float2 v[RS + 2 * P];
#pragma unroll
        for (int t = 0; t < RS + 2 * P; ++t) v[t] = sMid[(band * HR + rb + t) * TCP + cc];
        float cf[P + 1];
#pragma unroll
        for (int t = 0; t <= P; ++t) cf[t] = band == 0 ? cs.c[0][P + t] : cs.c[2][P + t];
#pragma unroll
        for (int r = 0; r < RS; ++r) {
          yy[r] = __ffma2_rn(bc2(cf[0]), v[r + P], yy[r]);
#pragma unroll
          for (int t = 1; t <= P; ++t)
            yy[r] = __ffma2_rn(bc2(cf[t]), __fadd2_rn(v[r + P - t], v[r + P + t]), yy[r]);
        }
      }
      {  // A on PA (skew)
        float2 v[RS + 2 * P];
#pragma unroll
        for (int t = 0; t < RS + 2 * P; ++t) v[t] = sMid[(2 * HR + rb + t) * TCP + cc];
#pragma unroll
        for (int r = 0; r < RS; ++r)
#pragma unroll
          for (int t = 1; t <= P; ++t)
            yy[r] = __ffma2_rn(bc2(cs.c[1][P + t]),
                               __ffma2_rn(v[r + P - t], bc2(-1.f), v[r + P + t]), yy[r]);
      }
#pragma unroll
      for (int r = 0; r < RS; ++r) {
        const int i = r0 + rb + r;
        const long long o1 = (long long)b * N + (long long)i * m + j;
        v5_emit(yy[r], i, j, o1, o1 + (long long)m * m, mode, m, P, BM, BS, al, be, w, y, rhs, epi,
                ec1, ec2, dotp, acc);
      }
    } else {  // boundary rows (band rows staged in shared memory)
#pragma unroll 1
      for (int r = 0; r < RS; ++r) {
        const int i = r0 + rb + r;
        if (i >= m) break;
        float2 yy = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int band = 0; band < 3; ++band) {
          const int x = band == 0 ? 0 : band == 1 ? 2 : 1;
#pragma unroll 1
          for (int k = 0; k < W; ++k)
            yy = __ffma2_rn(bc2(sRow[(x * W + k) * TR + rb + r]), sMid[(band * HR + rb + r + k) * TCP + cc], yy);
        }
        const long long o1 = (long long)b * N + (long long)i * m + j;
        v5_emit(yy, i, j, o1, o1 + (long long)m * m, mode, m, P, BM, BS, al, be, w, y, rhs, epi,
                ec1, ec2, dotp, acc);
      }
    }
  }
  if (dotp) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0)
      dotp[(size_t)b * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

template <int P>
static void set_v5_attr() {
  cudaFuncSetAttribute(apply2d_v5_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)V5Tile<P>::smem);
}


template <int P>
static bool launch_v5_P(int m, const float* bands, const StencilHost& sh, const float* w, float* y,
                        const float* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                        const int* active, cudaStream_t s) {
  using G = V5Tile<P>;
  Stencil<float> cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) cs.c[x][k] = k < 2 * P + 1 ? (float)sh.c[x][k] : 0.f;
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  dim3 grid((m + G::TC - 1) / G::TC, (m + G::TR - 1) / G::TR, B);
  if (dotp && (long long)grid.x * grid.y > kMaxPartials) return false;
  apply2d_v5_kernel<P><<<grid, 128, G::smem, s>>>(m, bands + (size_t)3 * m * (2 * P + 1), cs, w, y,
                                                  rhs, mode, c.alpha, c.beta, c.gsc, active, dotp,
                                                  g_epi<float>);
  count_launch();
  if (nblk) *nblk = grid.x * grid.y;
  return true;
}

static bool try_apply2d_v5(int m, int P, const float* bands, const float* w, float* y,
                           const float* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                           const int* active, cudaStream_t s) {
  StencilHost sh;
  if (!find_level(bands, sh) || sh.P != P || !stencil_folds(sh)) return false;
  switch (P) {
    case 1: return launch_v5_P<1>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 2: return launch_v5_P<2>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 3: return launch_v5_P<3>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 4: return launch_v5_P<4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 5: return launch_v5_P<5>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    case 6: return launch_v5_P<6>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s);
    default: return false;
  }
}

template <typename T, int P, int TR>
static void set_v2_attr() {
  cudaFuncSetAttribute(apply2d_v2_kernel<T, P, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       110 * 1024);
}
template <typename T, int P>
static void set_v2_attrs() {
  set_v2_attr<T, P, 16>();
  set_v2_attr<T, P, 8>();
  set_v2_attr<T, P, 4>();
}

// ------------------------------------------------------------------ generic banded axis pass
// out_o = sum_t coef_t * (X_t along `axis`) in_{src_t}, for up to 9 outputs per launch.
// Every array is one component [B][m]^d with its own batch stride.
struct AxisTerm {
  int src, band, coef;  // band: 0 = M, 1 = A, 2 = S; coef: 0 = 1, 1 = alpha, 2 = beta, 3 = gamma
};
template <typename T>
struct AxisParams {
  const T* in[9];
  long long in_bs[9];
  T* out[9];
  long long out_bs[9];
  int nt[9];
  AxisTerm t[9][3];
  int nout;
};

template <typename T>
__global__ void __launch_bounds__(256) axis_pass_kernel(AxisParams<T> prm, int d, int m, int P,
                                                        int axis, const T* __restrict__ bands,
                                                        const double* __restrict__ alpha,
                                                        const double* __restrict__ beta, const double* __restrict__ gsc,
                                                        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  long long npts = m;
  for (int l = 1; l < d; ++l) npts *= m;
  long long stride = 1;
  for (int l = axis + 1; l < d; ++l) stride *= m;
  const int W = 2 * P + 1;
  const T cf[4] = {T(1), T(alpha[b]), T(beta[b]), T((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0))};
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < npts;
       pt += (long long)gridDim.x * blockDim.x) {
    const int ia = (int)((pt / stride) % m);
    const int k0 = max(0, P - ia), k1 = min(W - 1, m - 1 - ia + P);
    for (int o = 0; o < prm.nout; ++o) {
      T acc = 0;
      for (int t = 0; t < prm.nt[o]; ++t) {
        const AxisTerm tm = prm.t[o][t];
        const T* in = prm.in[tm.src] + (long long)b * prm.in_bs[tm.src] + pt;
        const T* band = bands + (size_t)tm.band * m * W + (size_t)ia * W;
        T s = 0;
        for (int k = k0; k <= k1; ++k) s += band[k] * in[(long long)(k - P) * stride];
        acc += cf[tm.coef] * s;
      }
      prm.out[o][(long long)b * prm.out_bs[o] + pt] = acc;
    }
  }
}

// y = A w (3D) via three banded passes: axis x_3 -> nine arrays T_{X,c} = X_3 w_c,
// axis x_2 -> nine arrays P (grouped by the x_1 operator they feed), axis x_1 -> y.
template <typename T>
static int apply3d_multipass(int m, int P, const T* bands, const T* w, T* y, int B, Coef c,
                             const int* active, T* scratch, cudaStream_t s) {
  // scratch: 9 + 9 arrays of [B][m^3] followed by one [B][3 m^3] output buffer
  const long long n3 = (long long)m * m * m;
  const long long N = 3 * n3;
  T* Tm = scratch;              // 9 arrays [B][m^3]: index X*3 + comp (X: 0 M, 1 A, 2 S)
  T* Pm = scratch + 9 * n3 * B;  // 9 arrays: P1M,P1S,P1A,P2M,P2S,P2A,P3M,P3S,P3A
  const int threads = 256;
  long long blocks = (n3 + threads - 1) / threads;
  dim3 grid((unsigned)std::min<long long>(blocks, 65535), B);
  // pass 1: axis 2 (x_3)
  AxisParams<T> a{};
  for (int comp = 0; comp < 3; ++comp) {
    a.in[comp] = w + comp * n3;
    a.in_bs[comp] = N;
  }
  a.nout = 9;
  for (int X = 0; X < 3; ++X)
    for (int comp = 0; comp < 3; ++comp) {
      const int o = X * 3 + comp;
      a.out[o] = Tm + (long long)o * n3 * B;
      a.out_bs[o] = n3;
      a.nt[o] = 1;
      a.t[o][0] = AxisTerm{comp, X, 0};
    }
  axis_pass_kernel<T><<<grid, threads, 0, s>>>(a, 3, m, P, 2, bands, c.alpha, c.beta, c.gsc, active);
  // pass 2: axis 1 (x_2).  Inputs: T arrays (index X*3 + comp).
  AxisParams<T> q{};
  for (int i = 0; i < 9; ++i) {
    q.in[i] = Tm + (long long)i * n3 * B;
    q.in_bs[i] = n3;
  }
  auto TI = [](int X, int comp) { return X * 3 + comp; };  // X: 0 M, 1 A, 2 S
  const int M_ = 0, A_ = 1, S_ = 2;
  const int one = 0, al = 1, be = 2, ga = 3;
  q.nout = 9;
  for (int o = 0; o < 9; ++o) {
    q.out[o] = Pm + (long long)o * n3 * B;
    q.out_bs[o] = n3;
  }
  // P1M = alpha (M2 T_S1 + S2 T_M1); P1S = beta M2 T_M1; P1A = gamma (A2 T_M2 + M2 T_A3)
  q.nt[0] = 2; q.t[0][0] = {TI(S_, 0), M_, al}; q.t[0][1] = {TI(M_, 0), S_, al};
  q.nt[1] = 1; q.t[1][0] = {TI(M_, 0), M_, be};
  q.nt[2] = 2; q.t[2][0] = {TI(M_, 1), A_, ga}; q.t[2][1] = {TI(A_, 2), M_, ga};
  // P2M = alpha M2 T_S2 + beta S2 T_M2 + gamma A2 T_A3; P2S = alpha M2 T_M2; P2A = gamma A2 T_M1
  q.nt[3] = 3; q.t[3][0] = {TI(S_, 1), M_, al}; q.t[3][1] = {TI(M_, 1), S_, be};
  q.t[3][2] = {TI(A_, 2), A_, ga};
  q.nt[4] = 1; q.t[4][0] = {TI(M_, 1), M_, al};
  q.nt[5] = 1; q.t[5][0] = {TI(M_, 0), A_, ga};
  // P3M = alpha S2 T_M3 + beta M2 T_S3 + gamma A2 T_A2; P3S = alpha M2 T_M3; P3A = gamma M2 T_A1
  q.nt[6] = 3; q.t[6][0] = {TI(M_, 2), S_, al}; q.t[6][1] = {TI(S_, 2), M_, be};
  q.t[6][2] = {TI(A_, 1), A_, ga};
  q.nt[7] = 1; q.t[7][0] = {TI(M_, 2), M_, al};
  q.nt[8] = 1; q.t[8][0] = {TI(A_, 0), M_, ga};
  (void)one;
  axis_pass_kernel<T><<<grid, threads, 0, s>>>(q, 3, m, P, 1, bands, c.alpha, c.beta, c.gsc, active);
  // pass 3: axis 0 (x_1): y_c = M1 P_cM + S1 P_cS + A1 P_cA
  AxisParams<T> r{};
  for (int i = 0; i < 9; ++i) {
    r.in[i] = Pm + (long long)i * n3 * B;
    r.in_bs[i] = n3;
  }
  r.nout = 3;
  for (int comp = 0; comp < 3; ++comp) {
    r.out[comp] = y + comp * n3;
    r.out_bs[comp] = N;
    r.nt[comp] = 3;
    r.t[comp][0] = {comp * 3 + 0, M_, 0};
    r.t[comp][1] = {comp * 3 + 1, S_, 0};
    r.t[comp][2] = {comp * 3 + 2, A_, 0};
  }
  axis_pass_kernel<T><<<grid, threads, 0, s>>>(r, 3, m, P, 0, bands, c.alpha, c.beta, c.gsc, active);
  count_launch(3);
  return 0;
}


// ------------------------------------------------------------------ 3D fused apply
// One CTA: an (x_3, x_2) tile of 32 x T2 points and a chunk of output planes [k_lo, k_hi)
// along x_1.  It marches through the input planes q = k_lo - P .. k_hi + P - 1; for each plane
// it stages the haloed tile of w (3 components) in shared memory, applies the x_3 operators
// (9 arrays T_{X,c} = X_3 w_c on the tile plus P halo rows of x_2), then each thread forms its
// point's 9 x_2-results (grouped by the x_1 operator they feed, as in the multi-pass version)
// and scatters them into 2P+1 pending output planes held as a register shift register:
//   y_c[k] += M_1(k,q) P_cM[q] + S_1(k,q) P_cS[q] + A_1(k,q) P_cA[q],  |k - q| <= P.
// Plane k is complete once q = k + P has been handled (or the last plane, near the end of the
// domain); it then leaves through the epilogue (modes 0, 1, 2) and the planes shift by one (one
// loop body for every plane).  The next plane's tile is loaded into registers while the
// current one is computed.
// Central Toeplitz stencils come from the constant bank, boundary rows from bandT.
template <typename T>
__device__ __forceinline__ T band_coef(const Stencil<T>& cs, const T* const* BX, int m, int X,
                                       int i, int k) {  // X(i, i + k - P)
  return (i >= cs.lo && i < cs.hi) ? cs.c[X][k] : BX[X][(size_t)k * m + i];
}

template <typename T, int P, int T2>
__global__ void __launch_bounds__(32 * T2, 2) apply3d_stream_kernel(
    int m, int L, const T* __restrict__ bandT, Stencil<T> cs, const T* __restrict__ w,
    T* __restrict__ y, const T* __restrict__ rhs, int mode, const double* __restrict__ alpha,
    const double* __restrict__ beta, const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<T> epi) {
  constexpr int W = 2 * P + 1, T3 = 32;
  constexpr int HR = T2 + 2 * P, HC = T3 + 2 * P;
  const int nchunk = (m + L - 1) / L;
  const int b = blockIdx.z / nchunk, chunk = blockIdx.z - b * nchunk;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sw = reinterpret_cast<T*>(smem_raw);  // [3][HR][HC]
  T* st = sw + 3 * HR * HC;                // [9][HR][T3], index X * 3 + c (X: 0 M, 1 A, 2 S)
  const long long n3 = (long long)m * m * m, N = 3 * n3;
  const T* wb = w + (long long)b * N;
  const int i3_0 = blockIdx.x * T3, i2_0 = blockIdx.y * T2;
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  const int i2 = i2_0 + row, i3 = i3_0 + lane;
  const bool mine = i2 < m && i3 < m;
  const int k_lo = chunk * L, k_hi = min(m, k_lo + L);
  const T al = T(alpha[b]), be = T(beta[b]), ga = T((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  const T* BX[3] = {bandT, bandT + (size_t)W * m, bandT + (size_t)2 * W * m};
  T ec1 = 0, ec2 = 0;
  if (mode == 2) {
    double c1, c2;
    cheb_coef_cta(epi.lmax[b], epi.step, c1, c2);
    ec1 = T(c1);
    ec2 = T(c2);
  }
  T acc[W][3];  // acc[t]: pending output plane q - P + t (a shift register over the planes)
#pragma unroll
  for (int sl = 0; sl < W; ++sl) acc[sl][0] = acc[sl][1] = acc[sl][2] = T(0);
  double dacc = 0.0;
  const int q_begin = max(0, k_lo - P), q_end = min(m, k_hi + P);
  // the next plane's haloed tile, loaded into registers while the current one is computed
  constexpr int NE = (3 * HR * HC + 32 * T2 - 1) / (32 * T2);
  T pre[NE];
  auto load_plane = [&](int q) {
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int e = threadIdx.x + t * 32 * T2;
      if (e < 3 * HR * HC) {
        const int c = e / (HR * HC), rem = e - c * HR * HC;
        const int rr = rem / HC, cc = rem - rr * HC;
        const int g2 = i2_0 - P + rr, g3 = i3_0 - P + cc;
        pre[t] = (g2 >= 0 && g2 < m && g3 >= 0 && g3 < m)
                     ? wb[(long long)c * n3 + ((long long)q * m + g2) * m + g3]
                     : T(0);
      }
    }
  };
  if (q_begin < q_end) load_plane(q_begin);
#pragma unroll 1
  for (int q = q_begin; q < q_end + P; ++q) {
    if (q < q_end) {  // uniform over the CTA
      __syncthreads();
#pragma unroll
      for (int t = 0; t < NE; ++t) {
        const int e = threadIdx.x + t * 32 * T2;
        if (e < 3 * HR * HC) sw[e] = pre[t];
      }
      if (q + 1 < q_end) load_plane(q + 1);
      __syncthreads();
      for (int e = threadIdx.x; e < HR * T3; e += blockDim.x) {  // x_3 operators
        const int rr = e / T3, cc = e - rr * T3;
        const int g3 = i3_0 + cc;
        T t[9];
#pragma unroll
        for (int u = 0; u < 9; ++u) t[u] = T(0);
        if (g3 < m) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const T cM = band_coef(cs, BX, m, 0, g3, k), cA = band_coef(cs, BX, m, 1, g3, k),
                    cS = band_coef(cs, BX, m, 2, g3, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const T v = sw[(c * HR + rr) * HC + cc + k];
              t[0 * 3 + c] += cM * v;
              t[1 * 3 + c] += cA * v;
              t[2 * 3 + c] += cS * v;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 9; ++u) st[(u * HR + rr) * T3 + cc] = t[u];
      }
      __syncthreads();
      T PM[3], PS[3], PA[3];  // x_2 results of this point, grouped by the x_1 operator
#pragma unroll
      for (int c = 0; c < 3; ++c) PM[c] = PS[c] = PA[c] = T(0);
      if (mine) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const T cM = band_coef(cs, BX, m, 0, i2, k), cA = band_coef(cs, BX, m, 1, i2, k),
                  cS = band_coef(cs, BX, m, 2, i2, k);
          const int rr = row + k;
          const T tM1 = st[(0 * HR + rr) * T3 + lane], tM2 = st[(1 * HR + rr) * T3 + lane];
          const T tM3 = st[(2 * HR + rr) * T3 + lane], tA1 = st[(3 * HR + rr) * T3 + lane];
          const T tA2 = st[(4 * HR + rr) * T3 + lane], tA3 = st[(5 * HR + rr) * T3 + lane];
          const T tS1 = st[(6 * HR + rr) * T3 + lane], tS2 = st[(7 * HR + rr) * T3 + lane];
          const T tS3 = st[(8 * HR + rr) * T3 + lane];
          // component 1: M1[alpha (M2 S3 + S2 M3) w1], S1[beta M2 M3 w1], A1[gamma (A2 M3 w2 + M2 A3 w3)]
          PM[0] += al * (cM * tS1 + cS * tM1);
          PS[0] += be * (cM * tM1);
          PA[0] += ga * (cA * tM2 + cM * tA3);
          // component 2: S1[alpha M2 M3 w2], M1[alpha M2 S3 w2 + beta S2 M3 w2 + gamma A2 A3 w3], A1[gamma A2 M3 w1]
          PS[1] += al * (cM * tM2);
          PM[1] += al * (cM * tS2) + be * (cS * tM2) + ga * (cA * tA3);
          PA[1] += ga * (cA * tM1);
          // component 3: S1[alpha M2 M3 w3], M1[alpha S2 M3 w3 + beta M2 S3 w3 + gamma A2 A3 w2], A1[gamma M2 A3 w1]
          PS[2] += al * (cM * tM3);
          PM[2] += al * (cS * tM3) + be * (cM * tS3) + ga * (cA * tA2);
          PA[2] += ga * (cM * tA1);
        }
      }
#pragma unroll
      for (int dd = 0; dd < W; ++dd) {  // x_1 scatter: plane kk = q - (dd - P) is slot 2P - dd
        const int kk = q - (dd - P);
        if (kk >= k_lo && kk < k_hi) {
          const T cM = band_coef(cs, BX, m, 0, kk, dd), cA = band_coef(cs, BX, m, 1, kk, dd),
                  cS = band_coef(cs, BX, m, 2, kk, dd);
#pragma unroll
          for (int c = 0; c < 3; ++c)
            acc[2 * P - dd][c] += cM * PM[c] + cS * PS[c] + cA * PA[c];
        }
      }
    }
    // plane kd = q - P (slot 0) has received every contribution (q = kd + P, or the last plane)
    const int kd = q - P;
    if (kd >= k_lo && kd < k_hi && mine) {
      T Md[3], Sd[3];
      if (mode == 2) {
        const int I[3] = {kd, i2, i3};
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          Md[kx] = BX[0][(size_t)P * m + I[kx]];
          Sd[kx] = BX[2][(size_t)P * m + I[kx]];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long o = (long long)b * N + (long long)c * n3 + ((long long)kd * m + i2) * m + i3;
        const T v = acc[0][c];
        if (mode == 2) {
          cheb_epi(epi, o, rhs[o] - v, inv_diag3(al, be, c, Md, Sd), ec1, ec2);
        } else if (mode == 1) {
          const T r = rhs[o] - v;
          y[o] = r;
          if (dotp) dacc += (double)r * (double)r;
        } else {
          y[o] = v;
          if (dotp) dacc += (double)w[o] * (double)v;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 2 * P; ++t) {
      acc[t][0] = acc[t + 1][0];
      acc[t][1] = acc[t + 1][1];
      acc[t][2] = acc[t + 1][2];
    }
    acc[2 * P][0] = acc[2 * P][1] = acc[2 * P][2] = T(0);
  }
  if (dotp && mode != 2) {
    const double sum = block_sum(dacc);
    const int nblk = gridDim.x * gridDim.y * nchunk;
    const int blk = (chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) dotp[(size_t)b * nblk + blk] = sum;
  }
}

template <typename T, int P>
static size_t stream3d_smem() {
  constexpr int T2 = 8, HR = T2 + 2 * P, HC = 32 + 2 * P;
  return sizeof(T) * ((size_t)3 * HR * HC + (size_t)9 * HR * 32);
}

template <typename T, int P>
static void launch_stream3d(int m, const T* bands, const StencilHost& sh, const T* w, T* y,
                            const T* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                            const int* active, cudaStream_t s, const Epi<T>& epi) {
  Stencil<T> cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) cs.c[x][k] = k < 2 * P + 1 ? (T)sh.c[x][k] : T(0);
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  constexpr int L = 32;
  const int nchunk = (m + L - 1) / L;
  dim3 grid((m + 31) / 32, (m + 7) / 8, nchunk * B);
  apply3d_stream_kernel<T, P, 8><<<grid, 256, stream3d_smem<T, P>(), s>>>(
      m, L, bands + (size_t)3 * m * (2 * P + 1), cs, w, y, rhs, mode, c.alpha, c.beta, c.gsc, active,
      dotp, epi);
  count_launch();
  if (nblk) *nblk = grid.x * grid.y * nchunk;
}

// ---- autotuning table of the 3D apply: (precision bytes, m, P) -> 1 = streaming kernel,
// 2 = three banded passes (0 = not tuned: the static rule, streaming for FP32 with P <= 4)
static std::mutex g_tune3d_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned3d;
static int tuned3d_variant(size_t es, int m, int P) {
  std::lock_guard<std::mutex> lk(g_tune3d_mu);
  auto it = g_tuned3d.find(std::make_tuple((int)es, m, P));
  return it == g_tuned3d.end() ? 0 : it->second;
}

template <typename T>
static bool try_stream3d(int m, int P, const T* bands, const T* w, T* y, const T* rhs, int mode,
                         int B, Coef c, double* dotp, int* nblk, const int* active, cudaStream_t s,
                         const Epi<T>& epi) {
  // FP32 with p <= 4 only.  The kernel recomputes the x_3 results on the P halo rows of x_2
  // and the x_2/x_3 results on the P halo planes of each x_1 chunk, about 1.7x the arithmetic
  // of the three banded passes at p = 3.  FP32 is latency-bound and wins (m = 129: 347 vs
  // 500 us at p = 3, 154 vs 434 us at p = 2); FP64 is bound by the FP64 pipe (the passes
  // reach about 1 TFLOP/s) and loses by 3-4x, as does FP32 at p = 5.
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    StencilHost sh;
    if (!g_use_stream3d || !find_level(bands, sh) || sh.P != P) return false;
    if (tuned3d_variant(sizeof(T), m, P) == 2) return false;
    if (dotp && (long long)((m + 31) / 32) * ((m + 7) / 8) * ((m + 31) / 32) > kMaxPartials)
      return false;
    switch (P) {
      case 1: launch_stream3d<T, 1>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); return true;
      case 2: launch_stream3d<T, 2>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); return true;
      case 3: launch_stream3d<T, 3>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); return true;
      case 4: launch_stream3d<T, 4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); return true;
      default: return false;
    }
  }
}

template <typename T, int P>
static void set_stream3d_attr() {
  cudaFuncSetAttribute(apply3d_stream_kernel<T, P, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)stream3d_smem<T, P>());
}

// residual / dot post-pass for the multipass 3D apply
template <typename T>
__global__ void __launch_bounds__(256) post3d_kernel(long long N, const T* __restrict__ w,
                                                     const T* ytmp, T* y, const T* rhs,
                                                     int mode, const int* __restrict__ active,
                                                     double* __restrict__ dotp, int m, int P,
                                                     const T* __restrict__ bands,
                                                     const double* __restrict__ alpha,
                                                     const double* __restrict__ beta, Epi<T> epi) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long chunk = (N + gridDim.x - 1) / gridDim.x;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const long long base = (long long)b * N;
  double acc = 0.0;
  T ec1 = 0, ec2 = 0;
  if (mode == 2) {
    double c1, c2;
    cheb_coef_cta(epi.lmax[b], epi.step, c1, c2);
    ec1 = T(c1);
    ec2 = T(c2);
  }
  const int W = 2 * P + 1;
  const long long n3 = N / 3;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    T v = ytmp[base + i];
    if (mode == 2) {
      const int comp = (int)(i / n3);
      long long rem = i - comp * n3;
      const int i2 = (int)(rem % m), i1 = (int)((rem / m) % m), i0 = (int)(rem / ((long long)m * m));
      const int I[3] = {i0, i1, i2};
      T Md[3], Sd[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Md[k] = bands[(size_t)I[k] * W + P];
        Sd[k] = bands[(size_t)2 * m * W + I[k] * W + P];
      }
      cheb_epi(epi, base + i, rhs[base + i] - v, inv_diag3(T(alpha[b]), T(beta[b]), comp, Md, Sd),
               ec1, ec2);
      continue;
    }
    if (mode == 1) {
      v = rhs[base + i] - v;
      y[base + i] = v;
      if (dotp) acc += (double)v * (double)v;
    } else if (dotp) {
      acc += (double)w[base + i] * (double)v;
    }
  }
  if (dotp) {
    const double s = block_sum(acc);
    if (threadIdx.x == 0) dotp[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------ anisotropic meshes
// Section 5: n_l = nu_l n intervals along x_l, so every direction has its own m_l and its own 1D
// bands.  The operator is the same sum of Kronecker products (eq:matr_Amu / eq:matr_Amu3D), each
// factor in position l being the 1D matrix of direction l; it is applied by one banded pass per
// direction (d = 2: six intermediate arrays, d = 3: nine and nine), a thread per grid point.
template <typename T>
__global__ void __launch_bounds__(256) aniso_pass_kernel(AxisParams<T> prm, int npts, int stride,
                                                         int ma, int P, const T* __restrict__ bands,
                                                         const double* __restrict__ alpha,
                                                         const double* __restrict__ beta,
                                                         const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int W = 2 * P + 1;
  __shared__ T s_cf[4];
  if (threadIdx.x == 0) {
    s_cf[0] = T(1);
    s_cf[1] = T(alpha[b]);
    s_cf[2] = T(beta[b]);
    s_cf[3] = T(alpha[b] - beta[b]);
  }
  __syncthreads();
  for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < npts; pt += gridDim.x * blockDim.x) {
    const int ia = (pt / stride) % ma;
    const int k0 = max(0, P - ia), k1 = min(W - 1, ma - 1 - ia + P);
    for (int o = 0; o < prm.nout; ++o) {
      T acc = 0;
      for (int t = 0; t < prm.nt[o]; ++t) {
        const AxisTerm tm = prm.t[o][t];
        const T* in = prm.in[tm.src] + (long long)b * prm.in_bs[tm.src] + pt;
        const T* band = bands + ((size_t)tm.band * ma + ia) * W;
        T s = 0;
        for (int k = k0; k <= k1; ++k) s += band[k] * in[(long long)(k - P) * stride];
        acc += s_cf[tm.coef] * s;
      }
      prm.out[o][(long long)b * prm.out_bs[o] + pt] = acc;
    }
  }
}

// y = A w on an anisotropic mesh: ma[l] unknowns per component along x_l, band[l] the [3][ma[l]][W]
// row-major (M, A, S) bands of direction l.  Scratch: 6 (d = 2) or 18 (d = 3) arrays of
// [B][prod ma] plus, for mode 1, one [B][N] buffer.  Modes: 0 (y = A w, optional w^T y
// partials), 1 (y = rhs - A w, optional y^T y partials).
template <typename T>
int launch_apply_aniso(int d, const int* ma, int P, const T* const* band, const T* w, T* y,
                       const T* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                       const int* active, T* scratch, cudaStream_t s) {
  if (mode > 1) return 1;
  const int npc = d == 2 ? ma[0] * ma[1] : ma[0] * ma[1] * ma[2];  // points per component
  const long long N = (long long)d * npc;
  const int nint = d == 2 ? 6 : 18;
  T* yt = mode == 1 ? scratch + (long long)nint * npc * B : y;
  const dim3 grid((unsigned)std::min<long long>((npc + 255) / 256, 4096), B);
  const int M_ = 0, A_ = 1, S_ = 2, one = 0, al = 1, be = 2, ga = 3;
  (void)one;
  auto strd = [&](int axis) {
    int st = 1;
    for (int l = axis + 1; l < d; ++l) st *= ma[l];
    return st;
  };
  if (d == 2) {
    // x_2 pass: PM_c, PS_c, PA_c grouped by the x_1 operator they feed
    AxisParams<T> q{};
    q.in[0] = w;
    q.in[1] = w + npc;
    q.in_bs[0] = q.in_bs[1] = N;
    q.nout = 6;
    for (int o = 0; o < 6; ++o) {
      q.out[o] = scratch + (long long)o * npc * B;
      q.out_bs[o] = npc;
      q.nt[o] = 1;
    }
    q.t[0][0] = {0, S_, al};  // y1: M1 [alpha S2 w1]
    q.t[1][0] = {0, M_, be};  //     S1 [beta M2 w1]
    q.t[2][0] = {1, A_, ga};  //     A1 [gamma A2 w2]
    q.t[3][0] = {1, S_, be};  // y2: M1 [beta S2 w2]
    q.t[4][0] = {1, M_, al};  //     S1 [alpha M2 w2]
    q.t[5][0] = {0, A_, ga};  //     A1 [gamma A2 w1]
    aniso_pass_kernel<T><<<grid, 256, 0, s>>>(q, npc, strd(1), ma[1], P, band[1], c.alpha, c.beta,
                                              active);
    AxisParams<T> r{};
    for (int i = 0; i < 6; ++i) {
      r.in[i] = scratch + (long long)i * npc * B;
      r.in_bs[i] = npc;
    }
    r.nout = 2;
    for (int comp = 0; comp < 2; ++comp) {
      r.out[comp] = yt + comp * npc;
      r.out_bs[comp] = N;
      r.nt[comp] = 3;
      r.t[comp][0] = {comp * 3 + 0, M_, 0};
      r.t[comp][1] = {comp * 3 + 1, S_, 0};
      r.t[comp][2] = {comp * 3 + 2, A_, 0};
    }
    aniso_pass_kernel<T><<<grid, 256, 0, s>>>(r, npc, strd(0), ma[0], P, band[0], c.alpha, c.beta,
                                              active);
    count_launch(2);
  } else {
    T* Tm = scratch;
    T* Pm = scratch + 9LL * npc * B;
    AxisParams<T> a{};
    for (int comp = 0; comp < 3; ++comp) {
      a.in[comp] = w + comp * npc;
      a.in_bs[comp] = N;
    }
    a.nout = 9;
    for (int X = 0; X < 3; ++X)
      for (int comp = 0; comp < 3; ++comp) {
        const int o = X * 3 + comp;
        a.out[o] = Tm + (long long)o * npc * B;
        a.out_bs[o] = npc;
        a.nt[o] = 1;
        a.t[o][0] = AxisTerm{comp, X, 0};
      }
    aniso_pass_kernel<T><<<grid, 256, 0, s>>>(a, npc, strd(2), ma[2], P, band[2], c.alpha, c.beta,
                                              active);
    AxisParams<T> q{};
    for (int i = 0; i < 9; ++i) {
      q.in[i] = Tm + (long long)i * npc * B;
      q.in_bs[i] = npc;
    }
    auto TI = [](int X, int comp) { return X * 3 + comp; };
    q.nout = 9;
    for (int o = 0; o < 9; ++o) {
      q.out[o] = Pm + (long long)o * npc * B;
      q.out_bs[o] = npc;
    }
    q.nt[0] = 2; q.t[0][0] = {TI(S_, 0), M_, al}; q.t[0][1] = {TI(M_, 0), S_, al};
    q.nt[1] = 1; q.t[1][0] = {TI(M_, 0), M_, be};
    q.nt[2] = 2; q.t[2][0] = {TI(M_, 1), A_, ga}; q.t[2][1] = {TI(A_, 2), M_, ga};
    q.nt[3] = 3; q.t[3][0] = {TI(S_, 1), M_, al}; q.t[3][1] = {TI(M_, 1), S_, be};
    q.t[3][2] = {TI(A_, 2), A_, ga};
    q.nt[4] = 1; q.t[4][0] = {TI(M_, 1), M_, al};
    q.nt[5] = 1; q.t[5][0] = {TI(M_, 0), A_, ga};
    q.nt[6] = 3; q.t[6][0] = {TI(M_, 2), S_, al}; q.t[6][1] = {TI(S_, 2), M_, be};
    q.t[6][2] = {TI(A_, 1), A_, ga};
    q.nt[7] = 1; q.t[7][0] = {TI(M_, 2), M_, al};
    q.nt[8] = 1; q.t[8][0] = {TI(A_, 0), M_, ga};
    aniso_pass_kernel<T><<<grid, 256, 0, s>>>(q, npc, strd(1), ma[1], P, band[1], c.alpha, c.beta,
                                              active);
    AxisParams<T> r{};
    for (int i = 0; i < 9; ++i) {
      r.in[i] = Pm + (long long)i * npc * B;
      r.in_bs[i] = npc;
    }
    r.nout = 3;
    for (int comp = 0; comp < 3; ++comp) {
      r.out[comp] = yt + comp * npc;
      r.out_bs[comp] = N;
      r.nt[comp] = 3;
      r.t[comp][0] = {comp * 3 + 0, M_, 0};
      r.t[comp][1] = {comp * 3 + 1, S_, 0};
      r.t[comp][2] = {comp * 3 + 2, A_, 0};
    }
    aniso_pass_kernel<T><<<grid, 256, 0, s>>>(r, npc, strd(0), ma[0], P, band[0], c.alpha, c.beta,
                                              active);
    count_launch(3);
  }
  const int nb = partial_blocks(N);
  if (dotp || mode == 1) {
    post3d_kernel<T><<<dim3(nb, B), 256, 0, s>>>(N, w, yt, y, rhs, mode, active, dotp, 1, P,
                                                  band[0], c.alpha, c.beta, Epi<T>{});
    count_launch();
  }
  if (nblk) *nblk = nb;
  return 0;
}
template int launch_apply_aniso<double>(int, const int*, int, const double* const*, const double*,
                                        double*, const double*, int, int, Coef, double*, int*,
                                        const int*, double*, cudaStream_t);
template int launch_apply_aniso<float>(int, const int*, int, const float* const*, const float*,
                                       float*, const float*, int, int, Coef, double*, int*,
                                       const int*, float*, cudaStream_t);

// z = s .* z with s = 1 / sum_l c_{comp,l} lambda_l[k_l] (the FD-D scaling of an anisotropic
// mesh: c_{comp,l} = beta where l = comp, else alpha; lambda_l the generalized eigenvalues of
// direction l), z in the eigen-coordinates of every direction.
template <typename T>
__global__ void __launch_bounds__(256) fd_scale_aniso_kernel(int d, int m0, int m1, int m2,
                                                             const T* __restrict__ lam0,
                                                             const T* __restrict__ lam1,
                                                             const T* __restrict__ lam2,
                                                             const double* __restrict__ alpha,
                                                             const double* __restrict__ beta,
                                                             T* __restrict__ z,
                                                             const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int npc = m0 * m1 * (d == 3 ? m2 : 1);
  const int N = d * npc;
  const double al = alpha[b], be = beta[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int comp = i / npc;
    int rem = i - comp * npc;
    double lam[3];
    if (d == 2) {
      lam[0] = (double)lam0[rem / m1];
      lam[1] = (double)lam1[rem % m1];
    } else {
      lam[0] = (double)lam0[rem / (m1 * m2)];
      lam[1] = (double)lam1[(rem / m2) % m1];
      lam[2] = (double)lam2[rem % m2];
    }
    double den = 0.0;
    for (int l = 0; l < d; ++l) {
      // the term with S along x_l: its eigenvalue lambda_l, M elsewhere (eigenvalue 1)
      den += (l == comp ? be : al) * lam[l];
    }
    z[(long long)b * N + i] = (T)((double)z[(long long)b * N + i] / den);
  }
}

int partial_blocks(long long N) {
  long long nb = (N + 4095) / 4096;
  return (int)std::max<long long>(1, std::min<long long>(nb, 256));
}

template <typename T>
size_t apply2d_smem(int m, int P, int TR) {
  return sizeof(T) * ((size_t)3 * m * (2 * P + 1) + (size_t)2 * (TR + 2 * P) * m + (size_t)6 * TR * m);
}

static constexpr size_t kApplySmemCap = 200 * 1024;

// ---- autotuning table of the 2D apply: (precision bytes, m, P) -> variant
// 1 = v3 with 16-row tiles, 2 = v3 with 8-row tiles, 3 = v2, 4 = v1 (0 = not tuned).
// The tuner chooses between tilings of one algorithm (FP32: v3 with 16 or 8 rows per tile), which
// compute every output of the apply with the same operations in the same order.  The fused
// dot partials are grouped by tile, so a Krylov iterate can differ in its last bits between the
// two tilings; the choice is made once per (precision, m, p) and process, so within a process
// solves stay bit-identical across handles and batch sizes.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned;
static int tuned_variant(size_t es, int m, int P, int /*B*/) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple((int)es, m, P));
  return it == g_tuned.end() ? 0 : it->second;
}
int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      return v;
    cudaGetLastError();
    return 148;
  }();
  return n;
}
static std::atomic<int> g_use_v2{2};  // 2: v5 then v3 kernel (FP32), 3: v3 only, 1: v2 kernel, 0: v1 kernel
void set_apply_variant(int v) { g_use_v2 = v; }
static std::atomic<int> g_fp64_v3{0};    // FP64 2D apply: 0 = v2 (default), 1 = v3 (8 rows per tile)
static std::atomic<int> g_ff_forced{0};  // 1: every FP64 2D apply in double-FP32 (kernel checks)
static std::atomic<int> g_ff_kernel{2};  // double-FP32 2D apply: 2 = packed folded kernel, 1 = plain kernel
void set_apply_fp64_variant(int v) {
  g_fp64_v3 = v == 1;
  g_ff_forced = v == 2 || v == 3 || v == 4;
  g_ff_kernel = v == 4 ? 1 : 2;
}
// 3D designs.  g_use_pass3d: 1 = tuned pass kernels (FP64: generic axis passes), 2 = tuned pass
// kernels in FP64 too, 0 = generic axis passes only.  g_stream_forced: the streaming kernel
// whenever it applies (FP32, P <= 4).
static std::atomic<int> g_use_pass3d{1};
static std::atomic<int> g_stream_forced{0};
// 0: passes, 1: automatic (the autotuner may choose the streaming kernel), 2: generic axis
// passes, 3: streaming kernel forced, 4: tuned passes in FP64 as well
void set_apply3d_variant(int v) {
  g_use_stream3d = v == 1 || v == 3;
  g_stream_forced = v == 3;
  g_use_pass3d = v == 2 ? 0 : v == 4 ? 2 : 1;
}

static thread_local int g_ff_inner = 0;  // the calling thread's FP64 applies run in double-FP32
void set_fp64_emulated(int on) { g_ff_inner = on; }
int fp64_emulated() { return g_ff_inner || g_ff_forced; }

int prepare_kernels() {
  set_stream3d_attr<float, 1>(); set_stream3d_attr<float, 2>(); set_stream3d_attr<float, 3>();
  set_stream3d_attr<float, 4>();
  set_v3_attrs<float, 1>(); set_v3_attrs<float, 2>(); set_v3_attrs<float, 3>();
  set_v3_attrs<float, 4>(); set_v3_attrs<float, 5>(); set_v3_attrs<float, 6>();
  set_v3_attrs<double, 1>(); set_v3_attrs<double, 2>(); set_v3_attrs<double, 3>();
  set_v3_attrs<double, 4>(); set_v3_attrs<double, 5>(); set_v3_attrs<double, 6>();
  set_v2_attrs<float, 1>(); set_v2_attrs<float, 2>(); set_v2_attrs<float, 3>();
  set_v2_attrs<float, 4>(); set_v2_attrs<float, 5>(); set_v2_attrs<float, 6>();
  set_v2_attrs<double, 1>(); set_v2_attrs<double, 2>(); set_v2_attrs<double, 3>();
  set_v2_attrs<double, 4>(); set_v2_attrs<double, 5>(); set_v2_attrs<double, 6>();
  set_v5_attr<1>(); set_v5_attr<2>(); set_v5_attr<3>();
  set_v5_attr<4>(); set_v5_attr<5>(); set_v5_attr<6>();
  prepare_ff_kernels();
  cudaError_t e1 = cudaFuncSetAttribute(apply2d_kernel<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplySmemCap);
  cudaError_t e2 = cudaFuncSetAttribute(apply2d_kernel<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplySmemCap);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : 1;
}

template <typename T>
int launch_apply(int d, int m, int P, const T* bands, const T* w, T* y, const T* rhs, int mode,
                 int B, Coef c, double* dotp, int* nblk, const int* active, T* scratch,
                 cudaStream_t s, const Epi<T>* epi) {
  // Very large grids have more tiles than dot-partial slots: the apply then runs without its
  // fused partials and the fixed-order dot kernel supplies them (per solve, independent of the
  // batch, like the fused ones).
  if (dotp && mode != 2) {
    const long long tiles = d == 2 ? (long long)((m + 63) / 64) * ((m + 7) / 8)
                                   : (long long)((m + 31) / 32) * ((m + 7) / 8) * ((m + 31) / 32);
    if (tiles > kMaxPartials) {
      const int r = launch_apply<T>(d, m, P, bands, w, y, rhs, mode, B, c, nullptr, nullptr,
                                    active, scratch, s, epi);
      if (r != 0) return r;
      const long long N = d == 2 ? 2LL * m * m : 3LL * m * m * m;
      const int nb = partial_blocks(N);
      launch_dot<T>(mode == 1 ? y : w, y, N, B, dotp, nb, active, s);
      if (nblk) *nblk = nb;
      return 0;
    }
  }
  if (mode == 2) {
    if (!epi) return 1;
    g_epi<T> = *epi;
  } else {
    g_epi<T> = Epi<T>{};
  }
  if (d == 2) {
    if constexpr (sizeof(T) == 8) {
      if (fp64_emulated() &&
          try_apply2d_ff(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s, g_epi<double>,
                         g_ff_kernel))
        return 0;
    }
    if (sizeof(T) == 8 && g_use_v2 == 2 && g_fp64_v3 &&
        try_apply2d_v3<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s, 8))
      return 0;
    int tuned = g_use_v2 == 2 ? tuned_variant(sizeof(T), m, P, B) : 0;
    if constexpr (sizeof(T) == 4) {
      if (tuned == 5 && try_apply2d_v5(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
        return 0;
    }
    if (tuned == 1 && try_apply2d_v3<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s, 16))
      return 0;
    if (tuned == 2 && try_apply2d_v3<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s, 8))
      return 0;
    if (tuned == 3 && try_apply2d_v2<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
      return 0;
    if (tuned == 4 && mode != 2) goto plain_v1;
    // FP32: v5, then v3 (packed pairs); FP64: v2 first (v3's FP64 instantiation is register-bound)
    if constexpr (sizeof(T) == 4) {
      if (g_use_v2 == 2 && tuned == 0 &&
          try_apply2d_v5(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
        return 0;
    }
    if (g_use_v2 >= 2 && sizeof(T) == 4 &&
        try_apply2d_v3<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
      return 0;
    if (g_use_v2 >= 1 && try_apply2d_v2<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
      return 0;
    if (g_use_v2 >= 1 && try_apply2d_v3<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s))
      return 0;
  plain_v1:
    if (mode == 2) return 1;  // the plain kernel has no fused smoother epilogue
    int TR = sizeof(T) == 8 ? 4 : 8;
    while (TR > 1 && apply2d_smem<T>(m, P, TR) > kApplySmemCap) TR /= 2;
    size_t sm = apply2d_smem<T>(m, P, TR);
    if (sm > kApplySmemCap || (dotp && (m + TR - 1) / TR > kMaxPartials)) return 1;  // too large for v1
    dim3 grid((m + TR - 1) / TR, B);
    apply2d_kernel<T><<<grid, 256, sm, s>>>(m, P, TR, bands, w, y, rhs, mode, c.alpha, c.beta, c.gsc,
                                            active, dotp);
    count_launch();
    if (nblk) *nblk = grid.x;
    return 0;
  }
  const bool emu3 = sizeof(T) == 8 && fp64_emulated();
  const int v3d = sizeof(T) == 4 ? tuned3d_variant(sizeof(T), m, P) : 0;
  // the streaming kernel when forced or tuned to it; otherwise the passes (FP32: the tuned pass
  // kernels, measured faster at every size tried; FP64: the generic axis passes, which run at
  // the FP64 rate; double-FP32 when the caller's FP64 applies are emulated)
  if (!emu3 && (g_stream_forced || v3d == 1) &&
      try_stream3d<T>(m, P, bands, w, y, rhs, mode, B, c, dotp, nblk, active, s, g_epi<T>))
    return 0;
  const long long N = 3LL * m * m * m;
  T* ytmp = mode >= 1 ? scratch + 18LL * (N / 3) * B : y;
  bool done = false;
  if (g_use_pass3d) {
    if constexpr (sizeof(T) == 8) {
      if (emu3)
        done = launch_pass3d_ff(m, P, bands, w, ytmp, B, c, active,
                                reinterpret_cast<float2*>(scratch), s);
      else if (g_use_pass3d == 2)
        done = launch_pass3d_f64(m, P, bands, w, ytmp, B, c, active, scratch, s);
    } else {
      done = launch_pass3d_f32(m, P, bands, w, ytmp, B, c, active, scratch, s);
    }
  }
  if (!done) apply3d_multipass<T>(m, P, bands, w, ytmp, B, c, active, scratch, s);
  const int nb = partial_blocks(N);
  if (dotp || mode >= 1) {
    post3d_kernel<T><<<dim3(nb, B), 256, 0, s>>>(N, w, ytmp, y, rhs, mode, active, dotp, m, P,
                                                  bands, c.alpha, c.beta, g_epi<T>);
    count_launch();
  }
  if (nblk) *nblk = nb;
  return 0;
}

template int launch_apply<double>(int, int, int, const double*, const double*, double*,
                                  const double*, int, int, Coef, double*, int*, const int*,
                                  double*, cudaStream_t, const Epi<double>*);
template int launch_apply<float>(int, int, int, const float*, const float*, float*, const float*,
                                 int, int, Coef, double*, int*, const int*, float*, cudaStream_t,
                                 const Epi<float>*);

// ------------------------------------------------------------------ reductions and vectors
template <typename T, typename U>
__global__ void __launch_bounds__(256) dot_kernel(long long N, const T* __restrict__ a,
                                                  const U* __restrict__ bv,
                                                  const int* __restrict__ active,
                                                  double* __restrict__ part) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long chunk = (N + gridDim.x - 1) / gridDim.x;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const long long base = (long long)b * N;
  double acc = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    acc += (double)a[base + i] * (double)bv[base + i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = s;
}

template <typename T>
int launch_dot(const T* a, const T* b, long long N, int B, double* part, int nblk,
               const int* active, cudaStream_t s) {
  dot_kernel<T, T><<<dim3(nblk, B), 256, 0, s>>>(N, a, b, active, part);
  count_launch();
  return 0;
}
template int launch_dot<double>(const double*, const double*, long long, int, double*, int,
                                const int*, cudaStream_t);
template int launch_dot<float>(const float*, const float*, long long, int, double*, int,
                               const int*, cudaStream_t);

__global__ void sum_partials_kernel(const double* __restrict__ part, int nblk, int B,
                                    double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[(size_t)b * nblk + i];
  out[b] = s;
}

int launch_sum_partials(const double* part, int nblk, int B, double* out, cudaStream_t s) {
  sum_partials_kernel<<<(B + 127) / 128, 128, 0, s>>>(part, nblk, B, out);
  count_launch();
  return 0;
}

// Times the applicable 2D apply tilings on (m, P, B) with CUDA events on stream s (w, y:
// B-vector buffers; the call must not be inside a stream capture) and records the fastest.
template <typename T>
int tune_apply2d(int m, int P, const T* bands, const T* w, T* y, int B, Coef c, cudaStream_t s) {
  if (g_use_v2 != 2) return 0;
  const auto key = std::make_tuple((int)sizeof(T), m, P);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;  // first tuning of this shape sticks
  }
  if (sizeof(T) == 8) {  // FP64: v2 (no equivalent tiling alternative to time)
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = 3;
    return 3;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 0;
  float best = 1e30f;
  int bestv = 0;
  for (int v : {5, 1, 2}) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = v;
    }
    for (int rep = 0; rep < 2; ++rep)  // warm-up (and first-launch set-up)
      launch_apply<T>(2, m, P, bands, w, y, nullptr, 0, B, c, nullptr, nullptr, nullptr, nullptr, s);
    cudaEventRecord(e0, s);
    int bad = 0;
    for (int rep = 0; rep < 3; ++rep)
      bad |= launch_apply<T>(2, m, P, bands, w, y, nullptr, 0, B, c, nullptr, nullptr, nullptr, nullptr, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (bad == 0 && ms < best) {
      best = ms;
      bestv = v;
    }
  }
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = bestv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return bestv;
}
template int tune_apply2d<float>(int, int, const float*, const float*, float*, int, Coef, cudaStream_t);

// Times the two 3D apply designs (the streaming kernel, where it exists for this precision and
// P, and the three banded passes) on (m, P, B) with CUDA events on stream s and records the
// faster; both compute y = A w, the passes in a different summation order.  Not inside a stream
// capture.  Returns the chosen variant (1 streaming, 2 passes).
template <typename T>
int tune_apply3d(int m, int P, const T* bands, const T* w, T* y, int B, Coef c, T* scratch,
                 cudaStream_t s) {
  const auto key = std::make_tuple((int)sizeof(T), m, P);
  {
    std::lock_guard<std::mutex> lk(g_tune3d_mu);
    auto it = g_tuned3d.find(key);
    if (it != g_tuned3d.end()) return it->second;
  }
  if (sizeof(T) == 8 || P > 4 || !g_use_stream3d) {  // only the passes exist here
    std::lock_guard<std::mutex> lk(g_tune3d_mu);
    g_tuned3d[key] = 2;
    return 2;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 0;
  float best = 1e30f;
  int bestv = 0;
  for (int v = 1; v <= 2; ++v) {
    {
      std::lock_guard<std::mutex> lk(g_tune3d_mu);
      g_tuned3d[key] = v;
    }
    for (int rep = 0; rep < 2; ++rep)
      launch_apply<T>(3, m, P, bands, w, y, nullptr, 0, B, c, nullptr, nullptr, nullptr, scratch, s);
    cudaEventRecord(e0, s);
    int bad = 0;
    for (int rep = 0; rep < 3; ++rep)
      bad |= launch_apply<T>(3, m, P, bands, w, y, nullptr, 0, B, c, nullptr, nullptr, nullptr,
                             scratch, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (bad == 0 && ms < best) {
      best = ms;
      bestv = v;
    }
  }
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_tune3d_mu);
    g_tuned3d[key] = bestv ? bestv : 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return bestv;
}
template int tune_apply3d<float>(int, int, const float*, const float*, float*, int, Coef,
                                 float*, cudaStream_t);
template int tune_apply3d<double>(int, int, const double*, const double*, double*, int, Coef,
                                  double*, cudaStream_t);
template int tune_apply2d<double>(int, int, const double*, const double*, double*, int, Coef, cudaStream_t);

// Whether launch_apply supports mode 2 (fused smoother epilogue) for this level and batch.
template <typename T>
bool apply_can_fuse(int d, int m, int P, const T* bands, int B) {
  if (d == 3) return true;
  if (g_use_v2 < 1 || P < 1 || P > 6) return false;
  StencilHost sh;
  if (!find_level(bands, sh)) return false;
  return tuned_variant(sizeof(T), m, P, B) != 4;
}
template bool apply_can_fuse<float>(int, int, int, const float*, int);
template bool apply_can_fuse<double>(int, int, int, const double*, int);

}  // namespace cd

namespace cd {
template <typename T>
void launch_fd_scale_aniso(int d, const int* ma, const T* const* lam, int B, const double* alpha,
                           const double* beta, T* z, const int* active, cudaStream_t s) {
  const long long N = (long long)d * ma[0] * ma[1] * (d == 3 ? ma[2] : 1);
  const dim3 grid((unsigned)std::min<long long>((N + 255) / 256, 4096), B);
  fd_scale_aniso_kernel<T><<<grid, 256, 0, s>>>(d, ma[0], ma[1], d == 3 ? ma[2] : 1, lam[0], lam[1],
                                                d == 3 ? lam[2] : lam[1], alpha, beta, z, active);
  count_launch();
}
template void launch_fd_scale_aniso<double>(int, const int*, const double* const*, int,
                                            const double*, const double*, double*, const int*,
                                            cudaStream_t);
template void launch_fd_scale_aniso<float>(int, const int*, const float* const*, int, const double*,
                                           const double*, float*, const int*, cudaStream_t);
}  // namespace cd
