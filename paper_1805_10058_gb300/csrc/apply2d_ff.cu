// The 2D operator apply in double-FP32 arithmetic: FP64 vectors, every product and sum of the
// sum-factorised stencil (the Kronecker form of the 2D block matrix, Section 4.1, eq:matr_Amu)
// carried as an unevaluated sum of two FP32 numbers on the FP32 pipe.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "apply_shared.h"
#include "ffmath.h"

namespace cd {

// ------------------------------------------------------------------ 2D apply in double-FP32
// FP64 vectors, arithmetic in double-FP32 ("float-float": an unevaluated sum hi + lo of two FP32
// numbers, about 48 significant bits) on the FP32 pipe, which on GB300 issues 64 times the FP64
// rate.  Each FP64 input element of the tile is split once into (hi, lo) in shared memory; every
// product is an FMA two-product with the cross terms, every sum a two-sum (non-contracting _rn
// intrinsics); the x_2 results, scaled and grouped as in the FP32 kernel (PM, PS, PA), stay in
// shared memory as (hi, lo) pairs, and the x_1 pass forms y in double-FP32 and rounds it to FP64.
// Accuracy: about 1e-13 of (|A| |w|)_i, 30x coarser than FP64, used for the inner Krylov solves
// of the refinement loop (whose double-FP64 outer residual removes it).
struct StencilFF {
  float2 c[3][13];
  int lo, hi;
};


template <int P, int TR>
__global__ void __launch_bounds__(256, 2) apply2d_ff_kernel(
    int m, const float2* __restrict__ bandF, StencilFF cs, const double* __restrict__ w,
    double* __restrict__ y, const double* __restrict__ rhs, int mode,
    const double* __restrict__ alpha, const double* __restrict__ beta,
    const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<double> epi) {
  constexpr int W = 2 * P + 1, TC = 64, HR = TR + 2 * P, HC = TC + 2 * P;
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sw = reinterpret_cast<float2*>(smem_raw);  // [2][HR][HC] input tile, (hi, lo)
  float2* sp = sw + 2 * HR * HC;                      // [3][2][HR][TC] intermediates
  const long long N = 2LL * m * m;
  const double* wb = w + (long long)b * N;
  const int c0 = blockIdx.x * TC, r0 = blockIdx.y * TR;
  const float2 al = ff_split(alpha[b]), be = ff_split(beta[b]);
  const float2 ga = ff_split((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  const float2* BM = bandF;
  const float2* BA = bandF + (size_t)W * m;
  const float2* BS = bandF + (size_t)2 * W * m;
  // tile of w with halos, split once
  for (int idx = threadIdx.x; idx < 2 * HR * HC; idx += blockDim.x) {
    const int c = idx / (HR * HC), rem = idx - c * HR * HC;
    const int rr = rem / HC, cc = rem - rr * HC;
    const int row = r0 - P + rr, col = c0 - P + cc;
    float2 v = make_float2(0.f, 0.f);
    if (row >= 0 && row < m && col >= 0 && col < m)
      v = ff_split_bits(wb[(long long)c * m * m + (long long)row * m + col]);
    sw[idx] = v;
  }
  __syncthreads();
  // axis x_2 for rows r0-P .. r0+TR+P-1: S2, M2, A2 of both components, scaled and grouped
  for (int item = threadIdx.x; item < HR * TC; item += blockDim.x) {
    const int q = item / TC, cc = item - q * TC;
    const int row = r0 - P + q, j = c0 + cc;
    float2 tM[2], tA[2], tS[2];
    for (int c = 0; c < 2; ++c) tM[c] = tA[c] = tS[c] = make_float2(0.f, 0.f);
    if (row >= 0 && row < m && j < m) {
      const bool interior = j >= cs.lo && j < cs.hi;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        float2 cM, cA, cS;
        if (interior) {
          cM = cs.c[0][k];
          cA = cs.c[1][k];
          cS = cs.c[2][k];
        } else {
          cM = BM[(size_t)k * m + j];
          cA = BA[(size_t)k * m + j];
          cS = BS[(size_t)k * m + j];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 v = sw[(c * HR + q) * HC + cc + k];
          ff_fma(tM[c], cM, v);
          ff_fma(tA[c], cA, v);
          ff_fma(tS[c], cS, v);
        }
      }
      for (int c = 0; c < 2; ++c) {
        tM[c] = ff_norm(tM[c]);
        tA[c] = ff_norm(tA[c]);
        tS[c] = ff_norm(tS[c]);
      }
    }
    // PM = (alpha S2 w1, beta S2 w2) feeds M1; PS = (beta M2 w1, alpha M2 w2) feeds S1;
    // PA = gamma (A2 w2, A2 w1) feeds A1
    sp[((0 * 2 + 0) * HR + q) * TC + cc] = ff_mul(al, tS[0]);
    sp[((0 * 2 + 1) * HR + q) * TC + cc] = ff_mul(be, tS[1]);
    sp[((1 * 2 + 0) * HR + q) * TC + cc] = ff_mul(be, tM[0]);
    sp[((1 * 2 + 1) * HR + q) * TC + cc] = ff_mul(al, tM[1]);
    sp[((2 * 2 + 0) * HR + q) * TC + cc] = ff_mul(ga, tA[1]);
    sp[((2 * 2 + 1) * HR + q) * TC + cc] = ff_mul(ga, tA[0]);
  }
  __syncthreads();
  // axis x_1: y_c = M1 PM_c + S1 PS_c + A1 PA_c
  double acc = 0.0, ec1 = 0.0, ec2 = 0.0;
  if (mode == 2) cheb_coef_cta(epi.lmax[b], epi.step, ec1, ec2);
  for (int item = threadIdx.x; item < TR * TC; item += blockDim.x) {
    const int r = item / TC, cc = item - r * TC;
    const int i = r0 + r, j = c0 + cc;
    if (i >= m || j >= m) continue;
    const bool interior = i >= cs.lo && i < cs.hi;
    float2 yy[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int k = 0; k < W; ++k) {
      float2 cM, cA, cS;
      if (interior) {
        cM = cs.c[0][k];
        cA = cs.c[1][k];
        cS = cs.c[2][k];
      } else {
        cM = BM[(size_t)k * m + i];
        cA = BA[(size_t)k * m + i];
        cS = BS[(size_t)k * m + i];
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        ff_fma(yy[c], cM, sp[((0 * 2 + c) * HR + r + k) * TC + cc]);
        ff_fma(yy[c], cS, sp[((1 * 2 + c) * HR + r + k) * TC + cc]);
        ff_fma(yy[c], cA, sp[((2 * 2 + c) * HR + r + k) * TC + cc]);
      }
    }
    const long long o1 = (long long)b * N + (long long)i * m + j, o2 = o1 + (long long)m * m;
    double y1 = ff_to_double(ff_norm(yy[0])), y2 = ff_to_double(ff_norm(yy[1]));
    if (mode == 2) {  // fused Chebyshev step with the stored 1 / diag(A)
      cheb_epi(epi, o1, rhs[o1] - y1, epi.dinv[o1], ec1, ec2);
      cheb_epi(epi, o2, rhs[o2] - y2, epi.dinv[o2], ec1, ec2);
      continue;
    }
    if (mode == 1) {
      y1 = rhs[o1] - y1;
      y2 = rhs[o2] - y2;
      if (dotp) acc += y1 * y1 + y2 * y2;
    } else if (dotp) {
      acc += w[o1] * y1 + w[o2] * y2;
    }
    y[o1] = y1;
    y[o2] = y2;
  }
  if (dotp) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0)
      dotp[(size_t)b * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

template <int P, int TR>
static size_t ff_smem() {
  return sizeof(float2) * ((size_t)2 * (TR + 2 * P) * (64 + 2 * P) + (size_t)6 * (TR + 2 * P) * 64);
}
template <int P, int TR>
static void set_ff_attr() {
  cudaFuncSetAttribute(apply2d_ff_kernel<P, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ff_smem<P, TR>());
}

template <int P>
static bool launch_ff_P(int m, const double* bands, const StencilHost& sh, const double* w, double* y,
                        const double* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                        const int* active, cudaStream_t s, const Epi<double>& epi) {
  constexpr int TR = 16;
  StencilFF cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) {
      const double v = k < 2 * P + 1 ? sh.c[x][k] : 0.0;
      const float h = (float)v;
      cs.c[x][k] = make_float2(h, (float)(v - (double)h));
    }
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  dim3 grid((m + 63) / 64, (m + TR - 1) / TR, B);
  apply2d_ff_kernel<P, TR><<<grid, 256, ff_smem<P, TR>(), s>>>(
      m, sh.ffT, cs, w, y, rhs, mode, c.alpha, c.beta, c.gsc, active, dotp, epi);
  count_launch();
  if (nblk) *nblk = grid.x * grid.y;
  return true;
}

// ------------------------------------------------------------------ 2D apply in double-FP32, v2
// The same operator and arithmetic type as apply2d_ff_kernel, rebuilt for issue rate:
//  * the two components of a grid point travel together as packed pairs, so every double-FP32
//    step is a packed FP32 instruction (FFMA2 / FADD2 / FMUL2) acting on (w1, w2) at once;
//  * in the interior, where the bands equal their central rows, the symmetric M and S and the
//    skew A are applied in folded form: c_0 x_0 + sum_t c_t (x_{-t} +- x_{+t}), the pair sums
//    shared by M and S along x_2 (about 2/3 of the double-FP32 multiply-adds of the plain form);
//  * shared memory rows have an odd number of 16-byte slots, so the column-wise x_2 pass (lanes
//    = rows) and the row-wise x_1 pass (lanes = columns) are both free of bank conflicts.
// Tile: TR = 24 (P <= 4) or 20 output rows x 32 columns per CTA of 128 threads; the x_2 pass
// covers the TR + 2P <= 32 rows of the halo, one row per lane.  The narrow variant (TR = 8, for
// grids too small to fill the GPU with wide tiles) hands the x_2 pass's (halo row, column group)
// pairs to all 128 threads, so a CTA's serial chain is about a third as long.
struct FF2 {  // two double-FP32 numbers: (h.x + l.x, h.y + l.y)
  float2 h, l;
};
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {  // a - b, one rounding
  return __ffma2_rn(b, f2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, f2(-1.f, -1.f)); }
// acc += c * x, c = ch + cl per lane
__device__ __forceinline__ void ff2_fma(FF2& acc, float2 ch, float2 cl, const FF2& x) {
  const float2 p = __fmul2_rn(ch, x.h);
  float2 e = __ffma2_rn(ch, x.h, neg2(p));
  e = __ffma2_rn(ch, x.l, e);
  e = __ffma2_rn(cl, x.h, e);
  const float2 sm = __fadd2_rn(acc.h, p);
  const float2 bb = sub2(sm, acc.h);
  const float2 er = __fadd2_rn(sub2(acc.h, sub2(sm, bb)), sub2(p, bb));
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(er, e));
  acc.h = sm;
}
// a + b and a - b (two-sum of the high parts; low parts added)
__device__ __forceinline__ FF2 ff2_add(const FF2& a, const FF2& b) {
  const float2 sm = __fadd2_rn(a.h, b.h);
  const float2 bb = sub2(sm, a.h);
  const float2 er = __fadd2_rn(sub2(a.h, sub2(sm, bb)), sub2(b.h, bb));
  return FF2{sm, __fadd2_rn(__fadd2_rn(a.l, b.l), er)};
}
__device__ __forceinline__ FF2 ff2_sub(const FF2& a, const FF2& b) {
  const float2 sm = sub2(a.h, b.h);
  const float2 bb = sub2(sm, a.h);
  const float2 er = sub2(sub2(a.h, sub2(sm, bb)), __fadd2_rn(b.h, bb));
  return FF2{sm, __fadd2_rn(sub2(a.l, b.l), er)};
}
__device__ __forceinline__ FF2 ff2_norm(const FF2& a) {
  const float2 sm = __fadd2_rn(a.h, a.l);
  return FF2{sm, sub2(a.l, sub2(sm, a.h))};
}
// (ch + cl) * x, normalised
__device__ __forceinline__ FF2 ff2_mul(float2 ch, float2 cl, const FF2& x) {
  const float2 p = __fmul2_rn(ch, x.h);
  float2 e = __ffma2_rn(ch, x.h, neg2(p));
  e = __ffma2_rn(ch, x.l, e);
  e = __ffma2_rn(cl, x.h, e);
  return ff2_norm(FF2{p, e});
}
__device__ __forceinline__ FF2 ld_ff2(const float4* p) {
  const float4 v = *p;
  return FF2{f2(v.x, v.y), f2(v.z, v.w)};
}
__device__ __forceinline__ void st_ff2(float4* p, const FF2& a) {
  *p = make_float4(a.h.x, a.h.y, a.l.x, a.l.y);
}

struct StencilFF2 {
  float c[3][2][13];  // [M, A, S][hi, lo][offset k = 0..2P], central rows
  int lo, hi;
};

template <int P, int TRV = 0>
struct FF2Tile {
  static constexpr int W = 2 * P + 1;
  static constexpr int TC = 32;
  static constexpr int TR = TRV ? TRV : P <= 4 ? 24 : 20;
  static constexpr int HR = TR + 2 * P;           // <= 32
  static constexpr int HC = TC + 2 * P;
  static constexpr int HCP = HC | 1;              // input row stride in float4 slots (odd)
  static constexpr int TCP = TC + 1;              // intermediate row stride (odd)
  static constexpr int NC = 4;                    // columns per lane in the x_2 pass
  static constexpr int RS = TR / 4;               // rows per lane in the x_1 pass
  // input tile | intermediates | band rows of the tile's columns (boundary tiles); the band rows
  // of the tile's rows reuse the input tile's space in the x_1 pass
  static constexpr size_t off_mid = sizeof(float4) * HR * HCP;
  static constexpr size_t off_col = off_mid + sizeof(float4) * 3 * HR * TCP;
  static constexpr size_t smem = off_col + sizeof(float2) * 3 * W * TC;
  static_assert(sizeof(float2) * 3 * W * TR <= off_mid, "row coefficients fit the input tile");
};

// y (or the residual, or the fused Chebyshev step) at one grid point from its double-FP32 pair
__device__ __forceinline__ void ff2_emit(const FF2& yy, long long o1, long long o2, int mode,
                                         const double* __restrict__ w, double* __restrict__ y,
                                         const double* __restrict__ rhs, const Epi<double>& epi,
                                         double ec1, double ec2, const double* dotp, double& acc) {
  const FF2 yn = ff2_norm(yy);
  if (mode == 2) {
    // fused Chebyshev step: r = rhs - A w in double-FP32, the correction d = c2 D^{-1} r
    // (+ c1 d_prev) in FP32 (a smoother step needs no more), x = x_prev + d with one FP64 add
    const float2 q1 = ff_split_bits(rhs[o1]), q2 = ff_split_bits(rhs[o2]);
    const FF2 rn = ff2_norm(ff2_sub(FF2{f2(q1.x, q2.x), f2(q1.y, q2.y)}, yn));
    const float c2 = (float)ec2, c1 = (float)ec1;
    float d1 = c2 * ff_split_bits(epi.dinv[o1]).x * rn.h.x;
    float d2 = c2 * ff_split_bits(epi.dinv[o2]).x * rn.h.y;
    if (epi.step > 0) {
      d1 = fmaf(c1, ff_split_bits(epi.dprev[o1]).x, d1);
      d2 = fmaf(c1, ff_split_bits(epi.dprev[o2]).x, d2);
    }
    const double e1 = f2d_bits(d1), e2 = f2d_bits(d2);
    epi.xout[o1] = __dadd_rn(epi.xprev[o1], e1);
    epi.xout[o2] = __dadd_rn(epi.xprev[o2], e2);
    if (epi.dout) {
      epi.dout[o1] = e1;
      epi.dout[o2] = e2;
    }
    if (epi.rout) {
      epi.rout[o1] = __dadd_rn(f2d_bits(rn.h.x), f2d_bits(rn.l.x));
      epi.rout[o2] = __dadd_rn(f2d_bits(rn.h.y), f2d_bits(rn.l.y));
    }
    return;
  }
  double y1 = __dadd_rn(f2d_bits(yn.h.x), f2d_bits(yn.l.x));
  double y2 = __dadd_rn(f2d_bits(yn.h.y), f2d_bits(yn.l.y));
  if (mode == 1) {
    y1 = rhs[o1] - y1;
    y2 = rhs[o2] - y2;
    if (dotp) acc += y1 * y1 + y2 * y2;
  } else if (dotp) {
    acc += w[o1] * y1 + w[o2] * y2;
  }
  y[o1] = y1;
  y[o2] = y2;
}

template <int P, int MODE, int TRV = 0>
__global__ void __launch_bounds__(128, TRV ? 4 : 3) apply2d_ff2_kernel(
    int m, const float2* __restrict__ bandF, StencilFF2 cs, const double* __restrict__ w,
    double* __restrict__ y, const double* __restrict__ rhs, int /*mode: MODE*/,
    const double* __restrict__ alpha, const double* __restrict__ beta,
    const double* __restrict__ gsc, const int* __restrict__ active, double* __restrict__ dotp,
    Epi<double> epi) {
  using G = FF2Tile<P, TRV>;
  constexpr int W = G::W, TC = G::TC, TR = G::TR, HR = G::HR, HC = G::HC, HCP = G::HCP;
  constexpr int TCP = G::TCP, NC = G::NC, RS = G::RS;
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sIn = reinterpret_cast<float4*>(smem_raw);                   // [HR][HCP]
  float4* sMid = reinterpret_cast<float4*>(smem_raw + G::off_mid);     // [3][HR][TCP]
  float2* sCol = reinterpret_cast<float2*>(smem_raw + G::off_col);     // [3][W][TC]
  float2* sRow = reinterpret_cast<float2*>(smem_raw);                  // [3][W][TR] (x_1 pass)
  const long long N = 2LL * m * m;
  const double* wb = w + (long long)b * N;
  const int c0 = blockIdx.x * TC, r0 = blockIdx.y * TR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool bcol = c0 < cs.lo || c0 + TC > cs.hi;  // tile holds non-Toeplitz columns
  const bool brow = r0 < cs.lo || r0 + TR > cs.hi;  // ... or rows
  {  // every load of the tile in flight before the first split (one memory latency per tile)
    constexpr int NE = (HR * HC + 127) / 128;
    double v1[NE], v2[NE];
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int rr = idx / HC, cc = idx - rr * HC;
      const int row = r0 - P + rr, col = c0 - P + cc;
      v1[t] = v2[t] = 0.0;
      if (idx < HR * HC && row >= 0 && row < m && col >= 0 && col < m) {
        const long long o = (long long)row * m + col;
        v1[t] = wb[o];
        v2[t] = wb[(long long)m * m + o];
      }
    }
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int rr = idx / HC, cc = idx - rr * HC;
      const float2 a = ff_split_bits(v1[t]), c = ff_split_bits(v2[t]);
      if (idx < HR * HC) sIn[rr * HCP + cc] = make_float4(a.x, c.x, a.y, c.y);
    }
  }
  if (bcol) {
    constexpr int NK = (3 * W * TC + 127) / 128;
    float2 v[NK];
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int xk = idx / TC, cc = idx - xk * TC;
      v[t] = idx < 3 * W * TC && c0 + cc < m ? bandF[(size_t)xk * m + c0 + cc] : f2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < NK; ++t)
      if (threadIdx.x + 128 * t < 3 * W * TC) sCol[threadIdx.x + 128 * t] = v[t];
  }
  // per-solve scalars as (hi, lo) pairs, split once per CTA (FP64 work stays off the threads)
  __shared__ float2 s_par[3];
  if (threadIdx.x == 0) {
    s_par[0] = ff_split(alpha[b]);
    s_par[1] = ff_split(beta[b]);
    s_par[2] = ff_split((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  }
  __syncthreads();
  const float2 al = s_par[0], be = s_par[1], ga = s_par[2];
  const float2 pmh = f2(al.x, be.x), pml = f2(al.y, be.y);  // PM = (alpha, beta) * S2 w
  const float2 psh = f2(be.x, al.x), psl = f2(be.y, al.y);  // PS = (beta, alpha) * M2 w
  const float2 gah = f2(ga.x, ga.x), gal = f2(ga.y, ga.y);  // PA = gamma * swap(A2 w)
  // ---- axis x_2: one (halo row q, group g of NC consecutive columns) per step; the wide tile
  // puts the rows on the lanes of each warp, the narrow tile spreads the pairs over the CTA
  auto x2_step = [&](const int q, const int g) {
    const int row = r0 - P + q;
    const bool rowok = row >= 0 && row < m;
      const int j0 = c0 + g * NC;
      if (rowok && j0 < m && j0 >= cs.lo && j0 + NC - 1 < cs.hi) {
        FF2 x[NC + 2 * P];
#pragma unroll
        for (int t = 0; t < NC + 2 * P; ++t) x[t] = ld_ff2(&sIn[q * HCP + g * NC + t]);
#pragma unroll
        for (int u = 0; u < NC; ++u) {
          FF2 tM{f2(0.f, 0.f), f2(0.f, 0.f)}, tS = tM, tA = tM;
          const FF2& xc = x[u + P];
          ff2_fma(tM, f2(cs.c[0][0][P], cs.c[0][0][P]), f2(cs.c[0][1][P], cs.c[0][1][P]), xc);
          ff2_fma(tS, f2(cs.c[2][0][P], cs.c[2][0][P]), f2(cs.c[2][1][P], cs.c[2][1][P]), xc);
#pragma unroll
          for (int t = 1; t <= P; ++t) {
            const FF2 sp = ff2_add(x[u + P - t], x[u + P + t]);
            const FF2 dp = ff2_sub(x[u + P + t], x[u + P - t]);
            const int k = P + t;
            ff2_fma(tM, f2(cs.c[0][0][k], cs.c[0][0][k]), f2(cs.c[0][1][k], cs.c[0][1][k]), sp);
            ff2_fma(tS, f2(cs.c[2][0][k], cs.c[2][0][k]), f2(cs.c[2][1][k], cs.c[2][1][k]), sp);
            ff2_fma(tA, f2(cs.c[1][0][k], cs.c[1][0][k]), f2(cs.c[1][1][k], cs.c[1][1][k]), dp);
          }
          const int cc = g * NC + u;
          tS = ff2_norm(tS);
          tM = ff2_norm(tM);
          tA = ff2_norm(tA);
          st_ff2(&sMid[(0 * HR + q) * TCP + cc], ff2_mul(pmh, pml, tS));
          st_ff2(&sMid[(1 * HR + q) * TCP + cc], ff2_mul(psh, psl, tM));
          st_ff2(&sMid[(2 * HR + q) * TCP + cc],
                 ff2_mul(gah, gal, FF2{f2(tA.h.y, tA.h.x), f2(tA.l.y, tA.l.x)}));
        }
      } else {  // boundary columns (band rows staged in shared memory) or outside the domain
#pragma unroll 1
        for (int u = 0; u < NC; ++u) {
          const int cc = g * NC + u;
          FF2 tM{f2(0.f, 0.f), f2(0.f, 0.f)}, tS = tM, tA = tM;
          if (rowok && c0 + cc < m) {
#pragma unroll 1
            for (int k = 0; k < W; ++k) {
              const FF2 xv = ld_ff2(&sIn[q * HCP + cc + k]);
              const float2 cM = sCol[(0 * W + k) * TC + cc], cA = sCol[(1 * W + k) * TC + cc],
                           cS = sCol[(2 * W + k) * TC + cc];
              ff2_fma(tM, f2(cM.x, cM.x), f2(cM.y, cM.y), xv);
              ff2_fma(tA, f2(cA.x, cA.x), f2(cA.y, cA.y), xv);
              ff2_fma(tS, f2(cS.x, cS.x), f2(cS.y, cS.y), xv);
            }
          }
          tS = ff2_norm(tS);
          tM = ff2_norm(tM);
          tA = ff2_norm(tA);
          st_ff2(&sMid[(0 * HR + q) * TCP + cc], ff2_mul(pmh, pml, tS));
          st_ff2(&sMid[(1 * HR + q) * TCP + cc], ff2_mul(psh, psl, tM));
          st_ff2(&sMid[(2 * HR + q) * TCP + cc],
                 ff2_mul(gah, gal, FF2{f2(tA.h.y, tA.h.x), f2(tA.l.y, tA.l.x)}));
        }
      }
  };
  if constexpr (TRV == 0) {
    if (lane < HR)
      for (int g = warp; g < TC / NC; g += 4) x2_step(lane, g);
  } else {
    for (int it = threadIdx.x; it < HR * (TC / NC); it += 128) x2_step(it % HR, it / HR);
  }
  __syncthreads();
  if (brow) {  // band rows of the tile's rows, into the input tile's space
    constexpr int NK = (3 * W * TR + 127) / 128;
    float2 v[NK];
#pragma unroll
    for (int t = 0; t < NK; ++t) {
      const int idx = threadIdx.x + 128 * t;
      const int xk = idx / TR, rr = idx - xk * TR;
      v[t] = idx < 3 * W * TR && r0 + rr < m ? bandF[(size_t)xk * m + r0 + rr] : f2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < NK; ++t)
      if (threadIdx.x + 128 * t < 3 * W * TR) sRow[threadIdx.x + 128 * t] = v[t];
    __syncthreads();
  }
  // ---- axis x_1: lane = column, RS rows per warp: y = M1 PM + S1 PS + A1 PA
  double acc = 0.0, ec1 = 0.0, ec2 = 0.0;
  if (MODE == 2) cheb_coef_cta(epi.lmax[b], epi.step, ec1, ec2);
  const int cc = lane, j = c0 + cc;
  const int rb = warp * RS;
  if (j < m) {
    if (r0 + rb >= cs.lo && r0 + rb + RS - 1 < cs.hi) {
      FF2 yy[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) yy[r] = FF2{f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll 1
      for (int band = 0; band < 2; ++band) {  // M on PM, S on PS (symmetric)
        const int x = band == 0 ? 0 : 2;
        FF2 v[RS + 2 * P];
#pragma unroll
        for (int t = 0; t < RS + 2 * P; ++t) v[t] = ld_ff2(&sMid[(band * HR + rb + t) * TCP + cc]);
        float ch[P + 1], cl[P + 1];
#pragma unroll
        for (int t = 0; t <= P; ++t) {
          ch[t] = x == 0 ? cs.c[0][0][P + t] : cs.c[2][0][P + t];
          cl[t] = x == 0 ? cs.c[0][1][P + t] : cs.c[2][1][P + t];
        }
#pragma unroll
        for (int r = 0; r < RS; ++r) {
          ff2_fma(yy[r], f2(ch[0], ch[0]), f2(cl[0], cl[0]), v[r + P]);
#pragma unroll
          for (int t = 1; t <= P; ++t)
            ff2_fma(yy[r], f2(ch[t], ch[t]), f2(cl[t], cl[t]), ff2_add(v[r + P - t], v[r + P + t]));
        }
      }
      {  // A on PA (skew)
        FF2 v[RS + 2 * P];
#pragma unroll
        for (int t = 0; t < RS + 2 * P; ++t) v[t] = ld_ff2(&sMid[(2 * HR + rb + t) * TCP + cc]);
#pragma unroll
        for (int r = 0; r < RS; ++r)
#pragma unroll
          for (int t = 1; t <= P; ++t)
            ff2_fma(yy[r], f2(cs.c[1][0][P + t], cs.c[1][0][P + t]),
                    f2(cs.c[1][1][P + t], cs.c[1][1][P + t]), ff2_sub(v[r + P + t], v[r + P - t]));
      }
#pragma unroll
      for (int r = 0; r < RS; ++r) {
        const long long o1 = (long long)b * N + (long long)(r0 + rb + r) * m + j;
        ff2_emit(yy[r], o1, o1 + (long long)m * m, MODE, w, y, rhs, epi, ec1, ec2, dotp, acc);
      }
    } else {  // boundary rows (band rows staged in shared memory)
#pragma unroll 1
      for (int r = 0; r < RS; ++r) {
        const int i = r0 + rb + r;
        if (i >= m) break;
        FF2 yy{f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll 1
        for (int band = 0; band < 3; ++band) {
          const int x = band == 0 ? 0 : band == 1 ? 2 : 1;
#pragma unroll 1
          for (int k = 0; k < W; ++k) {
            const float2 cX = sRow[(x * W + k) * TR + rb + r];
            ff2_fma(yy, f2(cX.x, cX.x), f2(cX.y, cX.y), ld_ff2(&sMid[(band * HR + rb + r + k) * TCP + cc]));
          }
        }
        const long long o1 = (long long)b * N + (long long)i * m + j;
        ff2_emit(yy, o1, o1 + (long long)m * m, MODE, w, y, rhs, epi, ec1, ec2, dotp, acc);
      }
    }
  }
  if (dotp) {
    const double sum = block_sum(acc);
    if (threadIdx.x == 0)
      dotp[(size_t)b * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

template <int P, int TRV>
static void set_ff2_attr() {
  cudaFuncSetAttribute(apply2d_ff2_kernel<P, 0, TRV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)FF2Tile<P, TRV>::smem);
  cudaFuncSetAttribute(apply2d_ff2_kernel<P, 1, TRV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)FF2Tile<P, TRV>::smem);
  cudaFuncSetAttribute(apply2d_ff2_kernel<P, 2, TRV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)FF2Tile<P, TRV>::smem);
}

// Central rows split into (hi, lo); false unless M and S are palindromes and A is skew with a
// zero centre (the folded interior form needs that exactly).
static bool stencil_ff2(const StencilHost& sh, StencilFF2& cs) {
  const int P = sh.P;
  if (!stencil_folds(sh)) return false;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) {
      const double v = k < 2 * P + 1 ? sh.c[x][k] : 0.0;
      const float h = (float)v;
      cs.c[x][0][k] = h;
      cs.c[x][1][k] = (float)(v - (double)h);
    }
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  return true;
}

// Tile rows of the double-FP32 2D apply: 0 = chosen by the grid size, else kNarrowRows or the wide
// tile (any other value).
static std::atomic<int> g_ff2_rows{0};  // set at every handle creation, from any thread
static constexpr int kNarrowRows = 8;
void set_ff2_rows(int rows) { g_ff2_rows = rows; }

template <int P, int TRV>
static void launch_ff2_PT(int m, const StencilFF2& cs, const float2* ffT, const double* w, double* y,
                          const double* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                          const int* active, cudaStream_t s, const Epi<double>& epi) {
  using G = FF2Tile<P, TRV>;
  dim3 grid((m + G::TC - 1) / G::TC, (m + G::TR - 1) / G::TR, B);
  // one instantiation per epilogue mode keeps each kernel's code within the instruction cache
  if (mode == 0)
    apply2d_ff2_kernel<P, 0, TRV><<<grid, 128, G::smem, s>>>(m, ffT, cs, w, y, rhs, mode, c.alpha,
                                                             c.beta, c.gsc, active, dotp, epi);
  else if (mode == 1)
    apply2d_ff2_kernel<P, 1, TRV><<<grid, 128, G::smem, s>>>(m, ffT, cs, w, y, rhs, mode, c.alpha,
                                                             c.beta, c.gsc, active, dotp, epi);
  else
    apply2d_ff2_kernel<P, 2, TRV><<<grid, 128, G::smem, s>>>(m, ffT, cs, w, y, rhs, mode, c.alpha,
                                                             c.beta, c.gsc, active, dotp, epi);
  count_launch();
  if (nblk) *nblk = grid.x * grid.y;
}

template <int P>
static bool launch_ff2_P(int m, const StencilHost& sh, const double* w, double* y,
                         const double* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                         const int* active, cudaStream_t s, const Epi<double>& epi) {
  using G = FF2Tile<P>;
  using GN = FF2Tile<P, kNarrowRows>;
  StencilFF2 cs;
  if (!stencil_ff2(sh, cs)) return false;
  // The wide tile while the grid fills at least two full waves of 3 CTAs per SM; below that a
  // wide tile's latency sets the launch time and the narrow tile (a third of the rows, its x_2
  // pass spread over the whole CTA) runs about three times as many shorter CTAs.
  const long long cols = (m + G::TC - 1) / G::TC;
  const long long wide = cols * ((m + G::TR - 1) / G::TR) * B;
  bool narrow = g_ff2_rows == 0 ? wide < 2LL * 3 * num_sms() : g_ff2_rows == kNarrowRows;
  const long long tiles = cols * (narrow ? (m + GN::TR - 1) / GN::TR : (m + G::TR - 1) / G::TR);
  if (dotp && tiles > kMaxPartials) {
    if (!narrow || cols * ((m + G::TR - 1) / G::TR) > kMaxPartials) return false;
    narrow = false;
  }
  if (narrow)
    launch_ff2_PT<P, kNarrowRows>(m, cs, sh.ffT, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
  else
    launch_ff2_PT<P, 0>(m, cs, sh.ffT, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
  return true;
}

bool try_apply2d_ff(int m, int P, const double* bands, const double* w, double* y,
                    const double* rhs, int mode, int B, Coef c, double* dotp, int* nblk,
                    const int* active, cudaStream_t s, const Epi<double>& epi, int kernel) {
  if (mode == 2 && !epi.dinv) return false;
  StencilHost sh;
  if (!find_level(bands, sh) || sh.P != P || !sh.ffT) return false;
  if (kernel == 2) {
    bool ok = false;
    switch (P) {
      case 1: ok = launch_ff2_P<1>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      case 2: ok = launch_ff2_P<2>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      case 3: ok = launch_ff2_P<3>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      case 4: ok = launch_ff2_P<4>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      case 5: ok = launch_ff2_P<5>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      case 6: ok = launch_ff2_P<6>(m, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi); break;
      default: break;
    }
    if (ok) return true;
  }
  if (dotp && (long long)((m + 63) / 64) * ((m + 15) / 16) > kMaxPartials) return false;
  switch (P) {
    case 1: return launch_ff_P<1>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    case 2: return launch_ff_P<2>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    case 3: return launch_ff_P<3>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    case 4: return launch_ff_P<4>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    case 5: return launch_ff_P<5>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    case 6: return launch_ff_P<6>(m, bands, sh, w, y, rhs, mode, B, c, dotp, nblk, active, s, epi);
    default: return false;
  }
}

void prepare_ff_kernels() {
  set_ff_attr<1, 16>(); set_ff_attr<2, 16>(); set_ff_attr<3, 16>();
  set_ff_attr<4, 16>(); set_ff_attr<5, 16>(); set_ff_attr<6, 16>();
  set_ff2_attr<1, 0>(); set_ff2_attr<2, 0>(); set_ff2_attr<3, 0>();
  set_ff2_attr<4, 0>(); set_ff2_attr<5, 0>(); set_ff2_attr<6, 0>();
  set_ff2_attr<1, kNarrowRows>(); set_ff2_attr<2, kNarrowRows>(); set_ff2_attr<3, kNarrowRows>();
  set_ff2_attr<4, kNarrowRows>(); set_ff2_attr<5, kNarrowRows>(); set_ff2_attr<6, kNarrowRows>();
}

}  // namespace cd
