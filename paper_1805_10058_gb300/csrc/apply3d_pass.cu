// The 3D operator apply as three tuned banded passes (sum factorisation of the Kronecker form
// of the 3D block matrix, Section 4.2, eq:matr_Amu3D), in FP32, FP64 or double-FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "apply_shared.h"
#include "ffmath.h"

namespace cd {

// ------------------------------------------------------------------ 3D apply: three tuned passes
// The three banded passes of the 3D operator (x_3: nine arrays T_{X,c} = X_3 w_c; x_2: nine
// arrays P grouped by the x_1 operator they feed; x_1: y_c = M_1 P_cM + S_1 P_cS + A_1 P_cA),
// each a kernel with the minimal 33 (2p+1) multiply-adds per grid point: along x_2 and x_1 a
// thread produces R consecutive rows from one register window of R + 2P inputs per array
// (coalesced across the warp along x_3), along x_3 one point from a window read through L1.
// Interior rows take the central stencil from the kernel parameters, boundary rows their band
// row.  Three arithmetic policies: FP32, FP64, and double-FP32 (FP64 input and output, the
// intermediates stored as (hi, lo) FP32 pairs, every multiply-add a double-FP32 one on the FP32
// pipe).
struct P3F32 {
  using In = float;
  using Mid = float;
  using V = float;
  using C = float;
  static __device__ __forceinline__ V zero() { return 0.f; }
  static __device__ __forceinline__ V in(const In* p) { return *p; }
  static __device__ __forceinline__ V mid(const Mid* p) { return *p; }
  static __device__ __forceinline__ void put_mid(Mid* p, V v) { *p = v; }
  static __device__ __forceinline__ In out(V v) { return v; }
  static __device__ __forceinline__ void fma(V& acc, C c, V x) { acc = fmaf(c, x, acc); }
  static __device__ __forceinline__ V mul(C c, V x) { return c * x; }
  static __device__ __forceinline__ C band(const float* bands, size_t i) { return bands[i]; }
  static __host__ __device__ __forceinline__ C cst(double v) { return (float)v; }
};
struct P3F64 {
  using In = double;
  using Mid = double;
  using V = double;
  using C = double;
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V in(const In* p) { return *p; }
  static __device__ __forceinline__ V mid(const Mid* p) { return *p; }
  static __device__ __forceinline__ void put_mid(Mid* p, V v) { *p = v; }
  static __device__ __forceinline__ In out(V v) { return v; }
  static __device__ __forceinline__ void fma(V& acc, C c, V x) { acc = ::fma(c, x, acc); }
  static __device__ __forceinline__ V mul(C c, V x) { return c * x; }
  static __device__ __forceinline__ C band(const double* bands, size_t i) { return bands[i]; }
  static __host__ __device__ __forceinline__ C cst(double v) { return v; }
};
struct P3FF {
  using In = double;
  using Mid = float2;
  using V = float2;  // (hi, lo)
  using C = float2;
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ V in(const In* p) { return ff_split_bits(*p); }
  static __device__ __forceinline__ V mid(const Mid* p) { return *p; }
  static __device__ __forceinline__ void put_mid(Mid* p, V v) { *p = ff_norm(v); }
  static __device__ __forceinline__ In out(V v) {
    const float2 n = ff_norm(v);
    return __dadd_rn(f2d_bits(n.x), f2d_bits(n.y));
  }
  static __device__ __forceinline__ void fma(V& acc, C c, V x) { ff_fma(acc, c, x); }
  static __device__ __forceinline__ V mul(C c, V x) { return ff_mul(c, x); }
  static __device__ __forceinline__ C band(const double* bands, size_t i) {
    return ff_split_bits(bands[i]);
  }
  static __host__ __device__ __forceinline__ C cst(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
};
__device__ __forceinline__ float add3(float a, float b) { return a + b; }
__device__ __forceinline__ double add3(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add3(float2 a, float2 b) {  // double-FP32 a + b
  const float sm = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(sm, a.x);
  const float er = __fadd_rn(__fsub_rn(a.x, __fsub_rn(sm, bb)), __fsub_rn(b.x, bb));
  return make_float2(sm, __fadd_rn(__fadd_rn(a.y, b.y), er));
}

template <typename Pol>
struct Stencil3 {
  typename Pol::C c[3][13];  // M, A, S central rows
  int lo, hi;
};
template <typename Pol>
struct Pass3Args {
  const typename Pol::In* w;   // [B][3][m^3] (pass 0)
  const float2* wsplit;        // double-FP32 policy: w split into (hi, lo) pairs, same layout
  typename Pol::Mid* t;        // 9 arrays [9][B][m^3] (pass 0 out, pass 1 in)
  typename Pol::Mid* q;        // 9 arrays (pass 1 out, pass 2 in)
  typename Pol::In* y;         // [B][3][m^3] (pass 2)
};

// band X applied along an axis to a window of R + 2P values:
// out[r] = (scaled ? scale : 1) * sum_k X(i0 + r, i0 + r - P + k) win[r + k]
template <typename Pol, int P, int R>
__device__ __forceinline__ void band_apply(const Stencil3<Pol>& cs, const typename Pol::In* bands,
                                           int m, int X, int i0, const typename Pol::V* win,
                                           typename Pol::C scale, bool scaled, typename Pol::V* out) {
  constexpr int W = 2 * P + 1;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    typename Pol::V acc = Pol::zero();
    if (i >= cs.lo && i < cs.hi) {
#pragma unroll
      for (int k = 0; k < W; ++k) Pol::fma(acc, cs.c[X][k], win[r + k]);
    } else if (i < m) {
#pragma unroll
      for (int k = 0; k < W; ++k) Pol::fma(acc, Pol::band(bands, ((size_t)X * m + i) * W + k), win[r + k]);
    }
    out[r] = scaled ? Pol::mul(scale, acc) : acc;
  }
}

// The same with the band index X known only at run time, the central rows read from shared
// memory (sc: [3][13]); the double-FP32 passes loop over their terms with it so that one copy of
// the term's code stays in the instruction cache.
template <typename Pol, int P, int R>
__device__ __forceinline__ void band_apply_rt(const typename Pol::C* sc, int lo, int hi,
                                              const typename Pol::In* bands, int m, int X, int i0,
                                              const typename Pol::V* win, typename Pol::V* out) {
  constexpr int W = 2 * P + 1;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    typename Pol::V acc = Pol::zero();
    if (i >= lo && i < hi) {
#pragma unroll
      for (int k = 0; k < W; ++k) Pol::fma(acc, sc[X * 13 + k], win[r + k]);
    } else if (i < m) {
#pragma unroll
      for (int k = 0; k < W; ++k) Pol::fma(acc, Pol::band(bands, ((size_t)X * m + i) * W + k), win[r + k]);
    }
    out[r] = acc;
  }
}

// Terms of the x_2 pass: (source T array X * 3 + comp, band X2 along x_2, scalar 0 alpha /
// 1 beta / 2 gamma, first term of its output, output written after the term or -1); the output
// order and the grouping are those of the unrolled pass below.
__constant__ signed char k_pass1_terms[15][6] = {
    {2, 0, 0, 0, 1, -1}, {0, 0, 2, 0, 0, 0},                        // P1M
    {0, 0, 0, 1, 1, 1},                                             // P1S
    {0, 1, 1, 2, 1, -1}, {1, 2, 0, 2, 0, 2},                        // P1A
    {2, 1, 0, 0, 1, -1}, {0, 1, 2, 1, 0, -1}, {1, 2, 1, 2, 0, 3},   // P2M
    {0, 1, 0, 0, 1, 4},                                             // P2S
    {0, 0, 1, 2, 1, 5},                                             // P2A
    {0, 2, 2, 0, 1, -1}, {2, 2, 0, 1, 0, -1}, {1, 1, 1, 2, 0, 6},   // P3M
    {0, 2, 0, 0, 1, 7},                                             // P3S
    {1, 0, 0, 2, 1, 8}};                                            // P3A

template <typename Pol, int P, int PASS, int R>
__global__ void __launch_bounds__(128) pass3d_kernel(int m, const typename Pol::In* __restrict__ bands,
                                                     Stencil3<Pol> cs, Pass3Args<Pol> a,
                                                     const double* __restrict__ alpha,
                                                     const double* __restrict__ beta,
                                                     const double* __restrict__ gsc,
                                                     const int* __restrict__ active) {
  using V = typename Pol::V;
  using C = typename Pol::C;
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ C s_par[3];
  if (threadIdx.x == 0) {
    s_par[0] = Pol::cst(alpha[b]);
    s_par[1] = Pol::cst(beta[b]);
    s_par[2] = Pol::cst((alpha[b] - beta[b]) * (gsc ? gsc[b] : 1.0));
  }
  constexpr bool kFF = std::is_same<V, float2>::value;
  __shared__ C s_c[kFF ? 3 * 13 : 1];
  if constexpr (kFF) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int t = 0; t < 3 * 13; ++t) s_c[t] = cs.c[t / 13][t % 13];
    }
  }
  __syncthreads();
  const C al = s_par[0], be = s_par[1], ga = s_par[2];
  const int n3 = m * m * m, nblk = (m + R - 1) / R;
  const int stride = PASS == 0 ? 1 : PASS == 1 ? m : m * m;
  const int items = PASS == 0 ? n3 : nblk * m * m;
  const long long B = gridDim.y;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    // (i0, i1, i2) of the first row this thread produces; the pass axis is blocked by R
    int i0, i1, i2;
    if (PASS == 0) {
      i2 = it % m;
      i1 = (it / m) % m;
      i0 = it / (m * m);
    } else if (PASS == 1) {
      i2 = it % m;
      i1 = ((it / m) % nblk) * R;
      i0 = it / (m * nblk);
    } else {
      i2 = it % m;
      i1 = (it / m) % m;
      i0 = (it / (m * m)) * R;
    }
    const int ia = PASS == 0 ? i2 : PASS == 1 ? i1 : i0;  // position along the pass axis
    const int base = (i0 * m + i1) * m + i2;              // point of the first row
    auto window = [&](auto loader, V* win) {
#pragma unroll
      for (int k = 0; k < R + 2 * P; ++k) {
        const int j = ia - P + k;
        win[k] = (j >= 0 && j < m) ? loader(base + (k - P) * stride) : Pol::zero();
      }
    };
    if constexpr (PASS == 0 && kFF) {
      V win[R + 2 * P], o[R];
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        const float2* wc = a.wsplit + ((long long)b * 3 + c) * n3;
        window([&](int idx) { return wc[idx]; }, win);
#pragma unroll
        for (int X = 0; X < 3; ++X) {
          band_apply_rt<Pol, P, R>(s_c, cs.lo, cs.hi, bands, m, X, ia, win, o);
          Pol::put_mid(a.t + ((long long)(X * 3 + c) * B + b) * n3 + base, o[0]);
        }
      }
    } else if constexpr (PASS == 0) {
      V win[R + 2 * P], o[R];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (std::is_same<V, float2>::value) {  // split once by the split kernel
          const float2* wc = a.wsplit + ((long long)b * 3 + c) * n3;
          window([&](int idx) { return wc[idx]; }, win);
        } else {
          const typename Pol::In* wc = a.w + ((long long)b * 3 + c) * n3;
          window([&](int idx) { return Pol::in(wc + idx); }, win);
        }
#pragma unroll
        for (int X = 0; X < 3; ++X) {
          band_apply<Pol, P, R>(cs, bands, m, X, ia, win, al, false, o);
          Pol::put_mid(a.t + ((long long)(X * 3 + c) * B + b) * n3 + base, o[0]);
        }
      }
    } else if constexpr (PASS == 1 && kFF) {
      // one term per trip (its window loaded, its band applied, scaled and summed)
      V win[R + 2 * P], tmp[R], acc[R];
#pragma unroll 1
      for (int t = 0; t < 15; ++t) {
        const int X = k_pass1_terms[t][0], comp = k_pass1_terms[t][1], X2 = k_pass1_terms[t][2];
        const int sid = k_pass1_terms[t][3], first = k_pass1_terms[t][4], o = k_pass1_terms[t][5];
        const typename Pol::Mid* src = a.t + ((long long)(X * 3 + comp) * B + b) * n3;
        window([&](int idx) { return Pol::mid(src + idx); }, win);
        band_apply_rt<Pol, P, R>(s_c, cs.lo, cs.hi, bands, m, X2, ia, win, tmp);
        const C sc = sid == 0 ? al : sid == 1 ? be : ga;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const V v = Pol::mul(sc, tmp[r]);
          acc[r] = first ? v : add3(acc[r], v);
        }
        if (o >= 0) {
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (ia + r < m) Pol::put_mid(a.q + ((long long)o * B + b) * n3 + base + r * stride, acc[r]);
        }
      }
    } else if constexpr (PASS == 1) {
      // P_cX arrays (index c*3 + {0: feeds M1, 1: feeds S1, 2: feeds A1}) from the T arrays
      // (index X*3 + comp, X: 0 M, 1 A, 2 S):
      // P1M = alpha (M2 T_S1 + S2 T_M1); P1S = beta M2 T_M1; P1A = gamma (A2 T_M2 + M2 T_A3)
      // P2M = alpha M2 T_S2 + beta S2 T_M2 + gamma A2 T_A3; P2S = alpha M2 T_M2; P2A = gamma A2 T_M1
      // P3M = alpha S2 T_M3 + beta M2 T_S3 + gamma A2 T_A2; P3S = alpha M2 T_M3; P3A = gamma M2 T_A1
      V acc[9][R];
#pragma unroll
      for (int o = 0; o < 9; ++o)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[o][r] = Pol::zero();
      V win[R + 2 * P], tmp[R];
      auto from = [&](int X, int comp) {
        const typename Pol::Mid* src = a.t + ((long long)(X * 3 + comp) * B + b) * n3;
        window([&](int idx) { return Pol::mid(src + idx); }, win);
      };
      auto addto = [&](int o, int X2, C sc) {  // acc[o] += sc * X2_2 win
        band_apply<Pol, P, R>(cs, bands, m, X2, ia, win, sc, true, tmp);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[o][r] = add3(acc[o][r], tmp[r]);
      };
      from(2, 0); addto(0, 0, al);                                   // T_S1
      from(0, 0); addto(0, 2, al); addto(1, 0, be); addto(5, 1, ga); // T_M1
      from(0, 1); addto(2, 1, ga); addto(3, 2, be); addto(4, 0, al); // T_M2
      from(1, 2); addto(2, 0, ga); addto(3, 1, ga);                  // T_A3
      from(2, 1); addto(3, 0, al);                                   // T_S2
      from(0, 2); addto(6, 2, al); addto(7, 0, al);                  // T_M3
      from(2, 2); addto(6, 0, be);                                   // T_S3
      from(1, 1); addto(6, 1, ga);                                   // T_A2
      from(1, 0); addto(8, 0, ga);                                   // T_A1
#pragma unroll
      for (int o = 0; o < 9; ++o)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (ia + r < m) Pol::put_mid(a.q + ((long long)o * B + b) * n3 + base + r * stride, acc[o][r]);
    } else if constexpr (kFF) {
      V win[R + 2 * P], tmp[R], yc[R];
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {  // P_cM with M1, P_cS with S1, P_cA with A1
        const int c = t / 3, g = t - 3 * c;
        const typename Pol::Mid* src = a.q + ((long long)t * B + b) * n3;
        window([&](int idx) { return Pol::mid(src + idx); }, win);
        band_apply_rt<Pol, P, R>(s_c, cs.lo, cs.hi, bands, m, g == 0 ? 0 : g == 1 ? 2 : 1, ia, win,
                                 tmp);
#pragma unroll
        for (int r = 0; r < R; ++r) yc[r] = g == 0 ? tmp[r] : add3(yc[r], tmp[r]);
        if (g == 2) {
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (ia + r < m) a.y[((long long)b * 3 + c) * n3 + base + r * stride] = Pol::out(yc[r]);
        }
      }
    } else {
      V win[R + 2 * P], tmp[R];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        V yc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) yc[r] = Pol::zero();
#pragma unroll
        for (int g = 0; g < 3; ++g) {  // P_cM with M1, P_cS with S1, P_cA with A1
          const typename Pol::Mid* src = a.q + ((long long)(c * 3 + g) * B + b) * n3;
          window([&](int idx) { return Pol::mid(src + idx); }, win);
          band_apply<Pol, P, R>(cs, bands, m, g == 0 ? 0 : g == 1 ? 2 : 1, ia, win, al, false, tmp);
#pragma unroll
          for (int r = 0; r < R; ++r) yc[r] = add3(yc[r], tmp[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (ia + r < m) a.y[((long long)b * 3 + c) * n3 + base + r * stride] = Pol::out(yc[r]);
      }
    }
  }
}

// (hi, lo) FP32 pairs of an FP64 array, by integer operations
__global__ void __launch_bounds__(256) split_ff_kernel(long long n, const double* __restrict__ src,
                                                        float2* __restrict__ dst,
                                                        const int* __restrict__ active, long long per) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (active && !active[i / per]) continue;
    dst[i] = ff_split_bits(src[i]);
  }
}

template <typename Pol, int P>
static void launch_pass3d_P(int m, const typename Pol::In* bands, const StencilHost& sh,
                            const typename Pol::In* w, typename Pol::In* y, int B, Coef c,
                            const int* active, typename Pol::Mid* scratch, cudaStream_t s) {
  constexpr int R = 4;
  Stencil3<Pol> cs;
  for (int x = 0; x < 3; ++x)
    for (int k = 0; k < 13; ++k) cs.c[x][k] = Pol::cst(k < 2 * P + 1 ? sh.c[x][k] : 0.0);
  cs.lo = sh.lo;
  cs.hi = sh.hi;
  const long long n3 = (long long)m * m * m;
  // the q arrays' space holds the split input during the first pass (q is written by the second)
  Pass3Args<Pol> a{w, reinterpret_cast<const float2*>(scratch + 9 * n3 * B), scratch,
                   scratch + 9 * n3 * B, y};
  if constexpr (std::is_same<typename Pol::V, float2>::value) {
    split_ff_kernel<<<(unsigned)std::min<long long>((3 * n3 * B + 255) / 256, 16384), 256, 0, s>>>(
        3 * n3 * B, (const double*)w, reinterpret_cast<float2*>(scratch + 9 * n3 * B), active, 3 * n3);
    count_launch();
  }
  auto grid = [&](long long items) {
    return dim3((unsigned)std::min<long long>((items + 127) / 128, 16384), B);
  };
  const long long nblk = (m + R - 1) / R;
  pass3d_kernel<Pol, P, 0, 1><<<grid(n3), 128, 0, s>>>(m, bands, cs, a, c.alpha, c.beta, c.gsc, active);
  pass3d_kernel<Pol, P, 1, R><<<grid(nblk * m * m), 128, 0, s>>>(m, bands, cs, a, c.alpha, c.beta,
                                                                 c.gsc, active);
  pass3d_kernel<Pol, P, 2, R><<<grid(nblk * m * m), 128, 0, s>>>(m, bands, cs, a, c.alpha, c.beta,
                                                                 c.gsc, active);
  count_launch(3);
}

// y = A w (3D) by the three tuned passes; the FP64 policy P3FF computes in double-FP32.  False
// when the level is not registered or P is outside 1..6.
template <typename Pol>
static bool launch_pass3d(int m, int P, const typename Pol::In* bands, const typename Pol::In* w,
                          typename Pol::In* y, int B, Coef c, const int* active,
                          typename Pol::Mid* scratch, cudaStream_t s) {
  StencilHost sh;
  if (!find_level(bands, sh) || sh.P != P) return false;
  switch (P) {
    case 1: launch_pass3d_P<Pol, 1>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    case 2: launch_pass3d_P<Pol, 2>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    case 3: launch_pass3d_P<Pol, 3>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    case 4: launch_pass3d_P<Pol, 4>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    case 5: launch_pass3d_P<Pol, 5>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    case 6: launch_pass3d_P<Pol, 6>(m, bands, sh, w, y, B, c, active, scratch, s); return true;
    default: return false;
  }
}


bool launch_pass3d_f32(int m, int P, const float* bands, const float* w, float* y, int B, Coef c,
                       const int* active, float* scratch, cudaStream_t s) {
  return launch_pass3d<P3F32>(m, P, bands, w, y, B, c, active, scratch, s);
}
bool launch_pass3d_f64(int m, int P, const double* bands, const double* w, double* y, int B, Coef c,
                       const int* active, double* scratch, cudaStream_t s) {
  return launch_pass3d<P3F64>(m, P, bands, w, y, B, c, active, scratch, s);
}
bool launch_pass3d_ff(int m, int P, const double* bands, const double* w, double* y, int B, Coef c,
                      const int* active, float2* scratch, cudaStream_t s) {
  return launch_pass3d<P3FF>(m, P, bands, w, y, B, c, active, scratch, s);
}

}  // namespace cd
