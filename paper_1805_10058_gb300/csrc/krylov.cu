// Krylov vector kernels, per-solve scalar steps (one thread per solve, fixed-order sums of
// block partials, so every reduction is deterministic and independent of the batch mix),
// and the Kronecker fast-diagonalisation (FD) per-axis contractions.
#include <cuda_runtime.h>

#include <algorithm>

#include "krylov.h"

namespace cd {

__device__ __forceinline__ double warp_sum2(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum2(double v) {
  __shared__ double red[32];
  v = warp_sum2(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    s = warp_sum2(s);
  }
  return s;
}

__device__ __forceinline__ double psum(const double* part, int nblk, int b) {
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[(size_t)b * nblk + i];
  return s;
}

// ------------------------------------------------------------------ vector kernels
template <typename T>
__global__ void __launch_bounds__(256) copy_kernel(long long N, const T* __restrict__ src,
                                                   T* __restrict__ dst,
                                                   const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = src[base + i];
}

template <typename T>
__global__ void __launch_bounds__(256) zero_kernel(long long N, T* __restrict__ dst,
                                                   const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = T(0);
}

// x += a p; r -= a q; partial sums of r.r (and of r.zold when zold != nullptr)
template <typename T>
__global__ void __launch_bounds__(256) cg_update_kernel(long long N, T* __restrict__ x,
                                                        T* __restrict__ r, const T* __restrict__ p,
                                                        const T* __restrict__ q,
                                                        const T* __restrict__ zold,
                                                        const double* __restrict__ alpha,
                                                        const int* __restrict__ active,
                                                        double* __restrict__ part_rr,
                                                        double* __restrict__ part_rz) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long chunk = (N + gridDim.x - 1) / gridDim.x;
  const long long lo = (long long)blockIdx.x * chunk, hi = min(N, lo + chunk);
  const long long base = (long long)b * N;
  const T a = T(alpha[b]);
  double rr = 0.0, rz = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const long long k = base + i;
    x[k] += a * p[k];
    const T rn = r[k] - a * q[k];
    r[k] = rn;
    rr += (double)rn * (double)rn;
    if (zold) rz += (double)rn * (double)zold[k];
  }
  const double s = block_sum2(rr);
  if (threadIdx.x == 0) part_rr[(size_t)b * gridDim.x + blockIdx.x] = s;
  if (zold) {
    const double t = block_sum2(rz);
    if (threadIdx.x == 0) part_rz[(size_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256) xpay_kernel(long long N, const T* __restrict__ z,
                                                   T* __restrict__ p,
                                                   const double* __restrict__ beta,
                                                   const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long base = (long long)b * N;
  const T be = T(beta[b]);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    p[base + i] = z[base + i] + be * p[base + i];
}

// r32 = float(r64 / ||r64||) (IR: the inner solve sees a unit-norm right-hand side)
__global__ void __launch_bounds__(256) ir_cast_kernel(long long N, const double* __restrict__ r64,
                                                      float* __restrict__ r32,
                                                      const double* __restrict__ rnorm,
                                                      const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long base = (long long)b * N;
  const double s = 1.0 / rnorm[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    r32[base + i] = (float)(r64[base + i] * s);
}

// x64 += ||r64|| * double(e32)
__global__ void __launch_bounds__(256) ir_update_kernel(long long N, double* __restrict__ x64,
                                                        const float* __restrict__ e32,
                                                        const double* __restrict__ rnorm,
                                                        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long base = (long long)b * N;
  const double s = rnorm[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    x64[base + i] += s * (double)e32[base + i];
}

// ------------------------------------------------------------------ scalar steps
// State layout (device doubles / ints, each of length B): see PcgState.
__global__ void cg_init_kernel(int B, PcgState st, const double* part_rr, int nrr,
                               const double* part_rz, int nrz, const int* outer_active,
                               int keep_others) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const bool on = outer_active ? outer_active[b] != 0 : true;
  if (!on && keep_others) return;  // a solve of a session that is mid-way through its own PCG
  const double rr = psum(part_rr, nrr, b), rz = psum(part_rz, nrz, b);
  st.rr0[b] = rr;
  st.rr[b] = rr;
  st.rz[b] = rz;
  st.iters[b] = 0;
  if (!on) {
    st.active[b] = 0;
    return;
  }
  if (!(rr < 1e300) || !(rz == rz)) {  // NaN / Inf right-hand side
    st.status[b] = CD_BREAKDOWN;
    st.active[b] = 0;
  } else if (rr == 0.0) {
    st.status[b] = CD_OK;
    st.active[b] = 0;
  } else {
    st.status[b] = CD_NOT_CONVERGED;
    st.active[b] = 1;
  }
}

__global__ void cg_alpha_kernel(int B, PcgState st, const double* part_pq, int npq) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !st.active[b]) return;
  const double pq = psum(part_pq, npq, b);
  if (!(pq > 0.0) || !(pq < 1e300)) {
    st.status[b] = CD_BREAKDOWN;
    st.active[b] = 0;
    st.alpha[b] = 0.0;
    return;
  }
  st.alpha[b] = st.rz[b] / pq;
}

__global__ void cg_check_kernel(int B, PcgState st, const double* part_rr, int nrr,
                                const double* part_rzold, int nrz, const double* tol2v, int maxit) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !st.active[b]) return;
  const double rr = psum(part_rr, nrr, b);
  st.rr[b] = rr;
  if (part_rzold) st.rzold[b] = psum(part_rzold, nrz, b);
  const int it = st.iters[b] + 1;
  st.iters[b] = it;
  if (!(rr == rr)) {
    st.status[b] = CD_BREAKDOWN;
    st.active[b] = 0;
  } else if (rr <= tol2v[b] * st.rr0[b]) {
    st.status[b] = CD_OK;
    st.active[b] = 0;
  } else if (it >= maxit) {
    st.status[b] = CD_NOT_CONVERGED;
    st.active[b] = 0;
  }
}

__global__ void cg_beta_kernel(int B, PcgState st, const double* part_rz, int nrz, int flexible) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !st.active[b]) return;
  const double rzn = psum(part_rz, nrz, b);
  if (!(rzn > 0.0) || !(rzn < 1e300)) {
    st.status[b] = CD_BREAKDOWN;
    st.active[b] = 0;
    return;
  }
  const double num = flexible ? rzn - st.rzold[b] : rzn;
  st.beta[b] = num / st.rz[b];
  st.rz[b] = rzn;
}

__global__ void count_active_kernel(int B, const int* __restrict__ active, int* __restrict__ out) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int c = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) c += active[b] ? 1 : 0;
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) *out = s;
}

// Outer step of the refinement loop: rnorm = ||b - A x||; decide convergence against
// ||b|| (or give up after max_outer steps / maxit Krylov iterations in total); move an
// FP32-inner solve whose last step reduced the residual less than tenfold to the FP64
// group; set the per-solve inner tolerance (squared).
__global__ void ir_check_kernel(int B, const double* part_rr, int nrr, const double* bnorm2,
                                double* rnorm, double* rrprev, int* active, int* status,
                                double* relres, int* outer_it, int* grp, double* tol2v,
                                double tol2, double inner2, int max_outer,
                                const int* inner_total, int maxit, double floor2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  const double rr = psum(part_rr, nrr, b);
  rnorm[b] = sqrt(rr);
  relres[b] = bnorm2[b] > 0 ? sqrt(rr / bnorm2[b]) : 0.0;
  if (!(rr == rr) || !(rr < 1e300)) {
    status[b] = CD_BREAKDOWN;
    active[b] = 0;
    return;
  }
  if (rr <= tol2 * bnorm2[b]) {
    status[b] = CD_OK;
    active[b] = 0;
    return;
  }
  if (outer_it[b] >= max_outer || inner_total[b] >= maxit) {
    status[b] = CD_NOT_CONVERGED;
    active[b] = 0;
    return;
  }
  if (outer_it[b] > 0 && grp[b] == 2 && rr > 0.25 * rrprev[b]) {
    // an FP64 refinement step gained less than 2x: the FP64 attainable accuracy
    // (about eps ||A|| ||x|| / ||b||) is reached
    status[b] = CD_NOT_CONVERGED;
    active[b] = 0;
    return;
  }
  if (outer_it[b] > 0 && grp[b] == 0 && rr > 1e-2 * rrprev[b]) grp[b] = 2;
  rrprev[b] = rr;
  outer_it[b] += 1;
  if (grp[b] == 0) {
    tol2v[b] = inner2;
  } else {
    // aim at the final tolerance: rtol ||b|| relative to the current residual
    double t = tol2 * bnorm2[b] / rr;
    tol2v[b] = fmin(fmax(t, floor2), 0.25);
  }
}

// masks of the three inner groups and their counts: out[g] = #{b : active && grp == g}
__global__ void group_masks_kernel(int B, const int* active, const int* grp, int* m0, int* m1,
                                   int* m2, int* out) {
  __shared__ int c[4];
  if (threadIdx.x < 4) c[threadIdx.x] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int a = active[b];
    const int g = grp[b];
    m0[b] = a && g == 0;
    m1[b] = a && g == 1;
    m2[b] = a && g == 2;
    if (a) atomicAdd(&c[g], 1);
    if (a) atomicAdd(&c[3], 1);
  }
  __syncthreads();
  if (threadIdx.x < 4) out[threadIdx.x] = c[threadIdx.x];
}

// dst = src / rnorm (FP64 inner right-hand side of unit norm)
__global__ void __launch_bounds__(256) scale_div_kernel(long long N, const double* __restrict__ src,
                                                        double* __restrict__ dst,
                                                        const double* __restrict__ rnorm,
                                                        const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long base = (long long)b * N;
  const double s = 1.0 / rnorm[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = src[base + i] * s;
}

// x64 += rnorm * e64
__global__ void __launch_bounds__(256) ir_update64_kernel(long long N, double* __restrict__ x64,
                                                          const double* __restrict__ e,
                                                          const double* __restrict__ rnorm,
                                                          const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const long long base = (long long)b * N;
  const double s = rnorm[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    x64[base + i] += s * e[base + i];
}

template <typename S, typename D>
__global__ void __launch_bounds__(256) convert_kernel(long long N, const S* __restrict__ src,
                                                      D* __restrict__ dst,
                                                      const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = (D)src[base + i];
}

// ------------------------------------------------------------------ FD contraction
// Batched strided GEMM C[z](r, c) = sum_k A[z](r, k) B[z](k, c) with a fused eigenvalue
// scaling epilogue.  SIMT, BMxBN tile, TMxTN per thread, BK-deep shared-memory stages.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_strided_kernel(int Mr, int Nc, int K, const T* __restrict__ A, long long ars, long long acs,
                        long long abs_, const T* __restrict__ Bm, long long brs, long long bcs,
                        long long bbs, T* __restrict__ C, long long crs, long long ccs,
                        long long cbs, FdScale<T> sc, const int* __restrict__ active,
                        long long batch_per_solve) {
  const int z = blockIdx.z;
  if (active && batch_per_solve > 0 && !active[z / batch_per_solve]) return;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int nth = (BM / TM) * (BN / TN);
  const int tid = threadIdx.x;
  const int tr = tid / (BN / TN), tc = tid % (BN / TN);
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const T* Az = A + (long long)z * abs_;
  const T* Bz = Bm + (long long)z * bbs;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    if (acs == 1) {  // A contiguous along k
      for (int e = tid; e < BM * BK; e += nth) {
        const int rr = e / BK, kk = e % BK;
        const int gr = r0 + rr, gk = k0 + kk;
        As[kk][rr] = (gr < Mr && gk < K) ? Az[gr * ars + gk] : T(0);
      }
    } else {  // A contiguous along r
      for (int e = tid; e < BM * BK; e += nth) {
        const int rr = e % BM, kk = e / BM;
        const int gr = r0 + rr, gk = k0 + kk;
        As[kk][rr] = (gr < Mr && gk < K) ? Az[gr * ars + gk * acs] : T(0);
      }
    }
    for (int e = tid; e < BN * BK; e += nth) {  // B contiguous along c
      const int cc = e % BN, kk = e / BN;
      const int gc = c0 + cc, gk = k0 + kk;
      Bs[kk][cc] = (gc < Nc && gk < K) ? Bz[gk * brs + gc * bcs] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[kk][tr * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tc * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  T* Cz = C + (long long)z * cbs;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gr = r0 + tr * TM + i;
    if (gr >= Mr) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = c0 + tc * TN + j;
      if (gc >= Nc) continue;
      T v = acc[i][j];
      T* dst = Cz + gr * crs + gc * ccs;
      if (sc.mode) {
        // decode the multi-index of dst inside the [B][d][m]^d tensor
        long long off = dst - sc.base;
        const long long per = sc.per;
        const long long bc = off / per;
        long long rem = off - bc * per;
        const int bsol = (int)(bc / sc.d), comp = (int)(bc % sc.d);
        double den = sc.mode == 1 ? 0.0 : 1.0;
        for (int l = sc.d - 1; l >= 0; --l) {
          const int kl = (int)(rem % sc.m);
          rem /= sc.m;
          const double lam = (double)sc.lam[kl];
          if (sc.mode == 1)
            den += (l == comp ? sc.beta[bsol] : sc.alpha[bsol]) * lam;
          else
            den *= lam;
        }
        v = T((double)v / den);
      }
      *dst = v;
    }
  }
}

template <typename T>
static int fd_contract(int m, long long I, long long O, int B, const T* G, const T* in, T* out,
                       FdScale<T> sc, const int* active, cudaStream_t s);

// out = contraction of `in` along `axis` with the m x m matrix G: out_k = sum_j G[j][k] in_j.
template <typename T>
int launch_fd_axis(int d, int m, int axis, int B, const T* G, const T* in, T* out,
                   FdScale<T> sc, const int* active, cudaStream_t s) {
  long long I = 1;
  for (int l = axis + 1; l < d; ++l) I *= m;
  long long O = (long long)B * d;
  for (int l = 0; l < axis; ++l) O *= m;
  return fd_contract<T>(m, I, O, B, G, in, out, sc, active, s);
}

// The same along `axis` of an anisotropic tensor [B][d][ma[0]]..[ma[d-1]] (G: ma[axis]^2).
template <typename T>
int launch_fd_axis_aniso(int d, const int* ma, int axis, int B, const T* G, const T* in, T* out,
                         const int* active, cudaStream_t s) {
  long long I = 1;
  for (int l = axis + 1; l < d; ++l) I *= ma[l];
  long long O = (long long)B * d;
  for (int l = 0; l < axis; ++l) O *= ma[l];
  return fd_contract<T>(ma[axis], I, O, B, G, in, out, FdScale<T>{}, active, s);
}
template int launch_fd_axis_aniso<double>(int, const int*, int, int, const double*, const double*,
                                          double*, const int*, cudaStream_t);
template int launch_fd_axis_aniso<float>(int, const int*, int, int, const float*, const float*,
                                         float*, const int*, cudaStream_t);

// outer batch O (B solves), contraction length m, inner extent I
template <typename T>
static int fd_contract(int m, long long I, long long O, int B, const T* G, const T* in, T* out,
                       FdScale<T> sc, const int* active, cudaStream_t s) {
  long long per_solve_outer = O / B;
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
  if (I == 1) {
    // C[r][k] = sum_j in[r][j] G[j][k], rows r = all outer indices (batched over z by 65535 rows)
    const long long R = O;
    const long long rows_per_z = 65535LL * BM;
    const long long nz = (R + rows_per_z - 1) / rows_per_z;
    for (long long z0 = 0; z0 < nz; ++z0) {
      const long long rlo = z0 * rows_per_z;
      const int Rz = (int)std::min(rows_per_z, R - rlo);
      dim3 grid((m + BN - 1) / BN, (Rz + BM - 1) / BM, 1);
      gemm_strided_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(
          Rz, m, m, in + rlo * m, m, 1, 0, G, m, 1, 0, out + rlo * m, m, 1, 0, sc, nullptr, 0);
      count_launch();
    }
  } else {
    // for each outer o: C_o[k][i] = sum_j G[j][k] in_o[j][i]
    const long long zmax = 65535;
    for (long long o0 = 0; o0 < O; o0 += zmax) {
      const int nz = (int)std::min(zmax, O - o0);
      dim3 grid((unsigned)((I + BN - 1) / BN), (m + BM - 1) / BM, nz);
      const bool mask = active != nullptr && (o0 % per_solve_outer) == 0;
      gemm_strided_kernel<T, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(
          m, (int)I, m, G, 1, m, 0, in + o0 * m * I, I, 1, (long long)m * I, out + o0 * m * I, I,
          1, (long long)m * I, sc, mask ? active + o0 / per_solve_outer : nullptr,
          mask ? per_solve_outer : 0);
      count_launch();
    }
  }
  return 0;
}
template int launch_fd_axis<double>(int, int, int, int, const double*, const double*, double*,
                                    FdScale<double>, const int*, cudaStream_t);
template int launch_fd_axis<float>(int, int, int, int, const float*, const float*, float*,
                                   FdScale<float>, const int*, cudaStream_t);

// ------------------------------------------------------------------ launch wrappers
static inline dim3 vgrid(long long N, int B) {
  long long nb = (N + 255) / 256;
  nb = std::min<long long>(nb, 2048);
  return dim3((unsigned)std::max<long long>(nb, 1), B);
}

template <typename T>
void vcopy(long long N, int B, const T* src, T* dst, const int* active, cudaStream_t s) {
  copy_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, src, dst, active);
  count_launch();
}
template <typename T>
void vzero(long long N, int B, T* dst, const int* active, cudaStream_t s) {
  zero_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, dst, active);
  count_launch();
}
template <typename T>
void cg_update(long long N, int B, int nblk, T* x, T* r, const T* p, const T* q, const T* zold,
               const double* alpha, const int* active, double* part_rr, double* part_rz,
               cudaStream_t s) {
  cg_update_kernel<T><<<dim3(nblk, B), 256, 0, s>>>(N, x, r, p, q, zold, alpha, active, part_rr,
                                                    part_rz);
  count_launch();
}
template <typename T>
void xpay(long long N, int B, const T* z, T* p, const double* beta, const int* active,
          cudaStream_t s) {
  xpay_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, z, p, beta, active);
  count_launch();
}
void ir_cast(long long N, int B, const double* r64, float* r32, const double* rnorm,
             const int* active, cudaStream_t s) {
  ir_cast_kernel<<<vgrid(N, B), 256, 0, s>>>(N, r64, r32, rnorm, active);
  count_launch();
}
void ir_update(long long N, int B, double* x64, const float* e32, const double* rnorm,
               const int* active, cudaStream_t s) {
  ir_update_kernel<<<vgrid(N, B), 256, 0, s>>>(N, x64, e32, rnorm, active);
  count_launch();
}
static inline int sgrid(int B) { return (B + 127) / 128; }
void cg_init(int B, PcgState st, const double* prr, int nrr, const double* prz, int nrz,
             const int* outer_active, cudaStream_t s, int keep_others) {
  cg_init_kernel<<<sgrid(B), 128, 0, s>>>(B, st, prr, nrr, prz, nrz, outer_active, keep_others);
  count_launch();
}
void cg_alpha(int B, PcgState st, const double* ppq, int npq, cudaStream_t s) {
  cg_alpha_kernel<<<sgrid(B), 128, 0, s>>>(B, st, ppq, npq);
  count_launch();
}
void cg_check(int B, PcgState st, const double* prr, int nrr, const double* prz, int nrz,
              const double* tol2v, int maxit, cudaStream_t s) {
  cg_check_kernel<<<sgrid(B), 128, 0, s>>>(B, st, prr, nrr, prz, nrz, tol2v, maxit);
  count_launch();
}
void cg_beta(int B, PcgState st, const double* prz, int nrz, int flexible, cudaStream_t s) {
  cg_beta_kernel<<<sgrid(B), 128, 0, s>>>(B, st, prz, nrz, flexible);
  count_launch();
}
void count_active(int B, const int* active, int* out, cudaStream_t s) {
  count_active_kernel<<<1, 256, 0, s>>>(B, active, out);
  count_launch();
}
void ir_check(int B, const double* prr, int nrr, const double* bnorm2, double* rnorm,
              double* rrprev, int* active, int* status, double* relres, int* outer_it, int* grp,
              double* tol2v, double tol2, double inner2, int max_outer, const int* inner_total,
              int maxit, double floor2, cudaStream_t s) {
  ir_check_kernel<<<sgrid(B), 128, 0, s>>>(B, prr, nrr, bnorm2, rnorm, rrprev, active, status,
                                           relres, outer_it, grp, tol2v, tol2, inner2, max_outer,
                                           inner_total, maxit, floor2);
  count_launch();
}
void group_masks(int B, const int* active, const int* grp, int* m0, int* m1, int* m2, int* out,
                 cudaStream_t s) {
  group_masks_kernel<<<1, 256, 0, s>>>(B, active, grp, m0, m1, m2, out);
  count_launch();
}
void scale_div(long long N, int B, const double* src, double* dst, const double* rnorm,
               const int* active, cudaStream_t s) {
  scale_div_kernel<<<vgrid(N, B), 256, 0, s>>>(N, src, dst, rnorm, active);
  count_launch();
}
void ir_update64(long long N, int B, double* x64, const double* e, const double* rnorm,
                 const int* active, cudaStream_t s) {
  ir_update64_kernel<<<vgrid(N, B), 256, 0, s>>>(N, x64, e, rnorm, active);
  count_launch();
}
void to_f32(long long N, int B, const double* src, float* dst, const int* active, cudaStream_t s) {
  convert_kernel<double, float><<<vgrid(N, B), 256, 0, s>>>(N, src, dst, active);
  count_launch();
}
void to_f64(long long N, int B, const float* src, double* dst, const int* active, cudaStream_t s) {
  convert_kernel<float, double><<<vgrid(N, B), 256, 0, s>>>(N, src, dst, active);
  count_launch();
}

// ------------------------------------------------------------------ banded T solves
// One thread per pencil (a line of m values along the axis, at stride I): forward substitution
// with L, then backward substitution with L^T, each keeping the last q values in registers.
// Pencil (o, c): first value at o * m * I + c; consecutive threads take consecutive c, so the
// accesses of a warp are contiguous for every axis but the last.
template <typename T, int Q>
__global__ void __launch_bounds__(256) tband_kernel(int m, long long I, long long npencil,
                                                    long long opb, const T* __restrict__ Lb,
                                                    const T* __restrict__ dinv, const T* in,
                                                    T* out, const int* __restrict__ active) {
  const long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pid >= npencil) return;
  const long long o = pid / I, c = pid - o * I;
  if (active && !active[o / opb]) return;
  const T* x = in + o * m * I + c;
  T* y = out + o * m * I + c;
  T win[Q + 1];  // forward: win[t] = y_{i - Q + t}; backward: win[u] = x_{i + 1 + u}
#pragma unroll
  for (int t = 0; t <= Q; ++t) win[t] = T(0);
  for (int i = 0; i < m; ++i) {
    T v = x[(long long)i * I];
#pragma unroll
    for (int t = 0; t < Q; ++t) v -= Lb[(size_t)i * Q + t] * win[t];
    v *= dinv[i];
    y[(long long)i * I] = v;
#pragma unroll
    for (int t = 0; t + 1 < Q; ++t) win[t] = win[t + 1];
    if (Q > 0) win[Q - 1] = v;
  }
#pragma unroll
  for (int t = 0; t <= Q; ++t) win[t] = T(0);
  for (int i = m - 1; i >= 0; --i) {
    T v = y[(long long)i * I];
    // (L^T x)_i = sum_{u=0..Q} L(i + u, i) x_{i+u}, L(i + u, i) = Lb[(i + u) * Q + Q - u]
#pragma unroll
    for (int u = 1; u <= Q; ++u) v -= Lb[(size_t)(i + u) * Q + (Q - u)] * win[u - 1];
    v *= dinv[i];
    y[(long long)i * I] = v;
#pragma unroll
    for (int u = Q - 1; u > 0; --u) win[u] = win[u - 1];
    if (Q > 0) win[0] = v;
  }
}

template <typename T>
int launch_tband(int d, int m, int q, int B, const T* Lb, const T* dinv, const T* in, T* out,
                 const int* active, cudaStream_t s) {
  if (q < 0 || q > 5) return 1;
  for (int a = 0; a < d; ++a) {
    long long I = 1, opb = d;
    for (int l = a + 1; l < d; ++l) I *= m;
    for (int l = 0; l < a; ++l) opb *= m;
    const long long np = (long long)B * opb * I;
    const unsigned grid = (unsigned)((np + 255) / 256);
    const T* src = a == 0 ? in : out;
    switch (q) {
      case 0: tband_kernel<T, 0><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
      case 1: tband_kernel<T, 1><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
      case 2: tband_kernel<T, 2><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
      case 3: tband_kernel<T, 3><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
      case 4: tband_kernel<T, 4><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
      default: tband_kernel<T, 5><<<grid, 256, 0, s>>>(m, I, np, opb, Lb, dinv, src, out, active); break;
    }
    count_launch();
  }
  return 0;
}
template int launch_tband<double>(int, int, int, int, const double*, const double*, const double*,
                                  double*, const int*, cudaStream_t);
template int launch_tband<float>(int, int, int, int, const float*, const float*, const float*,
                                 float*, const int*, cudaStream_t);

template void vcopy<double>(long long, int, const double*, double*, const int*, cudaStream_t);
template void vcopy<float>(long long, int, const float*, float*, const int*, cudaStream_t);
template void vzero<double>(long long, int, double*, const int*, cudaStream_t);
template void vzero<float>(long long, int, float*, const int*, cudaStream_t);
template void cg_update<double>(long long, int, int, double*, double*, const double*,
                                const double*, const double*, const double*, const int*, double*,
                                double*, cudaStream_t);
template void cg_update<float>(long long, int, int, float*, float*, const float*, const float*,
                               const float*, const double*, const int*, double*, double*,
                               cudaStream_t);
template void xpay<double>(long long, int, const double*, double*, const double*, const int*,
                           cudaStream_t);
template void xpay<float>(long long, int, const float*, float*, const double*, const int*,
                          cudaStream_t);

}  // namespace cd
