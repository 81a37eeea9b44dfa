// Krylov post-smoothers of the finest multigrid level (Section 6.1, Section 6.2): `steps`
// iterations of right-preconditioned GMRES (P_MIM, MIM) or of PCG (P_WL) with the preconditioner
// T = I_d (x) T_m(m_{p-1}) (x) ... (eq:kron_precond), started from the current iterate, with
// per-solve scalars for a batch of B solves.  T^{-1} is applied by banded Cholesky solves along
// every axis (the banded factorisation route of Section 6.1).
//
// Reductions are per solve and in a fixed order (block partial sums, then a sequential sum over
// the blocks), so a solve gives the same bits alone and inside any batch.  GMRES orthogonalises by
// classical Gram-Schmidt applied twice (each pass: one multi-dot kernel, one update kernel).
#include <cuda_runtime.h>

#include <cmath>

#include "krylov.h"
#include "mg.h"

namespace cd {

namespace {

constexpr int kKsMaxDots = 8;

// part[(b * kKsMaxDots + i) * nblk + blk] = sum over the block of w * v_i, i < k (v_i = V + i*ldv)
template <typename T>
__global__ void __launch_bounds__(256) ks_mdot_kernel(long long N, int k, const T* __restrict__ w,
                                                      const T* __restrict__ V, long long ldv,
                                                      const int* __restrict__ active,
                                                      double* __restrict__ part, int nblk) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < N ? lo + chunk : N;
  double acc[kKsMaxDots];
  for (int i = 0; i < kKsMaxDots; ++i) acc[i] = 0.0;
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const double wv = (double)w[base + e];
    for (int i = 0; i < k; ++i) acc[i] += wv * (double)V[(long long)i * ldv + base + e];
  }
  __shared__ double red[kKsMaxDots][256];
  for (int i = 0; i < k; ++i) red[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int i = 0; i < k; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < k) part[((size_t)b * kKsMaxDots + threadIdx.x) * nblk + blockIdx.x] =
      red[threadIdx.x][0];
}

// hc[b * kKsMaxDots + i] = sum of the partials (fixed order); accumulate into H column j if H
__global__ void ks_hcol_kernel(int B, int k, const double* __restrict__ part, int nblk,
                               double* __restrict__ hc, double* __restrict__ H, int ldh, int j,
                               const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  for (int i = 0; i < k; ++i) {
    double s = 0.0;
    for (int t = 0; t < nblk; ++t) s += part[((size_t)b * kKsMaxDots + i) * nblk + t];
    if (!(s == s) || !(fabs(s) < 1e300)) s = 0.0;
    hc[(size_t)b * kKsMaxDots + i] = s;
    if (H) H[((size_t)b * (ldh + 1) + i) * ldh + j] += s;
  }
}

// w -= sum_i hc_i v_i  (and the block partial sums of w * w into part[(b*kKsMaxDots)*nblk + blk])
template <typename T>
__global__ void __launch_bounds__(256) ks_orth_kernel(long long N, int k, T* __restrict__ w,
                                                      const T* __restrict__ V, long long ldv,
                                                      const double* __restrict__ hc,
                                                      const int* __restrict__ active,
                                                      double* __restrict__ part, int nblk) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  const long long chunk = (N + nblk - 1) / nblk;
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < N ? lo + chunk : N;
  double h[kKsMaxDots];
  for (int i = 0; i < k; ++i) h[i] = hc[(size_t)b * kKsMaxDots + i];
  double acc = 0.0;
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    double v = (double)w[base + e];
    for (int i = 0; i < k; ++i) v -= h[i] * (double)V[(long long)i * ldv + base + e];
    const T tv = (T)v;
    w[base + e] = tv;
    acc += (double)tv * (double)tv;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[((size_t)b * kKsMaxDots) * nblk + blockIdx.x] = red[0];
}

// nrm[b] = sqrt(sum of the partials); inv[b] = 1 / nrm (0 when the norm vanishes); if H, it is
// stored as H(j+1, j); if beta0, as the initial residual norm
__global__ void ks_norm_kernel(int B, const double* __restrict__ part, int nblk,
                               double* __restrict__ inv, double* __restrict__ H, int ldh, int j,
                               double* __restrict__ beta0, const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  double s = 0.0;
  for (int t = 0; t < nblk; ++t) s += part[((size_t)b * kKsMaxDots) * nblk + t];
  double nrm = sqrt(s);
  if (!(nrm == nrm) || !(nrm < 1e300)) nrm = 0.0;
  inv[b] = nrm > 1e-300 ? 1.0 / nrm : 0.0;
  if (H) H[((size_t)b * (ldh + 1) + j + 1) * ldh + j] = nrm;
  if (beta0) beta0[b] = nrm;
}

template <typename T>
__global__ void __launch_bounds__(256) ks_scale_kernel(long long N, const T* __restrict__ src,
                                                       T* __restrict__ dst,
                                                       const double* __restrict__ sc,
                                                       const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  const double f = sc[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = (T)((double)src[base + i] * f);
}

__global__ void ks_zero_kernel(int n, double* __restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = 0.0;
}

// Least squares min || beta0 e_1 - H y || of the (k+1) x k Hessenberg matrix of every solve by
// Givens rotations (one thread per solve); columns whose rotated diagonal vanishes get y = 0.
__global__ void ks_lsq_kernel(int B, int k, const double* __restrict__ H,
                              const double* __restrict__ beta0, double* __restrict__ y,
                              const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  double R[kKsMaxDots][kKsMaxDots], g[kKsMaxDots + 1], cs[kKsMaxDots], sn[kKsMaxDots];
  const double* Hb = H + (size_t)b * (k + 1) * k;
  for (int i = 0; i <= k; ++i) g[i] = 0.0;
  g[0] = beta0[b];
  for (int j = 0; j < k; ++j) {
    double col[kKsMaxDots + 1];
    for (int i = 0; i <= k; ++i) col[i] = i <= j + 1 ? Hb[i * k + j] : 0.0;
    for (int i = 0; i < j; ++i) {  // earlier rotations
      const double t = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t;
    }
    const double a = col[j], c2 = col[j + 1];
    const double r = hypot(a, c2);
    if (r > 0.0) {
      cs[j] = a / r;
      sn[j] = c2 / r;
    } else {
      cs[j] = 1.0;
      sn[j] = 0.0;
    }
    col[j] = r;
    col[j + 1] = 0.0;
    const double t = cs[j] * g[j] + sn[j] * g[j + 1];
    g[j + 1] = -sn[j] * g[j] + cs[j] * g[j + 1];
    g[j] = t;
    for (int i = 0; i <= j; ++i) R[i][j] = col[i];
  }
  const double scale = fabs(R[0][0]);
  for (int j = k - 1; j >= 0; --j) {
    double v = g[j];
    for (int i = j + 1; i < k; ++i) v -= R[j][i] * y[(size_t)b * kKsMaxDots + i];
    const double dgl = R[j][j];
    y[(size_t)b * kKsMaxDots + j] = fabs(dgl) > 1e-14 * scale && dgl != 0.0 ? v / dgl : 0.0;
  }
}

// xout = xin + sum_j y_j z_j
template <typename T>
__global__ void __launch_bounds__(256) ks_combine_kernel(long long N, int k, const T* __restrict__ xin,
                                                         T* __restrict__ xout,
                                                         const T* __restrict__ Z, long long ldz,
                                                         const double* __restrict__ y,
                                                         const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  double yy[kKsMaxDots];
  for (int j = 0; j < k; ++j) yy[j] = y[(size_t)b * kKsMaxDots + j];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double v = (double)xin[base + i];
    for (int j = 0; j < k; ++j) v += yy[j] * (double)Z[(long long)j * ldz + base + i];
    xout[base + i] = (T)v;
  }
}

// PCG scalars from block partial sums (fixed order): mode 0: rz = sum; mode 1: a = rz / sum (the
// sum being p.q; 0 unless positive and finite); mode 2: bc = sum / rz, then rz = sum.
__global__ void ks_pcg_scalar_kernel(int B, int mode, const double* __restrict__ part, int nblk,
                                     double* __restrict__ rz, double* __restrict__ a,
                                     double* __restrict__ bc, const int* __restrict__ active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  double sm = 0.0;
  for (int t = 0; t < nblk; ++t) sm += part[(size_t)b * nblk + t];
  if (!(sm == sm) || !(fabs(sm) < 1e300)) sm = 0.0;
  if (mode == 0) {
    rz[b] = sm;
  } else if (mode == 1) {
    const double q = rz[b] / sm;
    a[b] = (sm > 0.0 && q == q && fabs(q) < 1e300) ? q : 0.0;
  } else {
    bc[b] = rz[b] > 0.0 ? sm / rz[b] : 0.0;
    rz[b] = sm;
  }
}

// x += a p; r -= a q
template <typename T>
__global__ void __launch_bounds__(256) ks_cg_update_kernel(long long N, T* __restrict__ x,
                                                           T* __restrict__ r,
                                                           const T* __restrict__ p,
                                                           const T* __restrict__ q,
                                                           const double* __restrict__ a,
                                                           const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  const double al = a[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    x[base + i] = (T)((double)x[base + i] + al * (double)p[base + i]);
    r[base + i] = (T)((double)r[base + i] - al * (double)q[base + i]);
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256) ks_xpay_kernel(long long N, const T* __restrict__ z,
                                                      T* __restrict__ p,
                                                      const double* __restrict__ be,
                                                      const int* __restrict__ active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const long long base = (long long)b * N;
  const double bt = be[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    p[base + i] = (T)((double)z[base + i] + bt * (double)p[base + i]);
}

inline dim3 vgrid(long long N, int B) {
  long long bl = (N + 255) / 256;
  if (bl > 512) bl = 512;
  return dim3((unsigned)bl, B);
}

}  // namespace

template <typename T>
static void ks_tsolve(MgData& mg, int B, const T* in, T* out, const int* active, cudaStream_t s) {
  const T* Lb = (const T*)(sizeof(T) == 8 ? mg.tLb64 : mg.tLb32);
  const T* dinv = (const T*)(sizeof(T) == 8 ? mg.tdinv64 : mg.tdinv32);
  launch_tband<T>(mg.d, mg.ml[0], mg.P - 1, B, Lb, dinv, in, out, active, s);
}

template <typename T>
static const T* fine_bands(const MgData& mg) {
  if (sizeof(T) == 8) return reinterpret_cast<const T*>(mg.bands64 + mg.boff[0]);
  return reinterpret_cast<const T*>(mg.bands32 + mg.boff[0]);
}

// Gram-Schmidt of w against V_0..V_{k-1}, applied twice (one multi-dot and one update kernel per
// pass); the coefficients are added into column j of H.  k = 0 only forms the partial sums of
// ||w||^2.  On exit mg.ks_part holds the partials of ||w||^2 (slot 0 of the multi-dot layout).
template <typename T>
static void ks_orthogonalise(MgData& mg, int B, int k, T* w, const T* V, long long ldv, int j,
                             const int* active, cudaStream_t s) {
  const long long N = mg.Nl[0];
  const int nb = partial_blocks(N);
  const int ldh = mg.ks_steps;
  for (int pass = 0; pass < (k > 0 ? 2 : 1); ++pass) {
    if (k > 0) {
      ks_mdot_kernel<T><<<dim3(nb, B), 256, 0, s>>>(N, k, w, V, ldv, active, mg.ks_part, nb);
      ks_hcol_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, k, mg.ks_part, nb, mg.ks_hc, mg.ks_H, ldh,
                                                     j, active);
      count_launch(2);
    }
    ks_orth_kernel<T><<<dim3(nb, B), 256, 0, s>>>(N, k, w, V, ldv, mg.ks_hc, active, mg.ks_part, nb);
    count_launch();
  }
}

// xout = xin + `steps` iterations of right-preconditioned GMRES on A x = b from xin, no restart:
// minimises ||b - A (xin + Z y)|| over Z = T^{-1} V, V an orthonormal basis of the Krylov space
// of A T^{-1} started from the residual (the PGMRES post-smoother of Section 6.1).
template <typename T>
void ks_pgmres(MgData& mg, int B, const T* b, const T* xin, T* xout, Coef c, const int* active,
               T* scr, cudaStream_t s) {
  const int k = mg.ks_steps;
  const long long N = mg.Nl[0];
  const int nb = partial_blocks(N);
  const int m = mg.ml[0];
  const T* bands = fine_bands<T>(mg);
  T* V = (T*)(sizeof(T) == 8 ? mg.ks64 : mg.ks32);
  const long long ld = (long long)N * mg.B;
  T* Z = V + (long long)(k + 1) * ld;
  ks_zero_kernel<<<(B * (k + 1) * k + 255) / 256, 256, 0, s>>>(B * (k + 1) * k, mg.ks_H);
  count_launch();
  launch_apply<T>(mg.d, m, mg.P, bands, xin, V, b, 1, B, c, nullptr, nullptr, active, scr, s);
  ks_orthogonalise<T>(mg, B, 0, V, V, ld, 0, active, s);  // partials of r.r
  ks_norm_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mg.ks_part, nb, mg.ks_inv, nullptr, k, 0,
                                                 mg.ks_beta0, active);
  ks_scale_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, V, V, mg.ks_inv, active);
  count_launch(2);
  for (int j = 0; j < k; ++j) {
    T* Vj = V + (long long)j * ld;
    T* Zj = Z + (long long)j * ld;
    T* W = V + (long long)(j + 1) * ld;
    ks_tsolve<T>(mg, B, Vj, Zj, active, s);
    launch_apply<T>(mg.d, m, mg.P, bands, Zj, W, nullptr, 0, B, c, nullptr, nullptr, active, scr, s);
    ks_orthogonalise<T>(mg, B, j + 1, W, V, ld, j, active, s);
    ks_norm_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mg.ks_part, nb, mg.ks_inv, mg.ks_H, k, j,
                                                   nullptr, active);
    ks_scale_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, W, W, mg.ks_inv, active);
    count_launch(2);
  }
  ks_lsq_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, k, mg.ks_H, mg.ks_beta0, mg.ks_y, active);
  ks_combine_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, k, xin, xout, Z, ld, mg.ks_y, active);
  count_launch(2);
}

// xout = xin + `steps` PCG iterations on A x = b from xin with the preconditioner T (the PCG
// post-smoother of Section 6.1, used by P_WL).
template <typename T>
void ks_pcg(MgData& mg, int B, const T* b, const T* xin, T* xout, Coef c, const int* active,
            T* scr, cudaStream_t s) {
  const int k = mg.ks_steps;
  const long long N = mg.Nl[0];
  const int nb = partial_blocks(N);
  const int m = mg.ml[0];
  const T* bands = fine_bands<T>(mg);
  T* base = (T*)(sizeof(T) == 8 ? mg.ks64 : mg.ks32);
  const long long ld = (long long)N * mg.B;
  T *R = base, *Zv = base + ld, *Pv = base + 2 * ld, *Q = base + 3 * ld;
  if (xout != xin) vcopy<T>(N, B, xin, xout, active, s);
  launch_apply<T>(mg.d, m, mg.P, bands, xout, R, b, 1, B, c, nullptr, nullptr, active, scr, s);
  ks_tsolve<T>(mg, B, R, Zv, active, s);
  vcopy<T>(N, B, Zv, Pv, active, s);
  launch_dot<T>(R, Zv, N, B, mg.ks_part, nb, active, s);
  ks_pcg_scalar_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, 0, mg.ks_part, nb, mg.ks_rz, nullptr,
                                                       nullptr, active);
  count_launch();
  for (int it = 0; it < k; ++it) {
    launch_apply<T>(mg.d, m, mg.P, bands, Pv, Q, nullptr, 0, B, c, nullptr, nullptr, active, scr, s);
    launch_dot<T>(Pv, Q, N, B, mg.ks_part, nb, active, s);
    ks_pcg_scalar_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, 1, mg.ks_part, nb, mg.ks_rz, mg.ks_a,
                                                         nullptr, active);
    ks_cg_update_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, xout, R, Pv, Q, mg.ks_a, active);
    count_launch(2);
    if (it + 1 == k) break;  // the last step needs no new direction
    ks_tsolve<T>(mg, B, R, Zv, active, s);
    launch_dot<T>(R, Zv, N, B, mg.ks_part, nb, active, s);
    ks_pcg_scalar_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, 2, mg.ks_part, nb, mg.ks_rz, nullptr,
                                                         mg.ks_b, active);
    ks_xpay_kernel<T><<<vgrid(N, B), 256, 0, s>>>(N, Zv, Pv, mg.ks_b, active);
    count_launch(2);
  }
}

template void ks_pgmres<double>(MgData&, int, const double*, const double*, double*, Coef,
                                const int*, double*, cudaStream_t);
template void ks_pgmres<float>(MgData&, int, const float*, const float*, float*, Coef, const int*,
                               float*, cudaStream_t);
template void ks_pcg<double>(MgData&, int, const double*, const double*, double*, Coef,
                             const int*, double*, cudaStream_t);
template void ks_pcg<float>(MgData&, int, const float*, const float*, float*, Coef, const int*,
                            float*, cudaStream_t);

}  // namespace cd
