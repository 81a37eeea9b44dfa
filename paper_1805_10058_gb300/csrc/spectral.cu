// Spectral validation on the GPU (Section 5): the d x d matrix-valued symbol f^{p,alpha,beta} of
// Theorem 5.1 (eq:f2D) / Theorem 5.5 (eq:f3D) and its eigenvalue functions sampled on the grid
// Gamma of Section 5.3, the Laplacian symbol (eq:lapl2D / eq:lapl3D) that bounds them
// (Theorems 5.2 / 5.6), and Lanczos estimates of the extremal eigenvalues of the matrix A itself.
//
// The 1D symbols (Theorem 3.1) are trigonometric polynomials whose coefficients are cardinal
// B-spline values at the integers: m_p uses phi_{2p+1}(p+1-k), a_p the first derivative and s_p
// the second, phi'_q(t) = phi_{q-1}(t) - phi_{q-1}(t-1) (Section 3.1).  They are formed on the host
// once and passed to the kernel; cos(k theta), sin(k theta) follow from one sincospi by the
// Chebyshev recurrences.  The eigenvalues of the 3 x 3 symbol are found by cyclic Jacobi rotations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "krylov.h"

namespace cd {

namespace {

constexpr int kMaxP = 8;

struct SymbolCoef {
  int p;
  double cm[kMaxP + 1], ca[kMaxP + 1], cs[kMaxP + 1];
  double alpha, beta;
  double wdiag[3];   // 2D: nu2/nu1, nu1/nu2; 3D: gamma_1..3
  double wcoup[3];   // 3D: delta_1..3 (2D: unused, 1)
};

double card(int q, double t) {
  if (q == 0) return (t >= 0.0 && t < 1.0) ? 1.0 : 0.0;
  return t / q * card(q - 1, t) + (q + 1 - t) / q * card(q - 1, t - 1.0);
}
double card_d1(int q, double t) { return card(q - 1, t) - card(q - 1, t - 1.0); }
double card_d2(int q, double t) { return card(q - 2, t) - 2.0 * card(q - 2, t - 1.0) + card(q - 2, t - 2.0); }

// m_p, a_p, s_p at theta = k pi / mg (Theorem 3.1)
__device__ __forceinline__ void sym1d(const SymbolCoef& c, int k, int mg, double& mv, double& av,
                                      double& sv) {
  double sn, cn;
  sincospi((double)k / (double)mg, &sn, &cn);
  double ck = 1.0, ckm = cn, sk = 0.0, skm = -sn;  // cos/sin of (j theta) and ((j-1) theta)
  mv = c.cm[0];
  av = 0.0;
  sv = -c.cs[0];
  for (int j = 1; j <= c.p; ++j) {
    const double cj = 2.0 * cn * ck - ckm, sj = 2.0 * cn * sk - skm;
    ckm = ck;
    ck = cj;
    skm = sk;
    sk = sj;
    mv += 2.0 * c.cm[j] * cj;
    av += -2.0 * c.ca[j] * sj;
    sv += -2.0 * c.cs[j] * cj;
  }
}

__device__ __forceinline__ void jacobi3(double a[3][3], double ev[3]) {
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    const double dg = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
    if (off <= 1e-300 + 1e-18 * dg) break;
    for (int pp = 0; pp < 2; ++pp)
      for (int q = pp + 1; q < 3; ++q) {
        const double apq = a[pp][q];
        if (apq == 0.0) continue;
        const double theta = (a[q][q] - a[pp][pp]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < 3; ++r) {  // columns pp, q
          const double x = a[r][pp], y = a[r][q];
          a[r][pp] = cs * x - sn * y;
          a[r][q] = sn * x + cs * y;
        }
        for (int r = 0; r < 3; ++r) {  // rows pp, q
          const double x = a[pp][r], y = a[q][r];
          a[pp][r] = cs * x - sn * y;
          a[q][r] = sn * x + cs * y;
        }
      }
  }
  ev[0] = a[0][0];
  ev[1] = a[1][1];
  ev[2] = a[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (ev[j] > ev[j + 1]) {
        const double t = ev[j];
        ev[j] = ev[j + 1];
        ev[j + 1] = t;
      }
}

// one thread per grid point (k_1, .., k_d), k_l = 1..mg: eigenvalues ascending, Laplacian symbol
__global__ void __launch_bounds__(256) symbol_eigs_kernel(int d, int mg, long long npts,
                                                          SymbolCoef c, double* __restrict__ lam,
                                                          double* __restrict__ lap) {
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  double mv[3], av[3], sv[3];
  long long rest = pt;
  for (int l = d - 1; l >= 0; --l) {
    const int k = (int)(rest % mg) + 1;
    rest /= mg;
    sym1d(c, k, mg, mv[l], av[l], sv[l]);
  }
  const double al = c.alpha, be = c.beta, ga = c.alpha - c.beta;
  if (d == 2) {
    const double ms = mv[0] * sv[1], sm = sv[0] * mv[1];
    const double f11 = al * c.wdiag[0] * ms + be * c.wdiag[1] * sm;
    const double f22 = al * c.wdiag[1] * sm + be * c.wdiag[0] * ms;
    const double f12 = -ga * av[0] * av[1];
    const double tr = 0.5 * (f11 + f22), df = 0.5 * (f11 - f22);
    const double r = sqrt(df * df + f12 * f12);
    lam[pt * 2 + 0] = tr - r;
    lam[pt * 2 + 1] = tr + r;
    if (lap) lap[pt] = c.wdiag[0] * ms + c.wdiag[1] * sm;
  } else {
    const double t0 = sv[0] * mv[1] * mv[2], t1 = mv[0] * sv[1] * mv[2], t2 = mv[0] * mv[1] * sv[2];
    const double g0 = c.wdiag[0] * t0, g1 = c.wdiag[1] * t1, g2 = c.wdiag[2] * t2;
    double a[3][3];
    a[0][0] = be * g0 + al * g1 + al * g2;
    a[1][1] = al * g0 + be * g1 + al * g2;
    a[2][2] = al * g0 + al * g1 + be * g2;
    a[0][1] = a[1][0] = -ga * c.wcoup[2] * av[0] * av[1] * mv[2];
    a[0][2] = a[2][0] = -ga * c.wcoup[1] * av[0] * mv[1] * av[2];
    a[1][2] = a[2][1] = -ga * c.wcoup[0] * mv[0] * av[1] * av[2];
    double ev[3];
    jacobi3(a, ev);
    lam[pt * 3 + 0] = ev[0];
    lam[pt * 3 + 1] = ev[1];
    lam[pt * 3 + 2] = ev[2];
    if (lap) lap[pt] = g0 + g1 + g2;
  }
}

// ---- Lanczos: per-solve scalars
__global__ void lz_alpha_kernel(int B, const double* __restrict__ part, int nblk, int j, int steps,
                                double* __restrict__ la, double* __restrict__ coef,
                                const int* __restrict__ live) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !live[b]) return;
  double s = 0.0;
  for (int t = 0; t < nblk; ++t) s += part[(size_t)b * nblk + t];
  la[(size_t)b * steps + j] = s;
  coef[b] = s;
}
__global__ void lz_beta_kernel(int B, const double* __restrict__ part, int nblk, int j, int steps,
                               double* __restrict__ lb, double* __restrict__ inv,
                               int* __restrict__ live, int* __restrict__ used) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !live[b]) return;
  double s = 0.0;
  for (int t = 0; t < nblk; ++t) s += part[(size_t)b * nblk + t];
  const double nrm = sqrt(s);
  lb[(size_t)b * steps + j] = nrm;
  used[b] = j + 1;
  if (!(nrm > 1e-280) || !(nrm < 1e300)) {  // invariant subspace found (or breakdown): stop here
    live[b] = 0;
    inv[b] = 0.0;
  } else {
    inv[b] = 1.0 / nrm;
  }
}
// w = (w - a v - bprev vprev) [then] vprev <- v, v <- w * inv (done by the caller's kernel below)
__global__ void __launch_bounds__(256) lz_orth_kernel(long long N, double* __restrict__ w,
                                                      const double* __restrict__ v,
                                                      const double* __restrict__ vprev,
                                                      const double* __restrict__ a,
                                                      const double* __restrict__ lbprev, int j,
                                                      int steps, const int* __restrict__ live) {
  const int b = blockIdx.y;
  if (!live[b]) return;
  const long long base = (long long)b * N;
  const double av = a[b], bv = j > 0 ? lbprev[(size_t)b * steps + j - 1] : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    w[base + i] = w[base + i] - av * v[base + i] - (j > 0 ? bv * vprev[base + i] : 0.0);
}
__global__ void __launch_bounds__(256) lz_next_kernel(long long N, const double* __restrict__ w,
                                                      double* __restrict__ v,
                                                      double* __restrict__ vprev,
                                                      const double* __restrict__ inv,
                                                      const int* __restrict__ live) {
  const int b = blockIdx.y;
  if (!live[b]) return;
  const long long base = (long long)b * N;
  const double f = inv[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    vprev[base + i] = v[base + i];
    v[base + i] = w[base + i] * f;
  }
}
__global__ void lz_norm_kernel(int B, const double* __restrict__ part, int nblk,
                               double* __restrict__ inv, int* __restrict__ live) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int t = 0; t < nblk; ++t) s += part[(size_t)b * nblk + t];
  const double nrm = sqrt(s);
  if (!(nrm > 1e-280) || !(nrm < 1e300)) {
    live[b] = 0;
    inv[b] = 0.0;
  } else {
    inv[b] = 1.0 / nrm;
  }
}
__global__ void __launch_bounds__(256) lz_scale_copy_kernel(long long N, const double* __restrict__ src,
                                                            double* __restrict__ dst,
                                                            const double* __restrict__ inv) {
  const int b = blockIdx.y;
  const long long base = (long long)b * N;
  const double f = inv[b];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[base + i] = src[base + i] * f;
}
__global__ void lz_init_kernel(int B, int* __restrict__ live, int* __restrict__ used) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    live[b] = 1;
    used[b] = 0;
  }
}

inline dim3 vgrid(long long N, int B) {
  long long bl = (N + 255) / 256;
  if (bl > 512) bl = 512;
  return dim3((unsigned)bl, B);
}

}  // namespace

// host: symbol coefficients of Theorem 3.1 and the anisotropy weights of Theorems 5.1 / 5.5
static SymbolCoef symbol_coef(int d, int p, double alpha, double beta, const double* nu) {
  SymbolCoef c{};
  c.p = p;
  const int q = 2 * p + 1;
  for (int k = 0; k <= p; ++k) {
    c.cm[k] = card(q, double(p + 1 - k));
    c.ca[k] = card_d1(q, double(p + 1 - k));
    c.cs[k] = card_d2(q, double(p + 1 - k));
  }
  c.alpha = alpha;
  c.beta = beta;
  double v[3] = {1.0, 1.0, 1.0};
  if (nu)
    for (int l = 0; l < d; ++l) v[l] = nu[l];
  if (d == 2) {
    c.wdiag[0] = v[1] / v[0];
    c.wdiag[1] = v[0] / v[1];
    c.wcoup[0] = c.wcoup[1] = c.wcoup[2] = 1.0;
  } else {
    const double prod = v[0] * v[1] * v[2];
    for (int l = 0; l < 3; ++l) {
      c.wdiag[l] = v[l] * v[l] / prod;
      c.wcoup[l] = 1.0 / v[l];
    }
  }
  return c;
}

int launch_symbol_eigs(int d, int p, double alpha, double beta, const double* nu, int mg,
                       double* lam, double* lap, cudaStream_t s) {
  if ((d != 2 && d != 3) || p < 1 || p > kMaxP || mg < 1) return 1;
  long long npts = 1;
  for (int l = 0; l < d; ++l) npts *= mg;
  const SymbolCoef c = symbol_coef(d, p, alpha, beta, nu);
  symbol_eigs_kernel<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(d, mg, npts, c, lam, lap);
  count_launch();
  return 0;
}

// `steps` Lanczos steps on the operator applied by `apply` (y = A x for B vectors of N) from
// the start vectors v0 (any nonzero vectors, normalised here): la[b * steps + j] = alpha_j,
// lb[b * steps + j] = beta_{j+1} of the tridiagonal matrix, used[b] = steps taken (fewer on an
// invariant subspace).  Workspace: v, w, vprev (B * N each), coef, inv (B), live (B), part
// (B * partial_blocks(N)).
void lanczos_run(long long N, int B, int steps, const double* v0, double* v, double* w,
                 double* vprev, double* la, double* lb, double* coef, double* inv, int* live,
                 int* used, double* part, void (*apply)(void*, const double*, double*), void* ctx,
                 cudaStream_t s) {
  const int nb = partial_blocks(N);
  lz_init_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, live, used);
  launch_dot<double>(v0, v0, N, B, part, nb, nullptr, s);
  lz_norm_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, part, nb, inv, live);
  lz_scale_copy_kernel<<<vgrid(N, B), 256, 0, s>>>(N, v0, v, inv);
  count_launch(3);
  for (int j = 0; j < steps; ++j) {
    apply(ctx, v, w);
    launch_dot<double>(w, v, N, B, part, nb, live, s);
    lz_alpha_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, part, nb, j, steps, la, coef, live);
    lz_orth_kernel<<<vgrid(N, B), 256, 0, s>>>(N, w, v, vprev, coef, lb, j, steps, live);
    launch_dot<double>(w, w, N, B, part, nb, live, s);
    lz_beta_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, part, nb, j, steps, lb, inv, live, used);
    lz_next_kernel<<<vgrid(N, B), 256, 0, s>>>(N, w, v, vprev, inv, live);
    count_launch(4);
  }
}

// Extremal eigenvalues of the symmetric tridiagonal matrix (diagonal a[0..k-1], off-diagonal
// b[0..k-2]) by bisection on the Sturm sequence count (host, FP64).
static int sturm_count(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    const double qq = q != 0.0 ? q : 1e-300;
    q = a[i] - x - b[i - 1] * b[i - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}
void tridiag_extremes(const double* a, const double* b, int k, double* lmin, double* lmax) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto kth = [&](int target) {  // smallest x with count(x) >= target
    double l = lo, h = hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (l + h);
      if (mid <= l || mid >= h) break;
      if (sturm_count(a, b, k, mid) >= target)
        h = mid;
      else
        l = mid;
    }
    return 0.5 * (l + h);
  };
  *lmin = kth(1);
  *lmax = kth(k);
}

}  // namespace cd
