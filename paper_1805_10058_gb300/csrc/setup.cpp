// Host setup (FP64): 1D IgA bands, the Toeplitz factor of T, Galerkin coarsening of
// bands, and small dense eigen-decompositions.  All of it is O(m p^2) or O(m^3) with
// m <= a few hundred and runs once per (p, n); results are cached by the solver.
#include <algorithm>
#include <limits>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include "cd_internal.h"

namespace cd {

// ------------------------------------------------------------------ errors / counters
static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};  // process-wide: solves may run on several threads
void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }
void count_launch(int k) { g_launches.fetch_add((uint64_t)(int64_t)k, std::memory_order_relaxed); }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ quadrature
// Gauss-Legendre nodes on [-1, 1] by Newton iteration on the Legendre polynomial of
// degree nq (three-term recurrence (k) P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}).
static void gauss_legendre(int nq, std::vector<double>& x, std::vector<double>& w) {
  x.assign(nq, 0.0);
  w.assign(nq, 0.0);
  for (int i = 0; i < nq; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (nq + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= nq; ++k) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = nq * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= nq; ++k) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = nq * (z * p0 - p1) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Values and first derivatives of the p+1 B-splines that are nonzero on knot span s
// (xi[s] <= x < xi[s+1]), by the Cox-de Boor triangle; N[j] is N_{s-p+j}.
static void eval_span(int p, const std::vector<double>& xi, int s, double x, double* N,
                      double* dN) {
  std::vector<double> tri((size_t)(p + 1) * (p + 1), 0.0);
  auto T = [&](int k, int j) -> double& { return tri[(size_t)k * (p + 1) + j]; };
  T(0, 0) = 1.0;
  for (int k = 1; k <= p; ++k) {
    for (int j = 0; j <= k; ++j) {
      int i = s - k + j;
      double v = 0.0;
      if (j >= 1) {
        double den = xi[i + k] - xi[i];
        if (den > 0) v += (x - xi[i]) / den * T(k - 1, j - 1);
      }
      if (j <= k - 1) {
        double den = xi[i + k + 1] - xi[i + 1];
        if (den > 0) v += (xi[i + k + 1] - x) / den * T(k - 1, j);
      }
      T(k, j) = v;
    }
  }
  for (int j = 0; j <= p; ++j) {
    N[j] = T(p, j);
    int i = s - p + j;
    double dv = 0.0;
    if (p >= 1) {
      if (j >= 1) {
        double den = xi[i + p] - xi[i];
        if (den > 0) dv += p * T(p - 1, j - 1) / den;
      }
      if (j <= p - 1) {
        double den = xi[i + p + 1] - xi[i + 1];
        if (den > 0) dv -= p * T(p - 1, j) / den;
      }
    }
    dN[j] = dv;
  }
}

void iga_bands(int p, int n, int P, Band& M, Band& A, Band& S) {
  const int nf = n + p;  // all B-splines of degree p
  std::vector<double> xi(n + 2 * p + 1);
  for (int i = 0; i < (int)xi.size(); ++i)
    xi[i] = i <= p ? 0.0 : (i >= n + p ? 1.0 : double(i - p) / n);
  const int W = 2 * p + 1;
  std::vector<double> Mf((size_t)nf * W, 0.0), Af((size_t)nf * W, 0.0), Sf((size_t)nf * W, 0.0);
  std::vector<double> g, gw;
  gauss_legendre(p + 1, g, gw);  // degree-2p integrands: exact
  std::vector<double> N(p + 1), dN(p + 1);
  for (int e = 0; e < n; ++e) {
    const int s = e + p;
    const double a = double(e) / n, b = double(e + 1) / n;
    for (int q = 0; q <= p; ++q) {
      const double x = a + (b - a) * 0.5 * (g[q] + 1.0);
      const double wq = gw[q] * 0.5 * (b - a);
      eval_span(p, xi, s, x, N.data(), dN.data());
      for (int j1 = 0; j1 <= p; ++j1)
        for (int j2 = 0; j2 <= p; ++j2) {
          const int i1 = s - p + j1, i2 = s - p + j2;
          const size_t at = (size_t)i1 * W + (i2 - i1 + p);
          Mf[at] += wq * N[j1] * N[j2];
          Af[at] += wq * N[j1] * dN[j2];  // int N_i N_j'
          Sf[at] += wq * dN[j1] * dN[j2];
        }
    }
  }
  const int m = nf - 2;
  const int WP = 2 * P + 1;
  for (Band* X : {&M, &A, &S}) {
    X->m = m;
    X->P = P;
    X->v.assign((size_t)m * WP, 0.0);
  }
  for (int i = 0; i < m; ++i)
    for (int k = -p; k <= p; ++k) {
      const int j = i + k;
      if (j < 0 || j >= m) continue;
      const size_t src = (size_t)(i + 1) * W + (k + p), srcT = (size_t)(j + 1) * W + (-k + p);
      const size_t dst = (size_t)i * WP + (k + P);
      M.v[dst] = 0.5 * (Mf[src] + Mf[srcT]);
      S.v[dst] = 0.5 * (Sf[src] + Sf[srcT]);
      A.v[dst] = 0.5 * (Af[src] - Af[srcT]);  // exactly skew: A^T = -A
    }
}

// Cardinal B-spline phi_q(t) by the recursion phi_q(t) = t/q phi_{q-1}(t) +
// (q+1-t)/q phi_{q-1}(t-1), phi_0 = indicator of [0, 1).
static double cardinal(int q, double t) {
  if (q == 0) return (t >= 0.0 && t < 1.0) ? 1.0 : 0.0;
  return t / q * cardinal(q - 1, t) + (q + 1 - t) / q * cardinal(q - 1, t - 1.0);
}

void toeplitz_T_band(int p, int m, int P, Band& T) {
  T.m = m;
  T.P = P;
  T.v.assign((size_t)m * (2 * P + 1), 0.0);
  for (int i = 0; i < m; ++i)
    for (int k = -(p - 1); k <= p - 1; ++k) {
      const int j = i + k;
      if (j < 0 || j >= m) continue;
      T.v[(size_t)i * (2 * P + 1) + (k + P)] = cardinal(2 * p - 1, double(p + k));
    }
}

bool tband_factor(int p, int m, std::vector<double>& Lb, std::vector<double>& dinv) {
  const int q = p - 1, P = p, W = 2 * P + 1;
  Band T;
  toeplitz_T_band(p, m, P, T);
  std::vector<double> L((size_t)m * (q + 1), 0.0);  // L[i][t] = L(i, i - q + t), t = q diagonal
  auto Lij = [&](int i, int j) -> double& { return L[(size_t)i * (q + 1) + (j - i + q)]; };
  for (int i = 0; i < m; ++i)
    for (int j = std::max(0, i - q); j <= i; ++j) {
      double s = T.v[(size_t)i * W + (j - i + P)];
      for (int k = std::max(0, i - q); k < j; ++k) s -= Lij(i, k) * Lij(j, k);
      if (i == j) {
        if (!(s > 0.0)) return false;
        Lij(i, i) = std::sqrt(s);
      } else {
        Lij(i, j) = s / Lij(j, j);
      }
    }
  Lb.assign((size_t)(m + q) * q, 0.0);
  dinv.assign(m, 0.0);
  for (int i = 0; i < m; ++i) {
    for (int t = 0; t < q; ++t)
      if (i - q + t >= 0) Lb[(size_t)i * q + t] = Lij(i, i - q + t);
    dinv[i] = 1.0 / Lij(i, i);
  }
  return true;
}

Band coarsen(const Band& X) {
  // Xc = P1^T X P1 with column J of P1 holding (1/2, 1, 1/2) on rows 2J, 2J+1, 2J+2
  // (0-based; rows >= m dropped).  The coarse half-band stays <= P.
  static const double wt[3] = {0.5, 1.0, 0.5};
  Band C;
  C.m = X.m / 2;
  C.P = X.P;
  const int WP = 2 * C.P + 1;
  C.v.assign((size_t)C.m * WP, 0.0);
  for (int I = 0; I < C.m; ++I)
    for (int J = std::max(0, I - C.P); J <= std::min(C.m - 1, I + C.P); ++J) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const int i = 2 * I + a, j = 2 * J + b;
          if (i < X.m && j < X.m) s += wt[a] * wt[b] * X.at(i, j);
        }
      C.v[(size_t)I * WP + (J - I + C.P)] = s;
    }
  return C;
}

std::vector<double> band_to_dense(const Band& X) {
  std::vector<double> D((size_t)X.m * X.m, 0.0);
  for (int i = 0; i < X.m; ++i)
    for (int j = std::max(0, i - X.P); j <= std::min(X.m - 1, i + X.P); ++j)
      D[(size_t)i * X.m + j] = X.at(i, j);
  return D;
}

// Cyclic Jacobi eigen-decomposition of a dense symmetric matrix (row-major, FP64):
// rotations chosen to annihilate a_pq (Golub & Van Loan, symmetric Schur step).
// Symmetric eigen-decomposition A = U diag(lam) U^T, lam ascending, U orthogonal (columns =
// eigenvectors).  Householder reduction to tridiagonal form, then implicit symmetric QR steps
// with the Wilkinson shift (Golub & Van Loan, Matrix Computations, Sections 8.3.1-8.3.3).  The
// orthogonal factor is kept transposed (row j of Qt = column j of Q) so that every reflection
// and rotation updates contiguous rows.
bool sym_eig(int m, const std::vector<double>& Ain, std::vector<double>& U,
             std::vector<double>& lam) {
  std::vector<double> a = Ain, Qt((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Qt[(size_t)i * m + i] = 1.0;
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * m + j]; };
  // 1. tridiagonalisation: for column k, the reflection H = I - tau v v^T (v on rows k+1..)
  //    maps A(k+1.., k) to alpha e_1; the trailing block becomes H B H = B - v w^T - w v^T with
  //    p = tau B v, w = p - (tau/2)(p^T v) v; Q <- Q H.
  std::vector<double> v(m), pv(m), u(m);
  for (int k = 0; k + 2 < m; ++k) {
    const int n0 = k + 1, len = m - n0;
    double nrm = 0.0;
    for (int i = 0; i < len; ++i) nrm += A(n0 + i, k) * A(n0 + i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double x0 = A(n0, k);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    for (int i = 0; i < len; ++i) v[i] = A(n0 + i, k);
    v[0] = x0 - alpha;
    double vv = 0.0;
    for (int i = 0; i < len; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double tau = 2.0 / vv;
    for (int i = 0; i < len; ++i) {  // p = tau B v
      const double* row = &a[(size_t)(n0 + i) * m + n0];
      double sum = 0.0;
      for (int j = 0; j < len; ++j) sum += row[j] * v[j];
      pv[i] = tau * sum;
    }
    double pTv = 0.0;
    for (int i = 0; i < len; ++i) pTv += pv[i] * v[i];
    const double K = 0.5 * tau * pTv;
    for (int i = 0; i < len; ++i) pv[i] -= K * v[i];  // w
    for (int i = 0; i < len; ++i) {
      double* row = &a[(size_t)(n0 + i) * m + n0];
      const double vi = v[i], wi = pv[i];
      for (int j = 0; j < len; ++j) row[j] -= vi * pv[j] + wi * v[j];
    }
    A(n0, k) = A(k, n0) = alpha;
    for (int i = 1; i < len; ++i) A(n0 + i, k) = A(k, n0 + i) = 0.0;
    // Q <- Q H: rows n0.. of Qt: Qt_j -= tau v_j (sum_l v_l Qt_l)
    std::fill(u.begin(), u.end(), 0.0);
    for (int l = 0; l < len; ++l) {
      const double* row = &Qt[(size_t)(n0 + l) * m];
      const double vl = v[l];
      for (int i = 0; i < m; ++i) u[i] += vl * row[i];
    }
    for (int l = 0; l < len; ++l) {
      double* row = &Qt[(size_t)(n0 + l) * m];
      const double f = tau * v[l];
      for (int i = 0; i < m; ++i) row[i] -= f * u[i];
    }
  }
  std::vector<double> d(m), e(std::max(m - 1, 1), 0.0);
  for (int i = 0; i < m; ++i) d[i] = A(i, i);
  for (int i = 0; i + 1 < m; ++i) e[i] = A(i + 1, i);
  // 2. implicit QR steps on the unreduced block [l, h] of the tridiagonal (d, e)
  auto rotate_rows = [&](int k, double c, double s) {  // Q <- Q R^T on columns k, k+1
    double* rk = &Qt[(size_t)k * m];
    double* rk1 = &Qt[(size_t)(k + 1) * m];
    for (int i = 0; i < m; ++i) {
      const double x = rk[i], y = rk1[i];
      rk[i] = c * x - s * y;
      rk1[i] = s * x + c * y;
    }
  };
  const double eps = std::numeric_limits<double>::epsilon();
  int h = m - 1, iters = 0;
  while (h > 0) {
    for (int i = 0; i < h; ++i)
      if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    if (e[h - 1] == 0.0) {
      --h;
      continue;
    }
    int l = h - 1;
    while (l > 0 && e[l - 1] != 0.0) --l;
    if (++iters > 60 * m) return false;
    // Wilkinson shift from the trailing 2 x 2 block
    const double del = 0.5 * (d[h - 1] - d[h]), bh = e[h - 1];
    const double mu = d[h] - bh * bh / (del + (del >= 0.0 ? 1.0 : -1.0) * std::hypot(del, bh));
    double x = d[l] - mu, z = e[l];
    for (int k = l; k < h; ++k) {
      // rotation R = [[c, -s], [s, c]] on rows / columns k, k+1 with R [x; z] = [r; 0]
      const double r = std::hypot(x, z);
      const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : -z / r;
      if (k > l) e[k - 1] = r;  // the bulge at (k+1, k-1) is annihilated
      const double ak = d[k], bk = e[k], qk = d[k + 1];
      d[k] = c * c * ak - 2.0 * c * s * bk + s * s * qk;
      d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * qk;
      e[k] = c * s * (ak - qk) + (c * c - s * s) * bk;
      if (k + 1 < h) {  // the column rotation reaches row k+2: new bulge at (k+2, k)
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      rotate_rows(k, c, s);
    }
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return d[x] < d[y]; });
  lam.resize(m);
  U.assign((size_t)m * m, 0.0);
  for (int c = 0; c < m; ++c) {
    lam[c] = d[order[c]];
    const double* q = &Qt[(size_t)order[c] * m];
    for (int i = 0; i < m; ++i) U[(size_t)i * m + c] = q[i];
  }
  return true;
}

static bool cholesky(int m, std::vector<double>& L) {  // in place, lower triangle
  for (int j = 0; j < m; ++j) {
    double s = L[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    if (!(s > 0)) return false;
    const double d = std::sqrt(s);
    L[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double t = L[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = t / d;
    }
    for (int k = j + 1; k < m; ++k) L[(size_t)j * m + k] = 0.0;
  }
  return true;
}

bool gen_eig(int m, const std::vector<double>& Md, const std::vector<double>& Sd,
             std::vector<double>& U, std::vector<double>& lam) {
  std::vector<double> L = Md;
  if (!cholesky(m, L)) return false;
  // Y = L^{-1} S (forward substitution column by column), C = L^{-1} Y^T
  std::vector<double> Y = Sd, C((size_t)m * m);
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      double s = Y[(size_t)i * m + c];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * Y[(size_t)k * m + c];
      Y[(size_t)i * m + c] = s / L[(size_t)i * m + i];
    }
  for (int c = 0; c < m; ++c)  // column c of C = L^{-1} (row c of Y)^T
    for (int i = 0; i < m; ++i) {
      double s = Y[(size_t)c * m + i];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * C[(size_t)k * m + c];
      C[(size_t)i * m + c] = s / L[(size_t)i * m + i];
    }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double v = 0.5 * (C[(size_t)i * m + j] + C[(size_t)j * m + i]);
      C[(size_t)i * m + j] = C[(size_t)j * m + i] = v;
    }
  std::vector<double> V;
  sym_eig(m, C, V, lam);
  // U = L^{-T} V (back substitution)
  U.assign((size_t)m * m, 0.0);
  for (int c = 0; c < m; ++c)
    for (int i = m - 1; i >= 0; --i) {
      double s = V[(size_t)i * m + c];
      for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * U[(size_t)k * m + c];
      U[(size_t)i * m + c] = s / L[(size_t)i * m + i];
    }
  return true;
}

bool spd_inverse(int n, std::vector<double>& a) {
  std::vector<double> L = a;
  if (!cholesky(n, L)) return false;
  // inverse column by column: L L^T x = e_c
  std::vector<double> inv((size_t)n * n, 0.0), y(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
      y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * inv[(size_t)k * n + c];
      inv[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
  }
  a.swap(inv);
  return true;
}

}  // namespace cd
