// Host setup (FP64): 1D IgA bands, the Toeplitz factor of T, Galerkin coarsening of
// bands, and small dense eigen-decompositions.  All of it is O(m p^2) or O(m^3) with
// m <= a few hundred and runs once per (p, n); results are cached by the solver.
#include <algorithm>
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
bool sym_eig(int m, const std::vector<double>& Ain, std::vector<double>& U,
             std::vector<double>& lam) {
  std::vector<double> a = Ain;
  U.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) U[(size_t)i * m + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return a[(size_t)i * m + j]; };
  double fro = 0.0;
  for (double v : a) fro += v * v;
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) off += at(i, j) * at(i, j);
    if (std::sqrt(off) <= 1e-17 * fro) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = at(p, q);
        if (std::fabs(apq) <= 1e-300) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
        at(p, q) = at(q, p) = 0.0;
        for (int k = 0; k < m; ++k) {
          double* row = &U[(size_t)k * m];
          const double ukp = row[p], ukq = row[q];
          row[p] = c * ukp - s * ukq;
          row[q] = s * ukp + c * ukq;
        }
      }
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return at(x, x) < at(y, y); });
  lam.resize(m);
  std::vector<double> Us((size_t)m * m);
  for (int c = 0; c < m; ++c) {
    lam[c] = at(order[c], order[c]);
    for (int i = 0; i < m; ++i) Us[(size_t)i * m + c] = U[(size_t)i * m + order[c]];
  }
  U.swap(Us);
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
