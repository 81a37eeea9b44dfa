"""1D IgA matrices (Section 3.2) and the 1D factor of the preconditioner T (Section 6.1).

Test infrastructure only (see ``oracle/__init__.py``).

M, A, S are eq:matr_M, eq:matr_A, eq:matr_S: Galerkin integrals of the
B-splines N_2..N_{n+p-1} (the ones that vanish at 0 and 1, eq:spline-boundary),
so each is m x m with m = n + p - 2.  They are computed by Gauss-Legendre
quadrature on every knot interval; the integrands are piecewise polynomials of
degree <= 2p, so p+1 points per interval integrate them exactly.
"""
from fractions import Fraction

import numpy as np

from . import bspline


def gauss_points(n, nq):
    """Gauss-Legendre points and weights, nq per interval [i/n, (i+1)/n], i = 0..n-1."""
    g, w = np.polynomial.legendre.leggauss(nq)
    left = np.arange(n, dtype=np.float64)[:, None] / n
    x = (left + (g[None, :] + 1.0) / (2.0 * n)).ravel()
    wt = np.tile(w / (2.0 * n), n)
    return x, wt


def eval_interior(p, n, x):
    """Values and derivatives of N_2..N_{n+p-1} at x: two arrays [len(x), m]."""
    v = bspline.basis(p, n, x)[:, 1:n + p - 1]
    g = bspline.basis_deriv(p, n, x)[:, 1:n + p - 1]
    return v, g


def full_matrices(p, n, nq=None):
    """M, A, S over all n+p B-splines (before the Dirichlet restriction)."""
    nq = nq or p + 1
    x, w = gauss_points(n, nq)
    v = bspline.basis(p, n, x)
    g = bspline.basis_deriv(p, n, x)
    M = v.T @ (w[:, None] * v)
    A = v.T @ (w[:, None] * g)  # A_ij = int N_i N_j'
    S = g.T @ (w[:, None] * g)
    return M, A, S


def matrices(p, n, nq=None):
    """(M, A, S) of eq:matr_M / eq:matr_A / eq:matr_S, each dense m x m, m = n+p-2."""
    M, A, S = full_matrices(p, n, nq)
    sl = slice(1, n + p - 1)
    return M[sl, sl].copy(), A[sl, sl].copy(), S[sl, sl].copy()


def interior_entry_exact(p, n, i, j, which):
    """Exact central entry of M, A or S for 1-based i, j in 2p..n-p-1 (Section 3.2).

    (M)_ij = phi_{2p+1}(p+1-(i-j)) / n, (A)_ij = -phi'_{2p+1}(p+1-(i-j)),
    (S)_ij = -n phi''_{2p+1}(p+1-(i-j)).
    """
    t = p + 1 - (i - j)
    q = 2 * p + 1
    if which == "M":
        return bspline.cardinal(q, t) / n
    if which == "A":
        return -bspline.cardinal(q, t, 1)
    if which == "S":
        return -n * bspline.cardinal(q, t, 2)
    raise ValueError(which)


def toeplitz_T(p, m):
    """T_m(m_{p-1}) of Section 6.1: entries phi_{2p-1}(p - i + j) for |i - j| < p, else 0."""
    T = np.zeros((m, m))
    for i in range(m):
        for j in range(max(0, i - p + 1), min(m, i + p)):
            T[i, j] = float(bspline.cardinal(2 * p - 1, p - i + j))
    return T


def toeplitz_T_exact_row(p):
    """The 2p-1 distinct coefficients phi_{2p-1}(p + k), k = -(p-1)..p-1, as Fractions."""
    return [bspline.cardinal(2 * p - 1, Fraction(p + k)) for k in range(-(p - 1), p)]
