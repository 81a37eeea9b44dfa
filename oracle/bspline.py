"""B-splines on the open uniform knot sequence and cardinal B-splines (Section 3.1).

Test infrastructure only (see ``oracle/__init__.py``).

Indices: the paper numbers the knots xi_1..xi_{2p+n+1} and the B-splines
N_1..N_{n+p} from one; arrays here are zero-based, so paper index i is
array index i-1.
"""
from fractions import Fraction

import numpy as np


def knot_vector(p, n):
    """Open uniform knots of Section 3.1: p+1 zeros, interior knots i/n, p+1 ones.

    Returns an array of length 2p+n+1 (xi_{i+p+1} = i/n for i = 0..n).
    """
    return np.concatenate([np.zeros(p), np.arange(n + 1, dtype=np.float64) / n, np.ones(p)])


def _degree0(xi, x):
    """N_i^0(x): indicator of [xi_i, xi_{i+1}) (Section 3.1 definition).

    At x == 1 the half-open convention gives all zeros; the last
    non-degenerate interval is closed there so that partition of unity holds
    on the whole of [0, 1].
    """
    lo, hi = xi[:-1], xi[1:]
    out = ((lo[None, :] <= x[:, None]) & (x[:, None] < hi[None, :])).astype(np.float64)
    at_end = x >= xi[-1]
    if np.any(at_end):
        last = np.nonzero(hi > lo)[0][-1]
        out[at_end, last] = 1.0
    return out


def basis_by_degree(p, n, x):
    """All B-spline values of degrees 0..p at the points x (Cox-de Boor recursion).

    Section 3.1: N_i^k(x) = (x - xi_i)/(xi_{i+k} - xi_i) N_i^{k-1}(x)
    + (xi_{i+k+1} - x)/(xi_{i+k+1} - xi_{i+1}) N_{i+1}^{k-1}(x), a fraction with
    a zero denominator taken as zero.  Returns a list whose entry k has shape
    [len(x), n + 2p - k].
    """
    xi = knot_vector(p, n)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    levels = [_degree0(xi, x)]
    for k in range(1, p + 1):
        prev = levels[-1]
        cnt = n + 2 * p - k
        cur = np.zeros((x.size, cnt))
        for i in range(cnt):
            d1 = xi[i + k] - xi[i]
            d2 = xi[i + k + 1] - xi[i + 1]
            if d1 > 0:
                cur[:, i] += (x - xi[i]) / d1 * prev[:, i]
            if d2 > 0:
                cur[:, i] += (xi[i + k + 1] - x) / d2 * prev[:, i + 1]
        levels.append(cur)
    return levels


def basis(p, n, x):
    """Values N_i^p(x), i = 1..n+p, shape [len(x), n+p]."""
    return basis_by_degree(p, n, x)[p]


def basis_deriv(p, n, x):
    """Derivatives (N_i^p)'(x), i = 1..n+p, by the differentiation formula of Section 3.1.

    (N_i^p)' = p (N_i^{p-1} / (xi_{i+p} - xi_i) - N_{i+1}^{p-1} / (xi_{i+p+1} - xi_{i+1})),
    a term with a zero denominator taken as zero.
    """
    if p == 0:
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        return np.zeros((x.size, n))
    xi = knot_vector(p, n)
    low = basis_by_degree(p, n, x)[p - 1]  # n + p + 1 functions of degree p-1
    out = np.zeros((low.shape[0], n + p))
    for i in range(n + p):
        d1 = xi[i + p] - xi[i]
        d2 = xi[i + p + 1] - xi[i + 1]
        if d1 > 0:
            out[:, i] += p * low[:, i] / d1
        if d2 > 0:
            out[:, i] -= p * low[:, i + 1] / d2
    return out


def cardinal(p, t, r=0):
    """r-th derivative of the cardinal B-spline phi_p at rational t, exactly.

    Section 3.1: phi_0 = indicator of [0, 1);
    phi_p(t) = t/p phi_{p-1}(t) + (p+1-t)/p phi_{p-1}(t-1);
    phi_p'(t) = phi_{p-1}(t) - phi_{p-1}(t-1).
    Valid for r <= p-1 at every t (and r = p away from the integers).
    """
    t = Fraction(t)
    if r > 0:
        return cardinal(p - 1, t, r - 1) - cardinal(p - 1, t - 1, r - 1)
    if p == 0:
        return Fraction(1) if 0 <= t < 1 else Fraction(0)
    return t / p * cardinal(p - 1, t) + (p + 1 - t) / p * cardinal(p - 1, t - 1)


def cardinal_float(p, t):
    """phi_p at float points (same recursion, vectorised), for plotting-free checks."""
    t = np.asarray(t, dtype=np.float64)
    if p == 0:
        return ((t >= 0) & (t < 1)).astype(np.float64)
    return t / p * cardinal_float(p - 1, t) + (p + 1 - t) / p * cardinal_float(p - 1, t - 1)
