"""Spectral symbols (Theorem 3.1, Lemma 3.2, Theorems 5.1 and 5.5, eq:lapl2D, eq:lapl3D).

Test infrastructure only (see ``oracle/__init__.py``).  All symbols are for
nu = (1, ..., 1) (equal n in every direction), so gamma_i = delta_i = 1.
"""
import numpy as np

from . import bspline


def _coeffs(p, r):
    """phi^{(r)}_{2p+1}(p+1-k), k = 0..p, as floats."""
    return [float(bspline.cardinal(2 * p + 1, p + 1 - k, r)) for k in range(p + 1)]


def m_sym(p, theta):
    """m_p(theta) = phi_{2p+1}(p+1) + 2 sum_k phi_{2p+1}(p+1-k) cos(k theta) (Thm 3.1a)."""
    c = _coeffs(p, 0)
    theta = np.asarray(theta, dtype=np.float64)
    return c[0] + 2 * sum(c[k] * np.cos(k * theta) for k in range(1, p + 1))


def a_sym(p, theta):
    """a_p(theta) = -2 sum_k phi'_{2p+1}(p+1-k) sin(k theta) (Thm 3.1b)."""
    c = _coeffs(p, 1)
    theta = np.asarray(theta, dtype=np.float64)
    return -2 * sum(c[k] * np.sin(k * theta) for k in range(1, p + 1))


def s_sym(p, theta):
    """s_p(theta) = -phi''_{2p+1}(p+1) - 2 sum_k phi''_{2p+1}(p+1-k) cos(k theta) (Thm 3.1c)."""
    c = _coeffs(p, 2)
    theta = np.asarray(theta, dtype=np.float64)
    return -c[0] - 2 * sum(c[k] * np.cos(k * theta) for k in range(1, p + 1))


def symbol_2d(p, alpha, beta, t1, t2):
    """The 2x2 symbol f^{p,alpha,beta}(t1, t2) of eq:f2D, shape [..., 2, 2]."""
    m1, m2 = m_sym(p, t1), m_sym(p, t2)
    s1, s2 = s_sym(p, t1), s_sym(p, t2)
    a1, a2 = a_sym(p, t1), a_sym(p, t2)
    f11 = alpha * m1 * s2 + beta * s1 * m2
    f22 = alpha * s1 * m2 + beta * m1 * s2
    f12 = -(alpha - beta) * a1 * a2
    return np.stack([np.stack([f11, f12], -1), np.stack([f12, f22], -1)], -2)


def eig_2d_closed(p, alpha, beta, t1, t2):
    """lambda_1 <= lambda_2 of the 2D symbol by eq:expres:eig:1 / eq:expres:eig:2."""
    m1, m2 = m_sym(p, t1), m_sym(p, t2)
    s1, s2 = s_sym(p, t1), s_sym(p, t2)
    a1, a2 = a_sym(p, t1), a_sym(p, t2)
    lp = m1 * s2 + s1 * m2
    lm = m1 * s2 - s1 * m2
    root = np.abs(alpha - beta) * np.sqrt(lm ** 2 + 4 * a1 ** 2 * a2 ** 2)
    return 0.5 * ((alpha + beta) * lp - root), 0.5 * ((alpha + beta) * lp + root)


def symbol_3d(p, alpha, beta, t1, t2, t3):
    """The 3x3 symbol of eq:f3D with gamma_i = delta_i = 1, shape [..., 3, 3]."""
    m = [m_sym(p, t) for t in (t1, t2, t3)]
    s = [s_sym(p, t) for t in (t1, t2, t3)]
    a = [a_sym(p, t) for t in (t1, t2, t3)]
    smm, msm, mms = s[0] * m[1] * m[2], m[0] * s[1] * m[2], m[0] * m[1] * s[2]
    f11 = beta * smm + alpha * msm + alpha * mms
    f22 = alpha * smm + beta * msm + alpha * mms
    f33 = alpha * smm + alpha * msm + beta * mms
    f12 = -(alpha - beta) * a[0] * a[1] * m[2]
    f13 = -(alpha - beta) * a[0] * m[1] * a[2]
    f23 = -(alpha - beta) * m[0] * a[1] * a[2]
    rows = [np.stack([f11, f12, f13], -1), np.stack([f12, f22, f23], -1), np.stack([f13, f23, f33], -1)]
    return np.stack(rows, -2)


def laplacian_sym(p, *thetas):
    """Scalar IgA Laplacian symbol: eq:lapl2D for two angles, eq:lapl3D for three."""
    d = len(thetas)
    m = [m_sym(p, t) for t in thetas]
    s = [s_sym(p, t) for t in thetas]
    out = 0.0
    for l in range(d):
        term = 1.0
        for k in range(d):
            term = term * (s[k] if k == l else m[k])
        out = out + term
    return out


def grid(m, d):
    """The grid Gamma of Section 5.3: theta_k = k pi / m, k = 1..m in each direction."""
    t = np.arange(1, m + 1) * np.pi / m
    return np.meshgrid(*([t] * d), indexing="ij")


def sampled_eigs(d, p, alpha, beta, m):
    """Lambda_1..Lambda_d of Section 5.3: eigenvalues of the symbol at every point of Gamma.

    Returns an array [m^d, d], each row ascending (Lambda_i is column i).
    """
    g = grid(m, d)
    f = symbol_2d(p, alpha, beta, *g) if d == 2 else symbol_3d(p, alpha, beta, *g)
    return np.linalg.eigvalsh(f.reshape(-1, d, d))
