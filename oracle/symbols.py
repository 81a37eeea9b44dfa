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


def symbol_2d(p, alpha, beta, t1, t2, nu=(1.0, 1.0)):
    """The 2x2 symbol f^{p,alpha,beta}(t1, t2) of eq:f2D (Theorem 5.1, n_l = n nu_l), shape
    [..., 2, 2]: the M (x) S terms carry nu_2 / nu_1, the S (x) M terms nu_1 / nu_2."""
    m1, m2 = m_sym(p, t1), m_sym(p, t2)
    s1, s2 = s_sym(p, t1), s_sym(p, t2)
    a1, a2 = a_sym(p, t1), a_sym(p, t2)
    r21, r12 = nu[1] / nu[0], nu[0] / nu[1]
    f11 = alpha * r21 * m1 * s2 + beta * r12 * s1 * m2
    f22 = alpha * r12 * s1 * m2 + beta * r21 * m1 * s2
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


def symbol_3d(p, alpha, beta, t1, t2, t3, nu=(1.0, 1.0, 1.0)):
    """The 3x3 symbol of eq:f3D (Theorem 5.5, n_l = n nu_l), shape [..., 3, 3], with
    gamma_i = nu_i^2 / (nu_1 nu_2 nu_3) weighting the terms whose S acts along x_i and
    delta_i = 1 / nu_i the coupling term whose M acts along x_i."""
    m = [m_sym(p, t) for t in (t1, t2, t3)]
    s = [s_sym(p, t) for t in (t1, t2, t3)]
    a = [a_sym(p, t) for t in (t1, t2, t3)]
    vol = nu[0] * nu[1] * nu[2]
    g = [nu[i] ** 2 / vol for i in range(3)]
    dl = [1.0 / nu[i] for i in range(3)]
    smm, msm, mms = g[0] * s[0] * m[1] * m[2], g[1] * m[0] * s[1] * m[2], g[2] * m[0] * m[1] * s[2]
    f11 = beta * smm + alpha * msm + alpha * mms
    f22 = alpha * smm + beta * msm + alpha * mms
    f33 = alpha * smm + alpha * msm + beta * mms
    f12 = -(alpha - beta) * dl[2] * a[0] * a[1] * m[2]
    f13 = -(alpha - beta) * dl[1] * a[0] * m[1] * a[2]
    f23 = -(alpha - beta) * dl[0] * m[0] * a[1] * a[2]
    rows = [np.stack([f11, f12, f13], -1), np.stack([f12, f22, f23], -1), np.stack([f13, f23, f33], -1)]
    return np.stack(rows, -2)


def laplacian_sym(p, *thetas, nu=None):
    """Scalar IgA Laplacian symbol: eq:lapl2D for two angles, eq:lapl3D for three; with nu the
    weighted forms of Sections 5.1 / 5.2 (2D: nu_2/nu_1 m s + nu_1/nu_2 s m; 3D: gamma_l)."""
    d = len(thetas)
    nu = (1.0,) * d if nu is None else tuple(nu)
    m = [m_sym(p, t) for t in thetas]
    s = [s_sym(p, t) for t in thetas]
    vol = float(np.prod(nu))
    out = 0.0
    for l in range(d):
        # weight of the term with S along x_l: nu_l^2 / prod(nu) (2D: nu_l / nu_other)
        term = nu[l] ** 2 / vol
        for k in range(d):
            term = term * (s[k] if k == l else m[k])
        out = out + term
    return out


def grid(m, d):
    """The grid Gamma of Section 5.3: theta_k = k pi / m_l, k = 1..m_l in direction l (m may be
    one size for every direction or one per direction)."""
    ms = (m,) * d if np.isscalar(m) else tuple(m)
    ts = [np.arange(1, ml + 1) * np.pi / ml for ml in ms]
    return np.meshgrid(*ts, indexing="ij")


def sampled_eigs(d, p, alpha, beta, m, nu=None):
    """Lambda_1..Lambda_d of Section 5.3: eigenvalues of the symbol at every point of Gamma.

    Returns an array [prod m_l, d], each row ascending (Lambda_i is column i).  ``nu`` selects
    the weighted symbol of an anisotropic mesh (its grid then has m_l = n_l + p - 2 points in
    direction l).
    """
    g = grid(m, d)
    nu = (1.0,) * d if nu is None else tuple(nu)
    f = symbol_2d(p, alpha, beta, *g, nu=nu) if d == 2 else symbol_3d(p, alpha, beta, *g, nu=nu)
    return np.linalg.eigvalsh(f.reshape(-1, d, d))
