"""The d-D curl-div Galerkin matrix and load vectors (Section 4, Section 6.2).

Test infrastructure only (see ``oracle/__init__.py``).

Unknown ordering (Section 4, eq:eq_1): component-major, w = [u^1; ...; u^d];
inside a component the Kronecker order of the tensor-product index
(i_1, ..., i_d), x_1 slowest and x_d fastest.  DoF count d * m^d with
m = n + p - 2.

``n`` is the number of intervals per direction, or a tuple (n_1, ..., n_d) of
per-direction counts: the anisotropic meshes n_l = nu_l n of Section 5 (the
spline space is then the tensor product of the 1D spaces of each direction,
and m_l = n_l + p - 2 unknowns per direction per component).

Two independent routes to the same matrix:

* ``galerkin_quadrature`` evaluates curl and div of every vector basis
  function psi^{p,c}_i = N_i e_c at the Gauss points of every element and
  forms alpha (curl psi_i, curl psi_j) + beta (div psi_i, div psi_j) directly
  from the bilinear form eq:curl-div.  Nothing about M, A, S or Kronecker
  products of matrices enters; the tensor-product basis is only evaluated
  (N_i(x) = prod_l N_{i_l}(x_l), the definition in Section 3.1).
* ``galerkin_kron`` writes out eq:matr_Amu (d = 2) and eq:matr_Amu3D (d = 3)
  term by term, with the transposes exactly as printed.
"""
import numpy as np
import scipy.sparse as sp

from . import iga1d


def axis_counts(d, n):
    """Per-direction interval counts: (n,) * d for an integer n, else the given tuple."""
    if np.isscalar(n):
        return (int(n),) * d
    ns = tuple(int(v) for v in n)
    if len(ns) != d:
        raise ValueError("one interval count per direction")
    return ns


def dofs(d, p, n):
    """Matrix size d * prod_l (n_l+p-2) (Section 5.1; d (n+p-2)^d on a uniform mesh)."""
    return d * int(np.prod([v + p - 2 for v in axis_counts(d, n)]))


def _kron_all(mats):
    out = mats[0]
    for mt in mats[1:]:
        out = sp.kron(out, mt, format="csr")
    return sp.csr_matrix(out)


def _eval_ops(d, p, n, nq, rows0=None):
    """Sparse evaluation operators at the tensor Gauss grid.

    Returns (vals, dx, w): vals [Q, m^d] maps coefficients of one component to
    point values; dx[l] [Q, m^d] maps them to d/dx_l at the points; w [Q] are the
    quadrature weights.  ``rows0`` restricts the x_1 points to a slice (the
    operators then cover only those points, in the same order).
    """
    ns = axis_counts(d, n)
    vs, gs, ws = [], [], []
    for l in range(d):  # the 1D Gauss grid and basis of direction l
        x, wl = iga1d.gauss_points(ns[l], nq)
        v, g = iga1d.eval_interior(p, ns[l], x)
        vs.append(sp.csr_matrix(v))
        gs.append(sp.csr_matrix(g))
        ws.append(wl)
    sl = slice(None) if rows0 is None else rows0
    vs[0], gs[0], ws[0] = vs[0][sl], gs[0][sl], ws[0][sl]
    vals = _kron_all(vs)
    dx = []
    for l in range(d):
        dx.append(_kron_all([gs[k] if k == l else vs[k] for k in range(d)]))
    w = ws[0]
    for l in range(1, d):
        w = np.kron(w, ws[l])
    return vals, dx, w


def curl_div_operators(d, p, n, nq=None, rows0=None):
    """Point-evaluation operators of curl and div over the vector basis.

    curl: d=2 gives the scalar curl u = d1 u2 - d2 u1;
          d=3 gives (d2 u3 - d3 u2, d3 u1 - d1 u3, d1 u2 - d2 u1) stacked.
    div:  d1 u1 + ... + dd ud.
    Returns (Ccurl, Cdiv, W) with W the quadrature weights repeated per curl row block.
    """
    nq = nq or p + 1
    vals, dx, w = _eval_ops(d, p, n, nq, rows0)
    if d == 2:
        Ccurl = sp.hstack([-dx[1], dx[0]], format="csr")
        wc = w
    elif d == 3:
        Ccurl = sp.bmat([
            [None, -dx[2], dx[1]],
            [dx[2], None, -dx[0]],
            [-dx[1], dx[0], None],
        ], format="csr")
        wc = np.concatenate([w, w, w])
    else:
        raise ValueError("d must be 2 or 3")
    Cdiv = sp.hstack(dx, format="csr")
    return Ccurl, Cdiv, wc, w


def galerkin_quadrature(d, p, n, alpha, beta, nq=None, parts=False):
    """alpha (curl u, curl v) + beta (div u, div v) on V_h, by Gauss quadrature (eq:curl-div).

    With ``parts=True`` returns (A_curl, A_div) separately (alpha = beta = 1 weights).
    """
    Ccurl, Cdiv, wc, w = curl_div_operators(d, p, n, nq)
    Acurl = (Ccurl.T @ sp.diags(wc) @ Ccurl).tocsr()
    Adiv = (Cdiv.T @ sp.diags(w) @ Cdiv).tocsr()
    if parts:
        return Acurl, Adiv
    return (alpha * Acurl + beta * Adiv).tocsr()


def galerkin_kron(d, p, n, alpha, beta, mats=None, parts=False):
    """eq:matr_Amu (d=2) / eq:matr_Amu3D (d=3), written term by term as printed.

    Each Kronecker factor in position l is the 1D matrix of direction l (the same matrix in
    every position on a uniform mesh; ``mats`` overrides it there).
    """
    ns = axis_counts(d, n)
    if mats is not None:
        per = [tuple(sp.csr_matrix(x) for x in mats)] * d
    else:
        per = [tuple(sp.csr_matrix(x) for x in iga1d.matrices(p, ns[l])) for l in range(d)]

    def K(*letters):
        """The Kronecker product of the named 1D matrices, letter l acting along x_{l+1}."""
        fs = []
        for l, c in enumerate(letters):
            M, A, S = per[l]
            fs.append({"M": M, "A": A, "T": A.T.tocsr(), "S": S}[c])
        return _kron_all(fs)
    # letters: M, S, A, and T for A^T, in the order of the printed factors
    if d == 2:
        curl = sp.bmat([[K("M", "S"), -K("T", "A")],
                        [-K("A", "T"), K("S", "M")]], format="csr")
        div = sp.bmat([[K("S", "M"), K("A", "T")],
                       [K("T", "A"), K("M", "S")]], format="csr")
    elif d == 3:
        curl = sp.bmat([
            [K("M", "M", "S") + K("M", "S", "M"), -K("T", "A", "M"), -K("T", "M", "A")],
            [-K("A", "T", "M"), K("S", "M", "M") + K("M", "M", "S"), -K("M", "T", "A")],
            [-K("A", "M", "T"), -K("M", "A", "T"), K("S", "M", "M") + K("M", "S", "M")],
        ], format="csr")
        div = sp.bmat([
            [K("S", "M", "M"), K("A", "T", "M"), K("A", "M", "T")],
            [K("T", "A", "M"), K("M", "S", "M"), K("M", "A", "T")],
            [K("T", "M", "A"), K("M", "T", "A"), K("M", "M", "S")],
        ], format="csr")
    else:
        raise ValueError("d must be 2 or 3")
    if parts:
        return curl, div
    return (alpha * curl + beta * div).tocsr()


def scalar_laplacian_kron(d, M, S):
    """The scalar IgA Laplacian: M(x)S + S(x)M in 2D, S(x)M(x)M + M(x)S(x)M + M(x)M(x)S in 3D."""
    M, S = sp.csr_matrix(M), sp.csr_matrix(S)
    terms = []
    for l in range(d):
        terms.append(_kron_all([S if k == l else M for k in range(d)]))
    out = terms[0]
    for t in terms[1:]:
        out = out + t
    return out.tocsr()


def block_diagonal(A, d):
    """D = blockdiag(A^(1,1), ..., A^(d,d)) of eq:diag, cut out of a sparse A."""
    N = A.shape[0] // d
    A = A.tocsr()
    blocks = [A[c * N:(c + 1) * N, c * N:(c + 1) * N] for c in range(d)]
    return sp.block_diag(blocks, format="csr")


# ---------------------------------------------------------------- load vectors

def manufactured_2d(x1, x2):
    """The 2D test field of Section 6.2 with its first derivatives.

    u1 = sin(2 pi q), u2 = cos(2 pi q) - 1, q = x1(1-x1) x2(1-x2).
    Returns (u, du) with u[c] and du[c][l] = d u_c / d x_l.
    """
    q = x1 * (1 - x1) * x2 * (1 - x2)
    dq = [(1 - 2 * x1) * x2 * (1 - x2), x1 * (1 - x1) * (1 - 2 * x2)]
    s, c = np.sin(2 * np.pi * q), np.cos(2 * np.pi * q)
    u = [s, c - 1.0]
    du = [[2 * np.pi * c * dq[l] for l in range(2)], [-2 * np.pi * s * dq[l] for l in range(2)]]
    return u, du


def manufactured_3d(x1, x2, x3):
    """The 3D test field of Section 6.2: u1 = sin(2 pi q), u2 = cos(2 pi q) - 1, u3 = u1 + u2,
    q = x1(1-x1) x2(1-x2) x3(1-x3)."""
    g = [x1 * (1 - x1), x2 * (1 - x2), x3 * (1 - x3)]
    dg = [1 - 2 * x1, 1 - 2 * x2, 1 - 2 * x3]
    q = g[0] * g[1] * g[2]
    dq = [dg[0] * g[1] * g[2], g[0] * dg[1] * g[2], g[0] * g[1] * dg[2]]
    s, c = np.sin(2 * np.pi * q), np.cos(2 * np.pi * q)
    u1, u2 = s, c - 1.0
    du1 = [2 * np.pi * c * dq[l] for l in range(3)]
    du2 = [-2 * np.pi * s * dq[l] for l in range(3)]
    du3 = [du1[l] + du2[l] for l in range(3)]
    return [u1, u2, u1 + u2], [du1, du2, du3]


def sine_field(ks):
    """u_c = prod_l sin(k_{c,l} pi x_l) (a smooth field vanishing on the boundary), ks [d][d] ints."""
    ks = np.asarray(ks)
    d = ks.shape[0]

    def field(*xs):
        """(u, du): the d components at the points xs and their first derivatives du[c][l]."""
        u, du = [], []
        for c in range(d):
            f = [np.sin(ks[c, l] * np.pi * xs[l]) for l in range(d)]
            fp = [ks[c, l] * np.pi * np.cos(ks[c, l] * np.pi * xs[l]) for l in range(d)]
            prod = np.ones_like(xs[0])
            for l in range(d):
                prod = prod * f[l]
            u.append(prod)
            dl = []
            for l in range(d):
                t = np.ones_like(xs[0])
                for k in range(d):
                    t = t * (fp[k] if k == l else f[k])
                dl.append(t)
            du.append(dl)
        return u, du
    return field


def _grid_points(d, n, nq, rows0=None):
    ns = axis_counts(d, n)
    xs = [iga1d.gauss_points(ns[l], nq)[0] for l in range(d)]
    if rows0 is not None:
        xs[0] = xs[0][rows0]
    grids = np.meshgrid(*xs, indexing="ij")
    return [g.ravel() for g in grids]


def _chunks(d, n, nq, budget=1_500_000):
    """Slices of the x_1 Gauss points so that each chunk holds about ``budget`` points."""
    ns = axis_counts(d, n)
    Q = ns[0] * nq
    rest = int(np.prod([v * nq for v in ns[1:]]))
    step = max(1, budget // rest)
    return [slice(s, min(Q, s + step)) for s in range(0, Q, step)]


def load_vector(d, p, n, alpha, beta, field, nq=None):
    """b_i = alpha (curl u, curl psi_i) + beta (div u, div psi_i) for an analytic u.

    For psi_i vanishing on the boundary this equals (L_{alpha,beta} u, psi_i) of
    eq:alfven-op after integrating by parts once, so only first derivatives of
    u are needed.  ``field(*xs) -> (u, du)``; nq defaults to p + 6 points per
    interval because the integrand is not polynomial.
    """
    nq = nq or p + 6
    b = 0.0
    for rows0 in _chunks(d, n, nq):
        Ccurl, Cdiv, wc, w = curl_div_operators(d, p, n, nq, rows0)
        xs = _grid_points(d, n, nq, rows0)
        _, du = field(*xs)
        if d == 2:
            curl_u = du[1][0] - du[0][1]
        else:
            curl_u = np.concatenate([du[2][1] - du[1][2], du[0][2] - du[2][0], du[1][0] - du[0][1]])
        div_u = sum(du[c][c] for c in range(d))
        b = b + alpha * (Ccurl.T @ (wc * curl_u)) + beta * (Cdiv.T @ (w * div_u))
    return b


def l2_error(d, p, n, coeffs, field, nq=None):
    """|| u - u_h ||_{L^2(Omega)} for u_h with coefficients ``coeffs`` (component-major)."""
    nq = nq or p + 6
    err2 = 0.0
    for rows0 in _chunks(d, n, nq):
        vals, _, w = _eval_ops(d, p, n, nq, rows0)
        xs = _grid_points(d, n, nq, rows0)
        u, _ = field(*xs)
        N = vals.shape[1]
        for c in range(d):
            uh = vals @ coeffs[c * N:(c + 1) * N]
            err2 += float(np.sum(w * (u[c] - uh) ** 2))
    return np.sqrt(err2)
