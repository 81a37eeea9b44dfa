"""Solvers of Section 6: CG, Gauss-Seidel, the Galerkin V-cycle, Krylov smoothers with T,
and the strategies MIM, P_MIM, P_WL (Section 6.2).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of points the paper leaves open (each is listed in the design notes):
* Stopping rule (Section 6.2): ||r_k|| / ||r_0|| < tol from x_0 = 0.
* Gauss-Seidel: "one Gauss-Seidel iteration" is one symmetric sweep, a
  forward lexicographic sweep over the component-major ordering followed by a
  backward one, on the assembled (Galerkin) matrix of the level.  With this
  reading the stand-alone MIM reproduces the MIM columns of Tables 1-4 to +-2
  iterations; a forward sweep alone needs 20-50% more iterations.
* P_MIM: the paper does not say how many MIM iterations one application of the
  preconditioner performs (for P_WL it says one).  Two V-cycles from zero
  reproduce the P_MIM columns of Tables 1-4 to +-1-2; one gives about 1.5x the
  printed counts.
* Level sizes: coarse size floor(m/2); coarse column J of the 1D prolongator
  holds 1/2, 1, 1/2 on fine rows 2J-1, 2J, 2J+1 (eq:projector-1d), rows past
  m dropped.  Coarsening stops at m <= ``m_min`` (default 1, i.e. the
  log2(n+p-1) levels of Section 6.2 when n+p-1 is a power of two); the
  coarsest system is solved directly.
* Krylov smoothers: ``steps`` iterations from the current iterate, PGMRES
  right-preconditioned without restart, PCG with the standard recurrence.
* A Krylov-smoothed V-cycle is not a fixed linear operator, so the outer CG of
  P_MIM and P_WL uses the flexible (Polak-Ribiere) update
  beta_k = r_{k+1}^T (z_{k+1} - z_k) / r_k^T z_k; ``flexible=False`` gives the
  textbook PCG update.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import iga1d


# ------------------------------------------------------------------ direct

def direct_solve(A, b):
    """w* = A^{-1} b by sparse LU (SuperLU) in FP64."""
    return spla.spsolve(sp.csc_matrix(A), b)


# ------------------------------------------------------------------ CG family

def cg(A, b, tol=1e-7, maxit=100000, precond=None, flexible=False, x0=None):
    """(Preconditioned) conjugate gradients; returns (x, iterations, relative residual history).

    Iteration k is counted when ||r_k||/||r_0|| < tol first holds (Section 6.2).
    """
    matvec = A if callable(A) else (lambda v: A @ v)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - matvec(x) if x0 is not None else b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = precond(r) if precond else r
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = matvec(p)
        a = rz / (p @ q)
        x = x + a * p
        r_new = r - a * q
        rel = np.linalg.norm(r_new) / r0
        hist.append(rel)
        if rel < tol:
            return x, k, hist
        z_new = precond(r_new) if precond else r_new
        rz_new = r_new @ z_new
        if flexible:
            beta = (r_new @ (z_new - z)) / rz
        else:
            beta = rz_new / rz
        p = z_new + beta * p
        r, z, rz = r_new, z_new, rz_new
    return x, maxit, hist


# ------------------------------------------------------------------ smoothers

def gauss_seidel(A, x, b, symmetric=True):
    """One Gauss-Seidel iteration (Section 6.1): the forward sweep (D + L) x' = b - U x,
    then (``symmetric``) the backward sweep (D + U) x'' = b - L x'."""
    A = sp.csr_matrix(A)
    lower = sp.tril(A, 0, format="csr")
    upper = sp.triu(A, 1, format="csr")
    x = spla.spsolve_triangular(lower, b - upper @ x, lower=True)
    if symmetric:
        strict_lower = sp.tril(A, -1, format="csr")
        upper_d = sp.triu(A, 0, format="csr")
        x = spla.spsolve_triangular(upper_d, b - strict_lower @ x, lower=False)
    return x


class TSolver:
    """Solve with T = I_d (x) T_m(m_{p-1}) (x) ... (eq:kron_precond), one LU per 1D factor.

    Section 6.1: (T_m(g_p))^{-1} is the Kronecker product of the inverses of the 1D
    banded factors, each applied through its LU factorisation.
    """

    def __init__(self, d, p, m):
        self.d, self.m = d, m
        self.lu = sla.lu_factor(iga1d.toeplitz_T(p, m))

    def __call__(self, r):
        d, m = self.d, self.m
        t = r.reshape([d] + [m] * d).copy()
        for ax in range(1, d + 1):
            t = np.moveaxis(t, ax, 0)
            sh = t.shape
            t = sla.lu_solve(self.lu, t.reshape(m, -1)).reshape(sh)
            t = np.moveaxis(t, 0, ax)
        return t.ravel()


def pcg_steps(A, b, x, steps, precond):
    """``steps`` PCG iterations on A x = b from the current iterate (post-smoother of Section 6.1)."""
    r = b - A @ x
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for _ in range(steps):
        if rz == 0.0:
            break
        q = A @ p
        a = rz / (p @ q)
        x = x + a * p
        r = r - a * q
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def pgmres_steps(A, b, x, steps, precond):
    """``steps`` iterations of right-preconditioned GMRES from the current iterate, no restart.

    Minimises ||b - A(x + T^{-1} V y)|| over the Krylov space of A T^{-1} (Section 6.1).
    """
    r = b - A @ x
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x
    n = b.size
    V = np.zeros((n, steps + 1))
    H = np.zeros((steps + 1, steps))
    Z = np.zeros((n, steps))
    V[:, 0] = r / beta
    k_used = steps
    for j in range(steps):
        Z[:, j] = precond(V[:, j])
        w = A @ Z[:, j]
        for i in range(j + 1):  # modified Gram-Schmidt
            H[i, j] = w @ V[:, i]
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-300:
            k_used = j + 1
            break
        V[:, j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k_used + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H[:k_used + 1, :k_used], e1, rcond=None)
    return x + Z[:, :k_used] @ y


# ------------------------------------------------------------------ multigrid

def prolongator_1d(m):
    """P of eq:projector-1d, m x floor(m/2): column J has 1/2, 1, 1/2 on rows 2J-1, 2J, 2J+1."""
    mc = m // 2
    rows, cols, vals = [], [], []
    for j in range(mc):
        for off, v in ((0, 0.5), (1, 1.0), (2, 0.5)):
            i = 2 * j + off
            if i < m:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, mc))


def block_prolongator(d, m):
    """I_d (x) P (x) ... (x) P of eq:2by2prol."""
    P1 = prolongator_1d(m)
    out = sp.identity(d, format="csr")
    for _ in range(d):
        out = sp.kron(out, P1, format="csr")
    return out.tocsr()


class Hierarchy:
    """Galerkin hierarchy A_{l+1} = P_l^T A_l P_l with R_l = P_l^T (Section 6.1)."""

    def __init__(self, A, d, m, m_min=1):
        self.d = d
        self.A = [sp.csr_matrix(A)]
        self.P = []
        self.m = [m]
        while m > m_min and m // 2 >= 1:
            P = block_prolongator(d, m)
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            m = m // 2
            self.m.append(m)
        self.coarse_lu = spla.splu(sp.csc_matrix(self.A[-1]))

    @property
    def levels(self):
        """Number of levels, the finest included."""
        return len(self.A)


def vcycle(H, b, x, fine_post, level=0):
    """One V-cycle (Section 6.1): 1 GS pre-smoothing step, coarse-grid correction,
    post-smoothing by ``fine_post(A, b, x)`` on level 0 and one GS step elsewhere."""
    A = H.A[level]
    if level == H.levels - 1:
        return H.coarse_lu.solve(b)
    x = gauss_seidel(A, x, b)
    r = b - A @ x
    e = vcycle(H, H.P[level].T @ r, np.zeros(H.P[level].shape[1]), fine_post, level + 1)
    x = x + H.P[level] @ e
    if level == 0:
        x = fine_post(A, b, x)
    else:
        x = gauss_seidel(A, x, b)
    return x


def make_post(kind, d, p, m):
    """p post-smoothing steps of PCG or PGMRES preconditioned by T (Section 6.2)."""
    T = TSolver(d, p, m)
    if kind == "pcg":
        return lambda A, b, x: pcg_steps(A, b, x, p, T)
    if kind == "pgmres":
        return lambda A, b, x: pgmres_steps(A, b, x, p, T)
    raise ValueError(kind)


def mim(A, b, d, p, m, tol=1e-7, maxit=1000, m_min=1):
    """MIM: the V-cycle with PGMRES-T post-smoothing used as a stand-alone iteration."""
    H = Hierarchy(A, d, m, m_min)
    post = make_post("pgmres", d, p, m)
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    for k in range(1, maxit + 1):
        x = vcycle(H, b, x, post)
        if np.linalg.norm(b - A @ x) / nb < tol:
            return x, k
    return x, maxit


def mim_preconditioner(A, d, p, m, cycles=2, m_min=1):
    """z = B(r): ``cycles`` MIM iterations (V-cycles with PGMRES-T post-smoothing) on
    A z = r from z = 0, the preconditioner of P_MIM (Section 6.2)."""
    H = Hierarchy(A, d, m, m_min)
    post = make_post("pgmres", d, p, m)

    def prec(r):
        z = np.zeros_like(r)
        for _ in range(cycles):
            z = vcycle(H, r, z, post)
        return z
    return prec


def p_mim(A, b, d, p, m, tol=1e-7, maxit=1000, m_min=1, flexible=True, cycles=2):
    """P_MIM: MIM iterations from zero (``cycles`` of them) as the preconditioner of CG."""
    prec = mim_preconditioner(A, d, p, m, cycles, m_min)
    x, k, _ = cg(A, b, tol, maxit, prec, flexible)
    return x, k


def p_wl(A, b, d, p, m, tol=1e-7, maxit=1000, m_min=1, flexible=True):
    """P_WL: one V-cycle (PCG-T post-smoothing) on the block diagonal D of eq:diag as CG preconditioner."""
    from .assemble import block_diagonal
    D = block_diagonal(A, d)
    H = Hierarchy(D, d, m, m_min)
    post = make_post("pcg", d, p, m)
    prec = lambda r: vcycle(H, r, np.zeros_like(r), post)  # noqa: E731
    x, k, _ = cg(A, b, tol, maxit, prec, flexible)
    return x, k


# ------------------------------------------------------------------ exact block inverses

def solve_D(A, d, r):
    """D^{-1} r with D = blockdiag(A^(1,1), ..., A^(d,d)) (eq:diag), by sparse LU."""
    from .assemble import block_diagonal
    return direct_solve(block_diagonal(A, d), r)


def generalized_eigs(M, S):
    """Eigenpairs of S u = lambda M u with U^T M U = I (dense LAPACK), ascending."""
    return sla.eigh(S, M)
