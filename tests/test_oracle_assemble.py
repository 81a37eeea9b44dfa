"""Pins for oracle/assemble.py: the bilinear form assembled by quadrature equals the printed
Kronecker forms (eq:matr_Amu, eq:matr_Amu3D); structure of the curl-div matrix (Section 5);
exact gradient / divergence-free null spaces; manufactured-solution convergence."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import assemble, iga1d, solvers


@pytest.mark.parametrize("d,p,n", [(2, 1, 4), (2, 2, 5), (2, 3, 6), (2, 4, 5), (3, 1, 3), (3, 2, 3), (3, 3, 4)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.1), (0.3, 7.0)])
def test_quadrature_assembly_equals_printed_kronecker_form(d, p, n, alpha, beta):
    Aq = assemble.galerkin_quadrature(d, p, n, alpha, beta)
    Ak = assemble.galerkin_kron(d, p, n, alpha, beta)
    assert Aq.shape == (assemble.dofs(d, p, n),) * 2
    scale = abs(Ak).max()
    assert abs(Aq - Ak).max() <= 1e-14 * scale


@pytest.mark.parametrize("d,p,n", [(2, 2, 6), (2, 4, 5), (3, 2, 4)])
def test_curl_plus_div_is_block_laplacian(d, p, n):
    M, A, S = iga1d.matrices(p, n)
    curl, div = assemble.galerkin_kron(d, p, n, 1.0, 1.0, parts=True)
    K = assemble.scalar_laplacian_kron(d, M, S)
    BK = sp.block_diag([K] * d, format="csr")
    assert abs(curl + div - BK).max() < 1e-13 * abs(BK).max()
    # alpha = beta: A = alpha blockdiag(K) (Section 5.1 / proof of Thm 5.6)
    A2 = assemble.galerkin_kron(d, p, n, 2.5, 2.5)
    assert abs(A2 - 2.5 * BK).max() < 1e-13 * abs(A2).max()
    # symmetric
    A3 = assemble.galerkin_kron(d, p, n, 1.0, 0.01)
    assert abs(A3 - A3.T).max() < 1e-14 * abs(A3).max()


@pytest.mark.parametrize("d,p,n", [(2, 1, 5), (2, 3, 5), (3, 2, 3)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.01), (1.0, 30.0), (4.0, 4.0)])
def test_loewner_bounds_and_definiteness(d, p, n, alpha, beta):
    """min(a,b) K <= A <= max(a,b) K: the matrix form of Theorems 5.2 / 5.6; hence A is SPD."""
    M, A, S = iga1d.matrices(p, n)
    K = assemble.scalar_laplacian_kron(d, M, S).toarray()
    BK = sla.block_diag(*([K] * d))
    Am = assemble.galerkin_kron(d, p, n, alpha, beta).toarray()
    ev = sla.eigh(Am, BK, eigvals_only=True)
    lo, hi = min(alpha, beta), max(alpha, beta)
    assert ev.min() >= lo * (1 - 1e-10) and ev.max() <= hi * (1 + 1e-10)
    np.linalg.cholesky(Am)


def _project(d, p, n, fn):
    """Coefficients of a field that lies in V_h, by L2 projection onto the interior basis."""
    nq = p + 3
    vals, _, w = assemble._eval_ops(d, p, n, nq)
    xs = assemble._grid_points(d, n, nq)
    comps = fn(*xs)
    G = (vals.T @ sp.diags(w) @ vals).toarray()
    out = [np.linalg.solve(G, vals.T @ (w * c)) for c in comps]
    resid = max(np.abs(vals @ o - c).max() for o, c in zip(out, comps))
    return np.concatenate(out), resid


def _bump(x):
    return x ** 2 * (1 - x) ** 2


def _dbump(x):
    return 2 * x * (1 - x) ** 2 - 2 * x ** 2 * (1 - x)


@pytest.mark.parametrize("p", [4, 5])
def test_gradient_and_divergence_free_fields_are_exact_null_vectors_2d(p):
    """phi = x^2(1-x)^2 y^2(1-y)^2: grad phi and curl phi lie in V_h when p >= 4; then
    A^curl grad(phi) = 0 and A^div curl(phi) = 0 (the null spaces as beta or alpha -> 0)."""
    n = 5
    g, r1 = _project(2, p, n, lambda x, y: [_dbump(x) * _bump(y), _bump(x) * _dbump(y)])
    c, r2 = _project(2, p, n, lambda x, y: [_bump(x) * _dbump(y), -_dbump(x) * _bump(y)])
    assert r1 < 1e-12 and r2 < 1e-12
    curl, div = assemble.galerkin_quadrature(2, p, n, 1.0, 1.0, parts=True)
    assert np.linalg.norm(curl @ g) < 1e-12 * np.linalg.norm(div @ g)
    assert np.linalg.norm(div @ c) < 1e-12 * np.linalg.norm(curl @ c)
    A = assemble.galerkin_kron(2, p, n, 1.0, 1e-6)
    # a gradient is a Rayleigh-quotient witness of the beta-scaled eigenvalues
    assert (g @ (A @ g)) / (g @ g) < 1e-4 * sp.linalg.eigsh(A, 1, which="LA", return_eigenvectors=False)[0]


def test_gradient_null_vector_3d():
    p, n = 4, 3
    fn = lambda x, y, z: [_dbump(x) * _bump(y) * _bump(z), _bump(x) * _dbump(y) * _bump(z),  # noqa: E731
                          _bump(x) * _bump(y) * _dbump(z)]
    g, r = _project(3, p, n, fn)
    assert r < 1e-12
    curl, div = assemble.galerkin_quadrature(3, p, n, 1.0, 1.0, parts=True)
    assert np.linalg.norm(curl @ g) < 1e-12 * np.linalg.norm(div @ g)


@pytest.mark.parametrize("d,p,ns", [(2, 1, (8, 16, 32)), (2, 2, (8, 16, 32)), (2, 3, (6, 12, 24)), (3, 2, (4, 8, 12))])
def test_manufactured_solution_converges_at_textbook_rate(d, p, ns):
    """L2 error of the Galerkin solution decays like h^{p+1} for a smooth field (IgA approximation
    theory; the paper states no rate)."""
    field = assemble.manufactured_2d if d == 2 else assemble.manufactured_3d
    errs = []
    for n in ns:
        A = assemble.galerkin_kron(d, p, n, 1.0, 0.1)
        b = assemble.load_vector(d, p, n, 1.0, 0.1, field)
        x = solvers.direct_solve(A, b)
        errs.append(assemble.l2_error(d, p, n, x, field))
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.35, rates


@pytest.mark.parametrize("d,p,n", [(2, 3, 5), (3, 2, 3)])
def test_block_diagonal_cut(d, p, n):
    A = assemble.galerkin_kron(d, p, n, 1.0, 0.2)
    D = assemble.block_diagonal(A, d)
    N = A.shape[0] // d
    Ad = A.toarray()
    for c in range(d):
        sl = slice(c * N, (c + 1) * N)
        np.testing.assert_array_equal(D.toarray()[sl, sl], Ad[sl, sl])
    assert abs(D).sum() < abs(A).sum()


# ---- anisotropic meshes (per-direction interval counts, Section 5)

@pytest.mark.parametrize("d,ns,p", [(2, (5, 9), 2), (2, (8, 3), 3), (3, (3, 5, 4), 2)])
def test_anisotropic_kron_form_equals_bilinear_form(d, ns, p):
    """The printed Kronecker form with the 1D matrices of each direction in their positions equals
    the bilinear form evaluated by quadrature on the anisotropic tensor mesh."""
    alpha, beta = 0.7, 2.5
    Aq = assemble.galerkin_quadrature(d, p, ns, alpha, beta)
    Ak = assemble.galerkin_kron(d, p, ns, alpha, beta)
    assert Aq.shape[0] == assemble.dofs(d, p, ns)
    assert abs(Aq - Ak).max() <= 1e-13 * abs(Aq).max()


def test_anisotropic_axis_swap():
    """Swapping x_1 and x_2 (and the two components) maps the bilinear form on an (n_1, n_2)
    mesh onto the one on (n_2, n_1): curl changes sign, div is unchanged."""
    p, n1, n2 = 3, 6, 10
    A12 = assemble.galerkin_kron(2, p, (n1, n2), 1.3, 0.4).toarray()
    A21 = assemble.galerkin_kron(2, p, (n2, n1), 1.3, 0.4).toarray()
    m1, m2 = n1 + p - 2, n2 + p - 2
    N = m1 * m2
    perm = np.empty(2 * N, dtype=int)  # new index (c', j, i) <- old (c, i, j), c' = 1 - c
    for c in range(2):
        for i in range(m1):
            for j in range(m2):
                perm[(1 - c) * N + j * m1 + i] = c * N + i * m2 + j
    np.testing.assert_allclose(A12[np.ix_(perm, perm)], A21, rtol=0, atol=1e-14 * np.abs(A12).max())


def test_anisotropic_uniform_tuple_and_loewner_bounds():
    """(n, n) gives the isotropic matrix; on an anisotropic mesh A^curl + A^div = blockdiag(K)
    and min(alpha,beta) K <= A <= max(alpha,beta) K still hold (matrix form of Thm 5.2)."""
    p = 2
    np.testing.assert_array_equal(assemble.galerkin_kron(2, p, (7, 7), 1.0, 0.3).toarray(),
                                  assemble.galerkin_kron(2, p, 7, 1.0, 0.3).toarray())
    ns, alpha, beta = (4, 9), 1.0, 0.05
    curl, div = assemble.galerkin_kron(2, p, ns, 1.0, 1.0, parts=True)
    K = (curl + div).toarray()
    N = K.shape[0] // 2
    assert np.abs(K[:N, N:]).max() <= 1e-14 * np.abs(K).max()
    A = assemble.galerkin_kron(2, p, ns, alpha, beta).toarray()
    import scipy.linalg as sla
    ev = sla.eigh(A, K, eigvals_only=True)
    assert ev.min() >= beta * (1 - 1e-10) and ev.max() <= alpha * (1 + 1e-10)
