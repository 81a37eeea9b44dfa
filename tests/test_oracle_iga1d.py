"""Pins for oracle/iga1d.py: exact central entries (Section 3.2), the p = 1 finite-element
closed forms, structure (symmetry, skew-symmetry, definiteness) and the matrix T of Section 6.1."""
import numpy as np
import pytest

from oracle import iga1d, symbols


@pytest.mark.parametrize("p,n", [(1, 8), (2, 12), (3, 14), (4, 17), (5, 19)])
def test_central_entries_are_cardinal_values(p, n):
    M, A, S = iga1d.matrices(p, n)
    assert M.shape == (n + p - 2, n + p - 2)
    for i in range(2 * p, n - p):  # 1-based rows 2p..n-p-1
        for j in range(max(1, i - p - 1), min(n + p - 2, i + p + 1) + 1):
            if not (2 * p <= j <= n - p - 1):
                continue
            for X, w in ((M, "M"), (A, "A"), (S, "S")):
                exact = float(iga1d.interior_entry_exact(p, n, i, j, w))
                assert abs(X[i - 1, j - 1] - exact) <= 1e-14 * max(1, n), (w, i, j)


def test_p1_finite_element_closed_forms():
    n = 9
    M, A, S = iga1d.matrices(1, n)
    m = n - 1
    I = np.eye(m)
    Sup = np.eye(m, k=1)
    Sdn = np.eye(m, k=-1)
    np.testing.assert_allclose(M, (4 * I + Sup + Sdn) / (6 * n), atol=1e-15)
    np.testing.assert_allclose(S, n * (2 * I - Sup - Sdn), atol=1e-12)
    np.testing.assert_allclose(A, 0.5 * (Sup - Sdn), atol=1e-15)


@pytest.mark.parametrize("p,n", [(1, 5), (2, 6), (3, 10), (5, 9), (6, 12)])
def test_structure(p, n):
    M, A, S = iga1d.matrices(p, n)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-16)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A, -A.T, rtol=0, atol=1e-14)  # A^T = -A (Section 3.2)
    assert np.linalg.eigvalsh(M).min() > 0 and np.linalg.eigvalsh(S).min() > 0
    # banded with half-bandwidth p
    idx = np.abs(np.subtract.outer(np.arange(M.shape[0]), np.arange(M.shape[0])))
    for X in (M, A, S):
        assert np.all(X[idx > p] == 0)


@pytest.mark.parametrize("p,n", [(1, 4), (3, 7), (5, 6)])
def test_full_mass_sums_to_one_and_quadrature_is_exact(p, n):
    Mf, Af, Sf = iga1d.full_matrices(p, n)
    assert abs(Mf.sum() - 1.0) < 1e-14  # integral of (sum_i N_i)^2 = 1
    assert np.abs(Sf.sum(1)).max() < 1e-10 * n  # derivative of the partition of unity is 0
    Mh, Ah, Sh = iga1d.full_matrices(p, n, nq=p + 4)
    np.testing.assert_allclose(Mh, Mf, atol=1e-15)
    np.testing.assert_allclose(Ah, Af, atol=1e-14)
    np.testing.assert_allclose(Sh, Sf, atol=1e-11 * n)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_central_rows_give_the_symbols(p):
    n = 40
    M, A, S = iga1d.matrices(p, n)
    i = n // 2
    th = np.linspace(-np.pi, np.pi, 33)
    k = np.arange(-p, p + 1)
    # T_m(f) has entries hat f_{i-j}: symbol = sum_k (row i, column i-k) e^{i k theta}
    msym = sum(n * M[i, i - kk] * np.cos(kk * th) for kk in k)
    ssym = sum(S[i, i - kk] / n * np.cos(kk * th) for kk in k)
    asym = sum((-1j * A[i, i - kk]) * np.exp(1j * kk * th) for kk in k)
    np.testing.assert_allclose(msym, symbols.m_sym(p, th), atol=1e-13)
    np.testing.assert_allclose(ssym, symbols.s_sym(p, th), atol=1e-11)
    np.testing.assert_allclose(asym.real, symbols.a_sym(p, th), atol=1e-13)
    assert abs(sum(n * M[i, i - kk] for kk in k) - 1.0) < 1e-13  # m_p(0) = 1


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_T_matrix(p):
    m = 25
    T = iga1d.toeplitz_T(p, m)
    if p == 1:
        np.testing.assert_array_equal(T, np.eye(m))  # Section 6.2: T is the identity at p = 1
    # T_m(m_{p-1}) coincides with the central part of n M^{p-1}
    if p >= 2:
        n = 60
        Mq, _, _ = iga1d.matrices(p - 1, n)
        i = n // 2
        for k in range(-(p - 1), p):
            assert abs(T[10, 10 + k] - n * Mq[i, i + k]) < 1e-13
    ev = np.linalg.eigvalsh(T)
    lo = symbols.m_sym(p - 1, np.pi) if p > 1 else 1.0
    # a Toeplitz matrix of a real even symbol has its eigenvalues in the range of the symbol
    assert ev.min() >= lo - 1e-12 and ev.max() <= 1 + 1e-12


def test_generalized_eigenvalues_p1_closed_form():
    from oracle import solvers
    n = 17
    M, A, S = iga1d.matrices(1, n)
    lam, U = solvers.generalized_eigs(M, S)
    m = n - 1
    th = np.arange(1, m + 1) * np.pi / (m + 1)
    exact = np.sort(6 * n ** 2 * (1 - np.cos(th)) / (2 + np.cos(th)))
    np.testing.assert_allclose(lam, exact, rtol=1e-12)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(m), atol=1e-12)
