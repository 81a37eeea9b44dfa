"""CPU pins of the library's host set-up code (no GPU): the 1D bands, their Galerkin
coarsening, the FD eigenbases and the banded Cholesky factor of T, through the host-only
C-ABI queries, against the oracle."""
import numpy as np
import pytest

from oracle import iga1d, solvers
from paper_1805_10058_gb300 import curldiv as cdl

CASES = [(1, 8), (2, 16), (3, 37), (4, 13), (5, 20), (6, 11)]


def dense(band, P):
    m = band.shape[0]
    out = np.zeros((m, m))
    for i in range(m):
        for k in range(2 * P + 1):
            j = i + k - P
            if 0 <= j < m:
                out[i, j] = band[i, k]
    return out


@pytest.mark.parametrize("p,n", CASES)
def test_bands_equal_oracle_matrices(p, n):
    (Mb, Ab, Sb), P = cdl.cd_setup_bands(p, n)
    for band, ref in zip((Mb, Ab, Sb), iga1d.matrices(p, n)):
        np.testing.assert_allclose(dense(band, P), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    A = dense(Ab, P)
    assert np.array_equal(A, -A.T)  # stored exactly skew (Section 3.2: A^T = -A)


@pytest.mark.parametrize("p,n", [(2, 16), (3, 37), (5, 20)])
def test_coarse_bands_are_galerkin_products(p, n):
    """Level l+1 = P^T X_l P with the 3-tap prolongator of Section 6.1, level by level."""
    (Mf, Af, Sf), P = cdl.cd_setup_bands(p, n, 0)
    fine = [dense(x, P) for x in (Mf, Af, Sf)]
    for level in (1, 2):
        (Mc, Ac, Sc), Pc = cdl.cd_setup_bands(p, n, level)
        Pr = solvers.prolongator_1d(fine[0].shape[0]).toarray()
        for X, band in zip(fine, (Mc, Ac, Sc)):
            ref = Pr.T @ X @ Pr
            np.testing.assert_allclose(dense(band, Pc), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        fine = [dense(x, Pc) for x in (Mc, Ac, Sc)]


@pytest.mark.parametrize("p,n", [(1, 12), (3, 20), (4, 33)])
def test_eigenbases(p, n):
    M, _, S = iga1d.matrices(p, n)
    U, lam = cdl.cd_setup_eig(p, n, 0)
    np.testing.assert_allclose(lam, solvers.generalized_eigs(M, S)[0], rtol=1e-10)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(M.shape[0]), atol=1e-11)
    np.testing.assert_allclose(S @ U, M @ U * lam, atol=1e-9 * lam.max())
    T = iga1d.toeplitz_T(p, n + p - 2)
    Q, lt = cdl.cd_setup_eig(p, n, 1)
    np.testing.assert_allclose(lt, np.linalg.eigvalsh(T), atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(T.shape[0]), atol=1e-12)
    np.testing.assert_allclose(T @ Q, Q * lt, atol=1e-12)


@pytest.mark.parametrize("p,n", CASES)
def test_banded_cholesky_of_T(p, n):
    m, q = n + p - 2, p - 1
    Lb, dinv = cdl.cd_setup_tband(p, n)
    L = np.diag(1.0 / dinv)
    for i in range(m):
        for t in range(q):
            j = i - q + t
            if j >= 0:
                L[i, j] = Lb[i, t]
            else:
                assert Lb[i, t] == 0.0
    assert not Lb[m:].any()  # padding rows past m
    T = iga1d.toeplitz_T(p, m)
    np.testing.assert_allclose(L @ L.T, T, rtol=0, atol=1e-14)
    if p == 1:
        np.testing.assert_array_equal(L, np.eye(m))  # T_m(m_0) = I (Section 6.2, p = 1)


def test_setup_queries_reject_invalid_arguments():
    lib = cdl.load()
    for args in [(0, 8, 0), (7, 8, 0), (2, 0, 0), (1, 1, 0), (2, 8, -1), (2, 8, 9)]:
        assert lib.cd_setup_bands(*args, None, None, None, None, None) == cdl.CD_EINVAL, args
    assert lib.cd_setup_eig(2, 8, 2, None, None) == cdl.CD_EINVAL
    assert lib.cd_setup_tband(7, 8, None, None) == cdl.CD_EINVAL
