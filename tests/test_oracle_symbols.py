"""Pins for oracle/symbols.py: Lemma 3.2, the closed-form eigenvalue functions
(eq:expres:eig:1/2), Theorems 5.2 / 5.6, and eigenvalues of the assembled matrices against
samples of the symbol on the grid Gamma (Section 5.3)."""
import numpy as np
import pytest

from oracle import assemble, iga1d, symbols

TH = np.linspace(-np.pi, np.pi, 401)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_lemma_3_2(p):
    m, a, s = symbols.m_sym(p, TH), symbols.a_sym(p, TH), symbols.s_sym(p, TH)
    # (a): m_p > 0, maximal at 0 and minimal at pi.  The printed lower bound (2/pi)^{2p} is
    # already violated at p = 1 (m_1(pi) = 1/3 < 4/pi^2); the bound with exponent 2p + 2 holds.
    half = TH >= 0
    assert np.all(np.diff(m[half]) <= 1e-15)
    assert m.min() >= (2 / np.pi) ** (2 * p + 2) and m.max() <= 1 + 1e-14
    assert symbols.m_sym(p, np.pi) < (2 / np.pi) ** (2 * p)
    assert abs(symbols.m_sym(p, 0.0) - 1.0) < 1e-14
    if p >= 1:
        np.testing.assert_allclose(s, symbols.m_sym(p - 1, TH) * (2 - 2 * np.cos(TH)), atol=1e-13)  # (b)
    assert symbols.s_sym(p, np.pi) <= 2 ** (2 - p) * s.max() + 1e-14
    gap = m * s - a ** 2  # (c), equality only at theta = 0
    assert gap.min() >= -1e-14
    assert np.all(gap[np.abs(TH) > 0.5] > 0)  # the zero at 0 has order 2p + 2, so stay away from it


def test_p1_symbols_closed_form():
    np.testing.assert_allclose(symbols.m_sym(1, TH), (2 + np.cos(TH)) / 3, atol=1e-15)
    np.testing.assert_allclose(symbols.s_sym(1, TH), 2 - 2 * np.cos(TH), atol=1e-15)
    np.testing.assert_allclose(symbols.a_sym(1, TH), -np.sin(TH), atol=1e-15)


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("beta", [0.5, 0.01, 20.0])
def test_2d_closed_form_and_bounds(p, beta):
    alpha = 1.0
    g1, g2 = np.meshgrid(TH[::8], TH[::8], indexing="ij")
    l1, l2 = symbols.eig_2d_closed(p, alpha, beta, g1, g2)
    ev = np.linalg.eigvalsh(symbols.symbol_2d(p, alpha, beta, g1, g2))
    sc = np.abs(ev).max()
    np.testing.assert_allclose(l1, ev[..., 0], atol=1e-13 * sc)
    np.testing.assert_allclose(l2, ev[..., 1], atol=1e-13 * sc)
    L = symbols.laplacian_sym(p, g1, g2)
    lo, hi = min(alpha, beta), max(alpha, beta)
    assert np.all(lo * L <= l1 + 1e-13 * sc) and np.all(l2 <= hi * L + 1e-13 * sc)  # Thm 5.2


@pytest.mark.parametrize("p", [2, 3, 5])
@pytest.mark.parametrize("beta", [0.5, 0.01, 20.0])
def test_3d_bounds(p, beta):
    alpha = 1.0
    lam = symbols.sampled_eigs(3, p, alpha, beta, 12)
    L = symbols.laplacian_sym(p, *[g.ravel() for g in symbols.grid(12, 3)])
    lo, hi = min(alpha, beta), max(alpha, beta)
    sc = lam.max()
    assert np.all(lo * L[:, None] <= lam + 1e-13 * sc) and np.all(lam <= hi * L[:, None] + 1e-13 * sc)


def test_equal_parameters_give_laplacian():
    g = symbols.grid(9, 3)
    lam = symbols.sampled_eigs(3, 3, 2.0, 2.0, 9)
    L = symbols.laplacian_sym(3, *[t.ravel() for t in g])
    np.testing.assert_allclose(lam, np.repeat(2.0 * L[:, None], 3, 1), rtol=1e-12)


@pytest.mark.parametrize("d,n,beta", [(2, 40, 0.5), (2, 40, 0.01), (3, 12, 0.5)])
def test_eigenvalues_follow_symbol_samples(d, n, beta):
    """Sorted eig(n^{d-2} A) against sorted samples of lambda_i(f) on Gamma (Section 5.3)."""
    p = 3
    m = n + p - 2
    A = assemble.galerkin_kron(d, p, n, 1.0, beta).toarray() * n ** (d - 2)
    ev = np.sort(np.linalg.eigvalsh(A))
    samp = np.sort(symbols.sampled_eigs(d, p, 1.0, beta, m).ravel())
    assert ev.size == samp.size
    err = np.abs(ev - samp) / samp.max()
    assert np.median(err) < 0.01 and np.quantile(err, 0.95) < 0.05
    if beta == 0.01 and d == 2:
        # about half of the spectrum is close to zero (Section 5.3, 2D, beta = 0.01)
        frac = np.mean(ev < 0.02 * ev.max())
        assert 0.35 < frac < 0.65


def test_symbol_sampling_refines_with_n():
    p, beta = 2, 0.1
    errs = []
    for n in (10, 20, 40):
        m = n + p - 2
        A = assemble.galerkin_kron(2, p, n, 1.0, beta).toarray()
        ev = np.sort(np.linalg.eigvalsh(A))
        samp = np.sort(symbols.sampled_eigs(2, p, 1.0, beta, m).ravel())
        errs.append(np.mean(np.abs(ev - samp)) / samp.max())
    assert errs[0] > errs[1] > errs[2]


def test_mass_matrix_spectrum_follows_m_p():
    p, n = 3, 120
    M, _, _ = iga1d.matrices(p, n)
    m = n + p - 2
    ev = np.sort(np.linalg.eigvalsh(n * M))
    samp = np.sort(symbols.m_sym(p, np.arange(1, m + 1) * np.pi / m))
    assert np.max(np.abs(ev - samp)) < 0.05


def test_3d_one_third_of_spectrum_near_zero_for_small_beta():
    """3D, beta = 0.01: about one third of the spectrum is almost zero (Section 5.3)."""
    p, n = 3, 8
    A = assemble.galerkin_kron(3, p, n, 1.0, 0.01).toarray() * n
    ev = np.linalg.eigvalsh(A)
    frac = np.mean(ev < 0.02 * ev.max())
    assert 0.23 < frac < 0.43, frac


# ---- anisotropic meshes n_l = n nu_l (Section 5, Theorems 5.1 / 5.5)

@pytest.mark.parametrize("d,ns,beta", [(2, (20, 40), 0.5), (2, (36, 12), 0.01), (3, (6, 12, 9), 0.5)])
def test_anisotropic_eigenvalues_follow_weighted_symbol(d, ns, beta):
    """Sorted eig(n^{d-2} A_n) for n = n nu against the sorted weighted symbol sampled on the
    per-direction grid (m_l points along x_l); the isotropic symbol of the same mesh size does
    not match, so a wrong weight or a swapped direction fails."""
    p = 3
    n = min(ns)
    nu = tuple(v / n for v in ns)
    ms = tuple(v + p - 2 for v in ns)
    A = assemble.galerkin_kron(d, p, ns, 1.0, beta).toarray() * n ** (d - 2)
    ev = np.sort(np.linalg.eigvalsh(A))
    samp = np.sort(symbols.sampled_eigs(d, p, 1.0, beta, ms, nu=nu).ravel())
    assert ev.size == samp.size
    err = np.abs(ev - samp) / samp.max()
    assert np.median(err) < 0.01 and np.quantile(err, 0.95) < 0.05
    iso = np.sort(symbols.sampled_eigs(d, p, 1.0, beta, ms).ravel())
    assert np.median(np.abs(ev - iso) / iso.max()) > 2 * np.median(err)


@pytest.mark.parametrize("d,nu", [(2, (1.0, 3.0)), (3, (2.0, 1.0, 0.5))])
def test_weighted_symbol_bounds(d, nu):
    """min(alpha,beta) L_p <= lambda_i(f) <= max(alpha,beta) L_p with the weighted Laplacian
    symbol (Theorems 5.2 / 5.6 on anisotropic meshes), equality at alpha = beta."""
    p, beta, mg = 3, 0.02, 14
    g = symbols.grid(mg, d)
    lam = symbols.sampled_eigs(d, p, 1.0, beta, mg, nu=nu)
    L = symbols.laplacian_sym(p, *g, nu=nu).ravel()
    sc = np.abs(lam).max()
    assert np.all(beta * L[:, None] <= lam + 1e-13 * sc) and np.all(lam <= L[:, None] + 1e-13 * sc)
    lam1 = symbols.sampled_eigs(d, p, 0.7, 0.7, mg, nu=nu)
    np.testing.assert_allclose(lam1, np.repeat(0.7 * L[:, None], d, 1), rtol=1e-12, atol=1e-14 * sc)
