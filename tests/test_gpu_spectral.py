"""Spectral validation on the GPU (Section 5) through the C-ABI: the symbol's eigenvalue functions
sampled on the grid Gamma (cd_symbol_eigs) against the oracle's symbols, their Laplacian bounds
(Theorems 5.2 / 5.6), and Lanczos extremal eigenvalues of A (cd_lanczos) against dense
eigenvalues and the matrix form of the bounds."""
import numpy as np
import pytest

from oracle import assemble, symbols

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402


def gpu_symbol(d, p, alpha, beta, mg, nu=None):
    lam = torch.empty(mg ** d * d, dtype=torch.float64, device="cuda")
    lap = torch.empty(mg ** d, dtype=torch.float64, device="cuda")
    cdl.cd_symbol_eigs(d, p, alpha, beta, mg, lam, lap, nu)
    torch.cuda.synchronize()
    return lam.cpu().numpy().reshape(-1, d), lap.cpu().numpy()


@pytest.mark.parametrize("d,p,beta,mg", [(2, 3, 0.5, 40), (2, 3, 0.01, 40), (2, 1, 7.0, 33),
                                         (2, 6, 1e-6, 64), (3, 2, 0.01, 12), (3, 4, 100.0, 9)])
def test_symbol_eigenvalues_match_oracle(d, p, beta, mg):
    lam, lap = gpu_symbol(d, p, 1.0, beta, mg)
    ref = symbols.sampled_eigs(d, p, 1.0, beta, mg)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-12 * scale)
    g = symbols.grid(mg, d)
    np.testing.assert_allclose(lap, symbols.laplacian_sym(p, *g).ravel(), rtol=0,
                               atol=1e-12 * np.abs(lap).max())
    # Theorems 5.2 / 5.6: min(alpha,beta) L_p <= lambda_i <= max(alpha,beta) L_p at every point
    lo, hi = min(1.0, beta), max(1.0, beta)
    tol = 1e-12 * scale
    assert np.all(lam >= lo * lap[:, None] - tol) and np.all(lam <= hi * lap[:, None] + tol)


@pytest.mark.parametrize("d,nu", [(2, (1.0, 2.0)), (3, (1.0, 0.5, 2.0))])
def test_anisotropic_symbol_bounds_and_scaling(d, nu):
    """Weighted symbols (Theorems 5.1 / 5.5 with n_l = n nu_l): the Laplacian bounds hold, nu = 1
    reproduces the isotropic symbol, and scaling nu by c scales the 3D symbol by 1/c (2D: 1)."""
    p, beta, mg = 3, 0.05, 16
    lam, lap = gpu_symbol(d, p, 1.0, beta, mg, nu)
    tol = 1e-12 * np.abs(lam).max()
    assert np.all(lam >= beta * lap[:, None] - tol) and np.all(lam <= lap[:, None] + tol)
    lam1, _ = gpu_symbol(d, p, 1.0, beta, mg, [1.0] * d)
    np.testing.assert_allclose(lam1, symbols.sampled_eigs(d, p, 1.0, beta, mg), rtol=0,
                               atol=1e-12 * np.abs(lam1).max())
    lam3, _ = gpu_symbol(d, p, 1.0, beta, mg, [3.0 * v for v in nu])
    factor = 1.0 if d == 2 else 1.0 / 3.0
    np.testing.assert_allclose(lam3, factor * lam, rtol=1e-12, atol=1e-13 * np.abs(lam).max())


@pytest.mark.parametrize("d,p,n,beta", [(2, 2, 12, 0.01), (2, 3, 10, 100.0), (3, 2, 5, 0.1)])
def test_lanczos_extremes_match_dense_eigenvalues(d, p, n, beta):
    N = cdl.cd_dofs(d, p, n)
    s = cdl.Solver(d, p, n, 1.0, beta, max_batch=2)
    v0 = torch.as_tensor(inputs.uniform_rhs(d, p, n, seed=9, nrhs=2).ravel(), device="cuda")
    steps = min(N, 400)
    lmin, lmax, _, _ = s.cd_lanczos(v0, steps, [1.0, 1.0], [beta, 1.0])
    for k, bk in enumerate((beta, 1.0)):
        ev = np.linalg.eigvalsh(assemble.galerkin_kron(d, p, n, 1.0, bk).toarray())
        assert abs(lmax[k] - ev[-1]) <= 1e-9 * ev[-1], (k, lmax[k], ev[-1])
        assert abs(lmin[k] - ev[0]) <= 1e-7 * ev[-1], (k, lmin[k], ev[0])


def test_lanczos_extremes_obey_the_laplacian_bounds_at_benchmark_size():
    """n = 256, p = 3: the matrix form of Theorem 5.2 puts the spectrum of A between
    min(alpha,beta) and max(alpha,beta) times that of the block Laplacian K = A(1, 1); the
    Lanczos estimates of the largest eigenvalues obey it.  (The largest eigenvalue of A itself lies
    above the maximum of the symbol samples: measured 1.57 against 1.09 at beta = 1e-3, an outlier
    of the boundary rows, which the spectral distribution of Theorem 5.1 does not constrain.)"""
    d, p, n = 2, 3, 256
    s = cdl.Solver(d, p, n, max_batch=3)
    v0 = torch.as_tensor(inputs.uniform_rhs(d, p, n, seed=4, nrhs=3).ravel(), device="cuda")
    betas = [1.0, 1e-3, 1e3]
    lmin, lmax, _, _ = s.cd_lanczos(v0, 300, [1.0] * 3, betas)
    kmax = lmax[0]
    for k in (1, 2):
        hi = max(1.0, betas[k])
        assert lmax[k] <= hi * kmax * (1 + 1e-6), (lmax[k], kmax)
        assert lmin[k] > 0
        lo = min(1.0, betas[k])
        assert lmax[k] >= lo * kmax * (1 - 1e-6), (lmax[k], kmax)
