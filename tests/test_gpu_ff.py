"""The 2D operator apply in double-FP32 arithmetic (FP64 vectors, float-float products and sums
on the FP32 pipe) through the C-ABI: elementwise against the oracle's assembled matrix, and the
refinement loop's inner FP64 solves with it (emulated_fp64) against the same solves with FP64
applies."""
import numpy as np
import pytest

from gpu_helpers import abs_matvec_bound, oracle_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402

# about 48 significant bits per operation over <= 3 (2p+1) terms per pass and two passes
FF_TOL = 5e-13


@pytest.mark.parametrize("kernel", ["ff1", "ff2", "ff2-wide", "ff2-narrow"])
@pytest.mark.parametrize("p,n,beta", [(1, 9, 1.0), (2, 40, 1e-6), (3, 70, 1e3), (4, 33, 0.01),
                                      (5, 41, 1e-6), (6, 30, 1e6), (3, 256, 1e-3)])
def test_double_fp32_apply_matches_oracle(p, n, beta, kernel, monkeypatch):
    """Both double-FP32 kernels: ff1 (plain band sums) and ff2 (packed pairs, folded interior
    stencils) with its tile chosen by the grid size, forced wide (24 or 20 rows) or narrow (8
    rows); sizes span several tiles with ragged tails in both axes."""
    kernel, _, rows = kernel.partition("-")
    monkeypatch.setenv("CURLDIV_APPLY_KERNEL_FP64", kernel)
    monkeypatch.setenv("CURLDIV_FF2_ROWS", {"": "0", "wide": "24", "narrow": "8"}[rows])
    d, B = 2, 3
    W = inputs.uniform_rhs(d, p, n, seed=31, nrhs=B)
    s = cdl.Solver(d, p, n, 1.0, beta, max_batch=B, autotune=0)
    w = torch.as_tensor(W.ravel(), device="cuda")
    y = torch.zeros_like(w)
    s.cd_apply(w, y)
    Y = y.cpu().numpy().reshape(B, -1)
    A = oracle_matrix(d, p, n, 1.0, beta)
    worst = 0.0
    for k in range(B):
        bound = abs_matvec_bound(A, W[k])
        err = np.abs(Y[k] - A @ W[k]) / bound
        worst = max(worst, float(err.max()))
    print("double-FP32 apply", kernel, "worst error / (|A||w|):", p, n, beta, worst)
    assert worst <= FF_TOL, worst


@pytest.mark.parametrize("rows", ["0", "24"])
@pytest.mark.parametrize("p,n", [(2, 62), (3, 61)])
def test_emulated_inner_solves_reach_rtol_like_fp64(p, n, rows, monkeypatch):
    """Extreme and moderate ratios in one batch: with double-FP32 inner applies the refinement loop
    still reaches rtol = 1e-10 for x + x_lo, in a comparable number of inner iterations (tiles
    chosen by the grid size, or the wide tile on every level)."""
    monkeypatch.setenv("CURLDIV_FF2_ROWS", rows)
    betas = [1e-6, 1e-3, 1.0, 1e6]
    B = len(betas)
    Bv = inputs.uniform_rhs(2, p, n, seed=2, nrhs=B)
    b = torch.as_tensor(Bv.ravel(), device="cuda")
    out = {}
    for emu in (1, 0):
        s = cdl.Solver(2, p, n, max_batch=B, precond=cdl.CD_PC_MG, rtol=1e-10, maxit=40000,
                       emulated_fp64=emu)
        x, xl = torch.zeros_like(b), torch.zeros_like(b)
        st, res = s.cd_solve_ext(b, x, xl, [1.0] * B, betas, check=False)
        assert st == cdl.CD_OK, (emu, res)
        assert all(r["relres"] <= 1e-10 for r in res), (emu, res)
        out[emu] = [r["iters_inner"] for r in res]
    print("inner iterations emulated / FP64:", out[1], out[0])
    for k in range(B):
        assert out[1][k] <= 1.6 * out[0][k] + 20, (k, out)


@pytest.mark.parametrize("p,n,beta", [(1, 7, 1.0), (2, 9, 1e-6), (3, 11, 1e3), (5, 6, 1e6),
                                      (4, 15, 1e-3), (6, 9, 1.0)])
def test_double_fp32_3d_apply_matches_oracle(p, n, beta, monkeypatch):
    """The 3D apply in double-FP32 (the three tuned passes with (hi, lo) FP32 intermediates),
    elementwise against the oracle's assembled matrix."""
    monkeypatch.setenv("CURLDIV_APPLY_KERNEL_FP64", "ff")
    d, B = 3, 2
    W = inputs.uniform_rhs(d, p, n, seed=33, nrhs=B)
    s = cdl.Solver(d, p, n, 1.0, beta, max_batch=B, autotune=0)
    w = torch.as_tensor(W.ravel(), device="cuda")
    y = torch.zeros_like(w)
    s.cd_apply(w, y)
    Y = y.cpu().numpy().reshape(B, -1)
    A = oracle_matrix(d, p, n, 1.0, beta)
    worst = 0.0
    for k in range(B):
        err = np.abs(Y[k] - A @ W[k]) / abs_matvec_bound(A, W[k])
        worst = max(worst, float(err.max()))
    print("double-FP32 3D apply, worst error / (|A||w|):", p, n, beta, worst)
    assert worst <= FF_TOL, worst


@pytest.mark.parametrize("precond", [cdl.CD_PC_FD_D, cdl.CD_PC_MG])
def test_emulated_inner_solves_reach_rtol_like_fp64_3d(precond):
    """3D: the FP64 inner group with double-FP32 applies (the tuned passes) reaches rtol = 1e-10
    for x + x_lo at extreme and moderate ratios, in a comparable number of inner iterations."""
    p, n = 2, 14
    betas = [1e-6, 1e-3, 1.0, 1e6]
    B = len(betas)
    Bv = inputs.uniform_rhs(3, p, n, seed=4, nrhs=B)
    b = torch.as_tensor(Bv.ravel(), device="cuda")
    out = {}
    for emu in (1, 0):
        s = cdl.Solver(3, p, n, max_batch=B, precond=precond, rtol=1e-10, maxit=40000,
                       emulated_fp64=emu)
        x, xl = torch.zeros_like(b), torch.zeros_like(b)
        st, res = s.cd_solve_ext(b, x, xl, [1.0] * B, betas, check=False)
        assert st == cdl.CD_OK, (emu, res)
        assert all(r["relres"] <= 1e-10 for r in res), (emu, res)
        out[emu] = [r["iters_inner"] for r in res]
        s.close()
    print("3D inner iterations emulated / FP64:", out[1], out[0])
    for k in range(B):
        assert out[1][k] <= 1.6 * out[0][k] + 20, (k, out)
