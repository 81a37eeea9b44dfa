"""The paper's multigrid strategies on the GPU (Section 6.1, Section 6.2) through the C-ABI:
P_MIM (CD_PC_MIM: two V-cycles per application with p PGMRES-T post-smoothing steps at the finest
level) and P_WL (CD_PC_WL: one V-cycle on D = blockdiag(A^(c,c)) with p PCG-T steps), on the
setting of Tables 1-2 (alpha = 1, manufactured right-hand side, zero initial guess, stop at
||r_k|| / ||r_0|| < 1e-7, FP64).

The GPU replaces the paper's sequential Gauss-Seidel by the parallel Chebyshev-Jacobi smoother,
so its counts are not expected to equal the printed ones; the tests hold them to a band around
Tables 1-2, check that they do not grow with n, and check the solution against the oracle."""
import numpy as np
import pytest

from conftest import paper_tables
from oracle import assemble, solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402

_cache = {}


def _rhs(d, p, n, beta):
    key = (d, p, n, beta)
    if key not in _cache:
        field = assemble.manufactured_2d if d == 2 else assemble.manufactured_3d
        _cache[key] = assemble.load_vector(d, p, n, 1.0, beta, field)
    return _cache[key]


def gpu_count(d, p, n, beta, pc):
    b = _rhs(d, p, n, beta)
    # every strategy on the paper's hierarchy (Section 6.1: coarsened to m <= 3 here)
    s = cdl.Solver(d, p, n, 1.0, beta, max_batch=1, precond=pc, precision=cdl.CD_PREC_FP64,
                   rtol=1e-7, maxit=5000, ext_residual=0, mg_m_min=3)
    bt = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    st, res = s.cd_solve(bt, x, check=False)
    return st, res[0], x.cpu().numpy(), b


ROWS = [r for r in paper_tables() if r["d"] == 2 and r["p"] <= 3 and r["n"] + r["p"] - 1 <= 64]


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"{r['table']}-p{r['p']}-n{r['n']}")
def test_p_mim_and_p_wl_follow_tables(row):
    d, p, n, beta = row["d"], row["p"], row["n"], row["beta"]
    out = {}
    for name, pc in (("pmim", cdl.CD_PC_MIM), ("pwl", cdl.CD_PC_WL), ("mg", cdl.CD_PC_MG)):
        st, res, x, b = gpu_count(d, p, n, beta, pc)
        assert st == cdl.CD_OK, (name, res)
        out[name] = res["iters_inner"]
        if name == "pmim":
            A = assemble.galerkin_kron(d, p, n, 1.0, beta)
            xs = solvers.direct_solve(A, b)
            assert np.linalg.norm(b - A @ x) <= 1.01e-7 * np.linalg.norm(b)
            assert np.linalg.norm(x - xs) <= 1e-4 * np.linalg.norm(xs)
    print(row["table"], p, n, "gpu", out, "paper", row["pmim"], row["pwl"])
    # measured on GB300: P_MIM within +-3 (p = 1: within 21%) of the printed counts, P_WL 0-21%
    # above them
    assert abs(out["pmim"] - row["pmim"]) <= max(3, 0.25 * row["pmim"]), (out, row)
    assert row["pwl"] - 3 <= out["pwl"] <= 1.3 * row["pwl"] + 3, (out, row)
    # the paper's ordering of the strategies, and the Krylov post-smoother's gain over the
    # V-cycle with the parallel smoother alone
    assert out["pmim"] < out["pwl"] and out["pmim"] < out["mg"], out


@pytest.mark.parametrize("p,beta", [(2, 0.1), (3, 0.01)])
def test_p_mim_is_flat_in_n_on_gpu(p, beta):
    ks = []
    for k in (4, 5, 6):
        n = 2 ** k - p + 1
        st, res, _, _ = gpu_count(2, p, n, beta, cdl.CD_PC_MIM)
        assert st == cdl.CD_OK, res
        ks.append(res["iters_inner"])
    print("p_mim over n", p, beta, ks)
    assert max(ks) - min(ks) <= 3, ks


@pytest.mark.parametrize("row", [r for r in paper_tables() if r["d"] == 3 and r["n"] + r["p"] - 1 == 16
                                 and r["p"] <= 3], ids=lambda r: f"{r['table']}-p{r['p']}-n{r['n']}")
def test_p_mim_3d_follows_tables(row):
    d, p, n, beta = 3, row["p"], row["n"], row["beta"]
    st, res, x, b = gpu_count(d, p, n, beta, cdl.CD_PC_MIM)
    assert st == cdl.CD_OK, res
    print(row["table"], p, n, "gpu", res["iters_inner"], "paper", row["pmim"])
    assert abs(res["iters_inner"] - row["pmim"]) <= 3, (res, row)


def test_krylov_smoothed_preconditioners_batch_invariant():
    """A solve gives the same bits alone and inside a batch with other parameters."""
    d, p, n = 2, 3, 14
    rng = np.random.default_rng(3)
    N = cdl.cd_dofs(d, p, n)
    B = rng.uniform(-1, 1, (3, N))
    betas = [0.1, 0.01, 10.0]
    for pc in (cdl.CD_PC_MIM, cdl.CD_PC_WL):
        s = cdl.Solver(d, p, n, max_batch=3, precond=pc, precision=cdl.CD_PREC_FP64, rtol=1e-9)
        xb = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        s.cd_solve(torch.as_tensor(B.ravel(), device="cuda"), xb, [1.0] * 3, betas)
        s1 = cdl.Solver(d, p, n, max_batch=1, precond=pc, precision=cdl.CD_PREC_FP64, rtol=1e-9)
        x1 = torch.zeros(N, dtype=torch.float64, device="cuda")
        s1.cd_solve(torch.as_tensor(B[1], device="cuda"), x1, [1.0], [betas[1]])
        assert torch.equal(xb[N:2 * N], x1), pc
