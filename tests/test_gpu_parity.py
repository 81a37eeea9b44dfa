"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic):
* operator apply, FP64: |y_gpu - y_ref|_i <= 1e-13 (|A||w|)_i  (a sum of <= 12(2p+1) products
  per entry, each rounding by <= 2^-53);
* operator apply, FP32 bands and vectors: <= 3e-5 (|A||w|)_i  (same count at 2^-24);
* FD solves in FP64: <= 1e-10 relative to the oracle's sparse-LU solve (dense transforms with
  condition number of U bounded by cond(M)^(1/2));
* solves: oracle-measured relative residual <= rtol (plus the FP64 rounding floor of the
  residual itself), and relative error <= 1e-9 where the solve is driven to rtol = 1e-13.
"""
import numpy as np
import pytest

from gpu_helpers import abs_matvec_bound, kron_rows, oracle_matrix
from oracle import assemble, iga1d, solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


APPLY_CASES = [(2, 1, 9), (2, 2, 16), (2, 3, 37), (2, 5, 30), (2, 2, 3), (2, 6, 60), (2, 4, 257),
               (3, 1, 5), (3, 2, 7), (3, 3, 9), (3, 4, 6)]


@pytest.mark.parametrize("variant", ["v5", "v3", "v2", "v1"])
@pytest.mark.parametrize("d,p,n", APPLY_CASES)
def test_apply_fp64_and_fp32_match_oracle(d, p, n, variant, monkeypatch):
    """Every 2D kernel (FP32: v5 folded tiles, v3 packed pairs; v2; plain shared-memory v1) and
    the 3D designs (streaming, the tuned three passes in FP32 and FP64, the generic axis passes)
    against the oracle."""
    if d == 3 and variant == "v5":
        pytest.skip("three 3D designs")
    if d == 3:
        monkeypatch.setenv("CURLDIV_APPLY3D_KERNEL",
                           {"v3": "stream", "v2": "pass64", "v1": "axis"}[variant])
    else:
        monkeypatch.setenv("CURLDIV_APPLY_KERNEL", variant)
        monkeypatch.setenv("CURLDIV_APPLY_KERNEL_FP64", "v3" if variant == "v3" else "v2")
    alphas = np.array([1.0, 0.5, 3.0])
    betas = np.array([0.1, 7.0, 3.0])
    s = cdl.Solver(d, p, n, max_batch=3, autotune=0)
    N = s.N
    W = inputs.uniform_rhs(d, p, n, seed=11, nrhs=3)
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    s.cd_apply(dev(W.ravel()), y, alphas, betas)
    Y = host(y).reshape(3, N)
    y32 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    s.cd_apply_f32(dev(W.ravel(), torch.float32), y32, alphas, betas)
    Y32 = host(y32).reshape(3, N)
    for k in range(3):
        A = oracle_matrix(d, p, n, alphas[k], betas[k])
        ref = A @ W[k]
        bound = abs_matvec_bound(A, W[k])
        assert np.all(np.abs(Y[k] - ref) <= 1e-13 * bound + 1e-300), k
        w32 = W[k].astype(np.float32).astype(np.float64)
        ref32 = A @ w32
        assert np.all(np.abs(Y32[k] - ref32) <= 3e-5 * abs_matvec_bound(A, w32) + 1e-30), k


@pytest.mark.parametrize("d,p,n,nsamp", [(2, 3, 256, 4000), (2, 4, 256, 2000), (3, 3, 64, 300),
                                         (3, 3, 128, 120)])
def test_apply_full_size_sampled(d, p, n, nsamp):
    """At the benchmark sizes: sampled outputs of the FP64 apply against the oracle's 1D
    matrices evaluated row by row."""
    s = cdl.Solver(d, p, n, max_batch=1, precond=cdl.CD_PC_NONE)
    w = inputs.uniform_rhs(d, p, n, seed=5)[0]
    y = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.cd_apply(dev(w), y, [1.0], [1e-3])
    Y = host(y)
    w32 = w.astype(np.float32).astype(np.float64)
    y32 = torch.zeros(s.N, dtype=torch.float32, device="cuda")
    s.cd_apply_f32(dev(w32, torch.float32), y32, [1.0], [1e-3])
    Y32 = host(y32)
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.integers(0, s.N, nsamp), [0, s.N - 1, s.N // d, s.N // d - 1]])
    ref, bound = kron_rows(d, p, n, 1.0, 1e-3, w, rows)
    assert np.all(np.abs(Y[rows] - ref) <= 1e-13 * bound)
    ref32, bound32 = kron_rows(d, p, n, 1.0, 1e-3, w32, rows)
    assert np.all(np.abs(Y32[rows] - ref32) <= 3e-5 * bound32)


def test_2d_large_grid_beyond_fused_partials():
    """m = 2047 (8.4M unknowns per solve): more apply tiles than fused dot-partial slots, so the
    apply runs without them and the dot kernel supplies the partials.  Sampled rows of the FP64
    and FP32 apply against the oracle's 1D matrices, then a multigrid solve of two right-hand
    sides whose true residual is estimated from sampled rows."""
    d, p, n = 2, 3, 2046
    s = cdl.Solver(d, p, n, max_batch=2, precision=cdl.CD_PREC_FP32_IR, precond=cdl.CD_PC_MG,
                   rtol=1e-9, maxit=3000)
    w = inputs.uniform_rhs(d, p, n, seed=5)[0]
    y = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.cd_apply(dev(w), y, [1.0], [0.3])
    w32 = w.astype(np.float32).astype(np.float64)
    y32 = torch.zeros(s.N, dtype=torch.float32, device="cuda")
    s.cd_apply_f32(dev(w32, torch.float32), y32, [1.0], [0.3])
    rng = np.random.default_rng(2)
    rows = np.concatenate([rng.integers(0, s.N, 300), [0, s.N - 1, s.N // 2, s.N // 2 - 1]])
    ref, bound = kron_rows(d, p, n, 1.0, 0.3, w, rows)
    assert np.all(np.abs(host(y)[rows] - ref) <= 1e-13 * bound)
    ref32, bound32 = kron_rows(d, p, n, 1.0, 0.3, w32, rows)
    assert np.all(np.abs(host(y32)[rows] - ref32) <= 3e-5 * bound32)
    Bv = inputs.uniform_rhs_seeds(d, p, n, [0, 1])
    x = torch.zeros(2 * s.N, dtype=torch.float64, device="cuda")
    st, res = s.cd_solve(dev(Bv.ravel()), x, [1.0, 1.0], [1.0, 0.3], check=False)
    assert st == cdl.CD_OK, res
    X = host(x).reshape(2, -1)
    for k, beta in enumerate([1.0, 0.3]):
        assert res[k]["relres"] <= 1e-9
        ax, _ = kron_rows(d, p, n, 1.0, beta, X[k], rows)
        r = Bv[k][rows] - ax
        est = np.sqrt(s.N / rows.size * np.sum(r ** 2)) / np.linalg.norm(Bv[k])
        assert est <= 3e-9, est


@pytest.mark.parametrize("d,p,n", [(2, 1, 7), (2, 3, 19), (2, 6, 30), (3, 2, 9), (3, 4, 6)])
def test_banded_T_solve_matches_oracle(d, p, n):
    """CD_PC_T_BAND (banded Cholesky of T_m along every axis) against the oracle's T solve
    (one LU of the 1D factor per axis, Section 6.1) and against the fast-diagonalisation
    inverse of the same T."""
    B = 2
    s = cdl.Solver(d, p, n, max_batch=B, precond=cdl.CD_PC_NONE)
    m = n + p - 2
    r = np.random.default_rng(p).uniform(-1, 1, B * s.N)
    ts = solvers.TSolver(d, p, m)
    ref = np.concatenate([ts(r[k * s.N:(k + 1) * s.N]) for k in range(B)])
    z = torch.zeros(B * s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_T_BAND, dev(r), z)
    Z = host(z)
    assert np.abs(Z - ref).max() <= 1e-12 * np.abs(ref).max()
    z32 = torch.zeros(B * s.N, dtype=torch.float32, device="cuda")
    s.cd_precond(cdl.CD_PC_T_BAND, dev(r, torch.float32), z32)
    assert np.abs(host(z32) - ref).max() <= 1e-4 * np.abs(ref).max()
    zf = torch.zeros(B * s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_FD_T, dev(r), zf)
    assert np.abs(host(zf) - Z).max() <= 1e-10 * np.abs(ref).max()


def test_bands_match_oracle_matrices():
    for p, n in [(1, 8), (2, 16), (3, 37), (5, 20)]:
        s = cdl.Solver(2, p, n, max_batch=1)
        (Mb, Ab, Sb), P = s.cd_get_bands(0)
        M, A, S = iga1d.matrices(p, n)
        m = n + p - 2
        for band, ref in ((Mb, M), (Ab, A), (Sb, S)):
            dense = np.zeros((m, m))
            for i in range(m):
                for k in range(2 * P + 1):
                    j = i + k - P
                    if 0 <= j < m:
                        dense[i, j] = band[i, k]
            np.testing.assert_allclose(dense, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_eigenbases():
    for p, n in [(1, 12), (3, 20), (4, 33)]:
        s = cdl.Solver(2, p, n, max_batch=1)
        M, A, S = iga1d.matrices(p, n)
        U, lam = s.cd_get_eig(0)
        ref = solvers.generalized_eigs(M, S)[0]
        np.testing.assert_allclose(lam, ref, rtol=1e-10)
        np.testing.assert_allclose(U.T @ M @ U, np.eye(M.shape[0]), atol=1e-11)
        np.testing.assert_allclose(S @ U, M @ U * lam, atol=1e-9 * lam.max())
        T = iga1d.toeplitz_T(p, n + p - 2)
        Q, lt = s.cd_get_eig(1)
        np.testing.assert_allclose(lt, np.linalg.eigvalsh(T), atol=1e-12)
        np.testing.assert_allclose(Q.T @ Q, np.eye(T.shape[0]), atol=1e-12)


@pytest.mark.parametrize("d,p,n", [(2, 2, 16), (2, 3, 29), (3, 2, 8), (3, 3, 7)])
def test_fd_preconditioners_match_direct_solves(d, p, n):
    s = cdl.Solver(d, p, n, max_batch=2)
    alphas, betas = np.array([1.0, 2.0]), np.array([0.01, 50.0])
    R = inputs.uniform_rhs(d, p, n, seed=3, nrhs=2)
    z = torch.zeros(2 * s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_FD_D, dev(R.ravel()), z, alphas, betas)
    Z = host(z).reshape(2, -1)
    z32 = torch.zeros(2 * s.N, dtype=torch.float32, device="cuda")
    s.cd_precond(cdl.CD_PC_FD_D, dev(R.ravel(), torch.float32), z32, alphas, betas)
    Z32 = host(z32).reshape(2, -1)  # tcgen05, TF32 operands
    s_simt = cdl.Solver(d, p, n, max_batch=2, fd_tensor_cores=0)
    z32s = torch.zeros(2 * s.N, dtype=torch.float32, device="cuda")
    s_simt.cd_precond(cdl.CD_PC_FD_D, dev(R.ravel(), torch.float32), z32s, alphas, betas)
    Z32s = host(z32s).reshape(2, -1)  # SIMT FP32
    for k in range(2):
        A = oracle_matrix(d, p, n, alphas[k], betas[k])
        ref = solvers.solve_D(A, d, R[k])
        assert np.linalg.norm(Z[k] - ref) <= 1e-10 * np.linalg.norm(ref)
        assert np.linalg.norm(Z32s[k] - ref) <= 1e-4 * np.linalg.norm(ref)
        # TF32 keeps 10 mantissa bits (unit roundoff 2^-11 ~ 4.9e-4) through four passes
        assert np.linalg.norm(Z32[k] - ref) <= 5e-3 * np.linalg.norm(ref)
    zt = torch.zeros(2 * s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_FD_T, dev(R.ravel()), zt, alphas, betas)
    ZT = host(zt).reshape(2, -1)
    Tsolve = solvers.TSolver(d, p, n + p - 2)
    for k in range(2):
        ref = Tsolve(R[k])
        assert np.linalg.norm(ZT[k] - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,p,n", [(2, 2, 16), (2, 3, 21), (3, 2, 11)])
def test_multigrid_transfers_match_prolongator(d, p, n):
    s = cdl.Solver(d, p, n, max_batch=2, precond=cdl.CD_PC_MG, mg_m_min=3)
    m, mc = s.level_m(0), s.level_m(1)
    P = solvers.block_prolongator(d, m)
    assert P.shape == (d * m ** d, d * mc ** d)
    F = inputs.uniform_rhs(d, p, n, seed=1, nrhs=2)
    C = np.random.default_rng(2).uniform(-1, 1, (2, P.shape[1]))
    c = torch.zeros(2 * P.shape[1], dtype=torch.float64, device="cuda")
    s.cd_restrict(0, dev(F.ravel()), c)
    np.testing.assert_allclose(host(c).reshape(2, -1), F @ P.toarray(), rtol=1e-14, atol=1e-14)
    f = dev(F.ravel())
    s.cd_prolong(0, dev(C.ravel()), f)
    np.testing.assert_allclose(host(f).reshape(2, -1), F + C @ P.T.toarray(), rtol=1e-14, atol=1e-14)


def _solve(d, p, n, alphas, betas, B, seeds, **opts):
    s = cdl.Solver(d, p, n, max_batch=max(B, 1), **opts)
    Bv = inputs.uniform_rhs_seeds(d, p, n, seeds)
    x = torch.zeros(B * s.N, dtype=torch.float64, device="cuda")
    st, res = s.cd_solve(dev(Bv.ravel()), x, alphas, betas, check=False)
    return st, res, Bv, host(x).reshape(B, -1)


SOLVE_CASES = [
    # (d, p, n, precision, precond)
    (2, 2, 16, cdl.CD_PREC_FP64, cdl.CD_PC_NONE),
    (2, 3, 24, cdl.CD_PREC_FP64, cdl.CD_PC_FD_D),
    (2, 3, 24, cdl.CD_PREC_FP32_IR, cdl.CD_PC_FD_D),
    (2, 2, 30, cdl.CD_PREC_FP32_IR, cdl.CD_PC_MG),
    (2, 4, 20, cdl.CD_PREC_FP64, cdl.CD_PC_MG),
    (2, 2, 20, cdl.CD_PREC_FP32_IR, cdl.CD_PC_FD_T),
    (3, 2, 8, cdl.CD_PREC_FP32_IR, cdl.CD_PC_FD_D),
    (3, 3, 7, cdl.CD_PREC_FP64, cdl.CD_PC_MG),
    (3, 2, 9, cdl.CD_PREC_FP32_IR, cdl.CD_PC_MG),
    (2, 3, 24, cdl.CD_PREC_FP64, cdl.CD_PC_T_BAND),
    (3, 2, 8, cdl.CD_PREC_FP32_IR, cdl.CD_PC_T_BAND),
]


@pytest.mark.parametrize("d,p,n,prec,pc", SOLVE_CASES)
def test_solves_match_oracle(d, p, n, prec, pc):
    alphas = np.array([1.0, 1.0, 1.0])
    betas = np.array([0.1, 1.0, 10.0])
    st, res, Bv, X = _solve(d, p, n, alphas, betas, 3, [0, 1, 2], precision=prec, precond=pc,
                            rtol=1e-13, maxit=20000)
    assert st == cdl.CD_OK, res
    for k in range(3):
        A = oracle_matrix(d, p, n, alphas[k], betas[k])
        xs = solvers.direct_solve(A, Bv[k])
        assert np.linalg.norm(Bv[k] - A @ X[k]) <= 2e-13 * np.linalg.norm(Bv[k]), res[k]
        assert np.linalg.norm(X[k] - xs) <= 1e-9 * np.linalg.norm(xs), res[k]
        assert res[k]["relres"] <= 1e-13 * 1.01


@pytest.mark.parametrize("prec", [cdl.CD_PREC_FP32_IR, cdl.CD_PREC_FP64])
def test_3d_multigrid_solve_spanning_tiles(prec):
    """3D, m = 34: several (x_3, x_2) tiles and x_1 chunks of the streaming apply, fused
    smoother epilogues on every level; residual checked on sampled rows of the oracle."""
    d, p, n = 3, 2, 34
    st, res, Bv, X = _solve(d, p, n, [1.0, 1.0], [0.2, 5.0], 2, [3, 4], precision=prec,
                            precond=cdl.CD_PC_MG, rtol=1e-10)
    assert st == cdl.CD_OK, res
    rows = np.random.default_rng(1).integers(0, X.shape[1], 600)
    for k, beta in enumerate([0.2, 5.0]):
        ax, _ = kron_rows(d, p, n, 1.0, beta, X[k], rows)
        r = Bv[k][rows] - ax
        est = np.sqrt(X.shape[1] / rows.size * np.sum(r ** 2)) / np.linalg.norm(Bv[k])
        assert est <= 3e-10, est
        assert res[k]["relres"] <= 1.01e-10


def test_config1_plain_cg_fp64():
    """2D, p = 2, n = 16, alpha = beta = 1, one uniform RHS (seed 0), plain CG to 1e-10."""
    st, res, Bv, X = _solve(2, 2, 16, [1.0], [1.0], 1, [0], precision=cdl.CD_PREC_FP64,
                            precond=cdl.CD_PC_NONE, rtol=1e-10)
    assert st == cdl.CD_OK
    A = oracle_matrix(2, 2, 16, 1.0, 1.0)
    xs = solvers.direct_solve(A, Bv[0])
    relres = np.linalg.norm(Bv[0] - A @ X[0]) / np.linalg.norm(Bv[0])
    assert relres <= 1e-10
    # error bound from the residual: ||x - x*|| <= ||A^{-1}|| ||r||
    lam_min = np.linalg.eigvalsh(A.toarray()).min()
    assert np.linalg.norm(X[0] - xs) <= relres * np.linalg.norm(Bv[0]) / lam_min * 1.01
    # iteration count of CG: the oracle's CG on the same system needs the same count +- 1
    _, k_or, _ = solvers.cg(A, Bv[0], 1e-10)
    assert abs(res[0]["iters_inner"] - k_or) <= 1


def test_batch_results_identical_to_single_solves():
    """Per-solve reductions have a fixed order, so a solve gives bit-identical results alone
    and inside a batch with other parameters."""
    d, p, n = 2, 3, 20
    alphas, betas = np.array([1.0, 1.0, 1.0, 1.0]), np.array([1e-2, 1.0, 5.0, 1e2])
    seeds = [4, 5, 6, 7]
    for pc in (cdl.CD_PC_FD_D, cdl.CD_PC_MG):
        st, res, Bv, X = _solve(d, p, n, alphas, betas, 4, seeds, precond=pc)
        for k in range(4):
            st1, res1, _, X1 = _solve(d, p, n, alphas[k:k + 1], betas[k:k + 1], 1, seeds[k:k + 1],
                                      precond=pc)
            np.testing.assert_array_equal(X[k], X1[0])
            assert res[k]["iters_inner"] == res1[0]["iters_inner"]


def test_host_entry_point_and_error_statuses():
    d, p, n = 2, 2, 12
    s = cdl.Solver(d, p, n, max_batch=2)
    b = inputs.uniform_rhs(d, p, n, 9, 2).ravel().copy()
    x = np.zeros_like(b)
    st, res = s.cd_solve_host(b, x, [1.0, 1.0], [0.5, 2.0])
    assert st == cdl.CD_OK
    A = oracle_matrix(d, p, n, 1.0, 0.5)
    assert np.linalg.norm(b[:s.N] - A @ x[:s.N]) <= 1.01e-10 * np.linalg.norm(b[:s.N])
    # NaN right-hand side -> breakdown status, no exception, other solves unaffected
    b2 = b.copy()
    b2[3] = np.nan
    st, res = s.cd_solve_host(b2, x, [1.0, 1.0], [0.5, 2.0])
    assert res[0]["status"] == cdl.CD_BREAKDOWN and res[1]["status"] == cdl.CD_OK
    # maxit exhaustion -> NOT_CONVERGED
    s2 = cdl.Solver(d, p, n, max_batch=1, precision=cdl.CD_PREC_FP64, precond=cdl.CD_PC_NONE, maxit=3)
    st, res = s2.cd_solve_host(b[:s.N].copy(), x[:s.N].copy(), [1.0], [0.5])
    assert st == cdl.CD_NOT_CONVERGED and res[0]["status"] == cdl.CD_NOT_CONVERGED
    # invalid parameters and batch sizes
    with pytest.raises(cdl.CurlDivError):
        s.cd_apply(dev(b), dev(b), [1.0, -1.0], [1.0, 1.0])
    with pytest.raises(cdl.CurlDivError):
        s.cd_apply(dev(np.zeros(3 * s.N)), dev(np.zeros(3 * s.N)))


@pytest.mark.parametrize("p,n,beta", [(2, 16, 0.3), (3, 13, 50.0), (5, 12, 1e3), (4, 9, 1e-2)])
def test_mg_single_level_is_the_dense_inverse(p, n, beta):
    """2D multigrid on a mesh at or below its coarsest size (m <= 16): the V-cycle is the dense
    coarse solve alone, whose SPD inverse (2 m^2 >= 128 unknowns) is formed on the GPU by
    blocked Gauss-Jordan elimination (orders 242-512, full and ragged panels and tiles), so
    cd_precond(MG) r = A^{-1} r up to the conditioning."""
    s = cdl.Solver(2, p, n, max_batch=2, precond=cdl.CD_PC_MG)
    assert s.cd_levels() == 1
    R = inputs.uniform_rhs(2, p, n, seed=9, nrhs=2)
    z = torch.zeros(2 * s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_MG, dev(R.ravel()), z, [1.0, 1.0], [beta, 1.0 / beta])
    Z = host(z).reshape(2, -1)
    for k, bk in enumerate([beta, 1.0 / beta]):
        A = oracle_matrix(2, p, n, 1.0, bk)
        zs = solvers.direct_solve(A, R[k])
        assert np.linalg.norm(Z[k] - zs) <= 1e-10 * np.linalg.norm(zs), k
