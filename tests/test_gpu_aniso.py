"""Anisotropic meshes (Section 5: n_l = nu_l n intervals along x_l) through the C-ABI
(cd_create_aniso): the operator apply against the oracle's matrix assembled on the same mesh,
solves against sparse LU, the FD-D preconditioner against the block-diagonal solve, and the
argument checks.  Sizes span several thread blocks with ragged ends in every direction."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_helpers import abs_matvec_bound
from oracle import assemble, solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


APPLY = [(2, 1, (7, 19)), (2, 2, (5, 33)), (2, 3, (40, 9)), (2, 5, (11, 6)),
         (3, 1, (4, 9, 5)), (3, 2, (3, 5, 4)), (3, 3, (7, 4, 6)), (3, 4, (5, 3, 8))]


@pytest.mark.parametrize("d,p,ns", APPLY)
def test_aniso_apply_matches_oracle(d, p, ns):
    alphas, betas = np.array([1.0, 0.3, 2.0]), np.array([0.05, 4.0, 2.0])
    s = cdl.Solver(d, p, ns, max_batch=3, precond=cdl.CD_PC_NONE)
    N = s.N
    assert N == assemble.dofs(d, p, ns)
    W = inputs.uniform_rhs(d, p, ns, seed=17, nrhs=3)
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    s.cd_apply(dev(W.ravel()), y, alphas, betas)
    Y = host(y).reshape(3, N)
    y32 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    s.cd_apply_f32(dev(W.ravel(), torch.float32), y32, alphas, betas)
    Y32 = host(y32).reshape(3, N)
    for k in range(3):
        A = assemble.galerkin_kron(d, p, ns, alphas[k], betas[k])
        assert np.all(np.abs(Y[k] - A @ W[k]) <= 1e-13 * abs_matvec_bound(A, W[k]) + 1e-300), k
        w32 = W[k].astype(np.float32).astype(np.float64)
        assert np.all(np.abs(Y32[k] - A @ w32) <= 3e-5 * abs_matvec_bound(A, w32) + 1e-30), k


@pytest.mark.parametrize("d,p,ns,prec,pc", [
    (2, 2, (12, 30), cdl.CD_PREC_FP64, cdl.CD_PC_NONE),
    (2, 3, (24, 8), cdl.CD_PREC_FP64, cdl.CD_PC_FD_D),
    (2, 3, (10, 27), cdl.CD_PREC_FP32_IR, cdl.CD_PC_FD_D),
    (3, 2, (4, 8, 6), cdl.CD_PREC_FP32_IR, cdl.CD_PC_FD_D),
    (3, 3, (6, 4, 5), cdl.CD_PREC_FP64, cdl.CD_PC_FD_D),
])
def test_aniso_solves_match_sparse_lu(d, p, ns, prec, pc):
    alphas, betas = np.array([1.0, 1.0, 1.0]), np.array([0.1, 1.0, 1e3])
    s = cdl.Solver(d, p, ns, max_batch=3, precision=prec, precond=pc, rtol=1e-12, maxit=20000)
    Bv = np.stack([inputs.uniform_rhs(d, p, ns, seed=sd)[0] for sd in (3, 4, 5)])
    x = torch.zeros(3 * s.N, dtype=torch.float64, device="cuda")
    st, res = s.cd_solve(dev(Bv.ravel()), x, alphas, betas, check=False)
    assert st == cdl.CD_OK, res
    X = host(x).reshape(3, -1)
    for k in range(3):
        A = assemble.galerkin_kron(d, p, ns, alphas[k], betas[k])
        xs = solvers.direct_solve(A, Bv[k])
        assert np.linalg.norm(Bv[k] - A @ X[k]) <= 2e-12 * np.linalg.norm(Bv[k]), res[k]
        assert np.linalg.norm(X[k] - xs) <= 1e-8 * np.linalg.norm(xs), res[k]


@pytest.mark.parametrize("d,p,ns", [(2, 3, (9, 21)), (3, 2, (5, 3, 7))])
def test_aniso_fd_d_is_the_block_diagonal_inverse(d, p, ns):
    """cd_precond(FD_D) = D^{-1} r with D = blockdiag(A^(c,c)) of the anisotropic matrix (FP64),
    and at alpha = beta (A = D) the preconditioned CG converges in one iteration."""
    alpha, beta = 1.0, 0.2
    s = cdl.Solver(d, p, ns, max_batch=1, precision=cdl.CD_PREC_FP64, precond=cdl.CD_PC_FD_D,
                   rtol=1e-12)
    r = inputs.uniform_rhs(d, p, ns, seed=8)[0]
    z = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    s.cd_precond(cdl.CD_PC_FD_D, dev(r), z, [alpha], [beta])
    D = assemble.block_diagonal(assemble.galerkin_kron(d, p, ns, alpha, beta), d).tocsc()
    zr = spla.spsolve(D, r)
    assert np.linalg.norm(host(z) - zr) <= 1e-10 * np.linalg.norm(zr)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    st, res = s.cd_solve(dev(r), x, [0.7], [0.7])
    assert st == cdl.CD_OK and res[0]["iters_inner"] <= 2, res


def test_aniso_argument_checks():
    with pytest.raises(cdl.CurlDivError):
        cdl.Solver(2, 2, (5, 9), precond=cdl.CD_PC_MG)
    with pytest.raises(cdl.CurlDivError):
        cdl.Solver(2, 2, (5, 0))
    s = cdl.Solver(2, 2, (5, 9), precond=cdl.CD_PC_NONE)
    assert s.cd_levels() == 0
    r = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    with pytest.raises(cdl.CurlDivError):
        s.cd_precond(cdl.CD_PC_FD_D, r, torch.zeros_like(r))
