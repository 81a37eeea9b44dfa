"""The allocation-free 3D apply (cd_apply3d_static) against the handle-based cd_apply.

cd_apply3d_static serves callers that may not allocate device memory (a host framework that
owns the whole device pool, or a latency-critical path that cannot take cudaMalloc's implicit
synchronisation).  Its work arrays live in a fixed static device array shared by all calls,
so this test checks two calls in a row (the second sees the first call's leftovers) against
the existing entry point, within the FP64 apply tolerance of the parity tests.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_helpers import abs_matvec_bound, oracle_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402


def test_static_apply_matches_cd_apply_twice():
    cases = [(3, 6, 1.0, 0.02, 2, 21), (2, 9, 0.7, 30.0, 3, 22)]  # (p, n, alpha, beta, nrhs, seed)
    for p, n, alpha, beta, nrhs, seed in cases:
        W = inputs.uniform_rhs(3, p, n, seed=seed, nrhs=nrhs)
        w = torch.as_tensor(W.ravel(), device="cuda")
        s = cdl.Solver(3, p, n, alpha, beta, max_batch=nrhs)
        y_ref = torch.zeros_like(w)
        s.cd_apply(w, y_ref)
        y = torch.full_like(w, float("nan"))
        cdl.cd_apply3d_static(p, n, alpha, beta, w, y)
        torch.cuda.synchronize()
        Y, Yr = y.cpu().numpy().reshape(nrhs, -1), y_ref.cpu().numpy().reshape(nrhs, -1)
        A = oracle_matrix(3, p, n, alpha, beta)
        for k in range(nrhs):
            bound = abs_matvec_bound(A, W[k])
            assert np.all(np.abs(Y[k] - Yr[k]) <= 1e-13 * bound), (p, n, k)


def test_static_apply_rejects_oversized_requests():
    p, n = 3, 70  # m = 71: one right-hand side needs more than the 48 MiB scratch
    N = cdl.cd_dofs(3, p, n)
    w = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(w)
    st = cdl.cd_apply3d_static(p, n, 1.0, 1.0, w, y, check=False)
    assert st == cdl.CD_EINVAL
    assert b"48 MiB" in cdl.load().cd_last_error()
