"""The allocation-free 3D apply (cd_apply3d_static) against the oracle and against cd_apply.

cd_apply3d_static serves callers that may not allocate device memory (a host framework that
owns the whole device pool, or a latency-critical path that cannot take cudaMalloc's implicit
synchronisation).  Its work arrays live in a fixed static device array shared by all calls,
so this test checks two calls in a row (the second sees the first call's leftovers) against
the oracle's assembled A w and against the existing entry point, within the FP64 apply
tolerance of the parity tests, and checks that a call leaves the device's free memory
unchanged.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_helpers import abs_matvec_bound, oracle_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402


CASES = [(3, 6, 1.0, 0.02, 2, 21), (2, 9, 0.7, 30.0, 3, 22)]  # (p, n, alpha, beta, nrhs, seed)


def test_static_apply_matches_oracle_and_cd_apply_twice():
    for p, n, alpha, beta, nrhs, seed in CASES:
        W = inputs.uniform_rhs(3, p, n, seed=seed, nrhs=nrhs)
        w = torch.as_tensor(W.ravel(), device="cuda")
        s = cdl.Solver(3, p, n, alpha, beta, max_batch=nrhs)
        y_ref = torch.zeros_like(w)
        s.cd_apply(w, y_ref)
        A = oracle_matrix(3, p, n, alpha, beta)
        Yr = y_ref.cpu().numpy().reshape(nrhs, -1)
        for call in range(2):
            y = torch.full_like(w, float("nan"))
            cdl.cd_apply3d_static(p, n, alpha, beta, w, y)
            torch.cuda.synchronize()
            Y = y.cpu().numpy().reshape(nrhs, -1)
            for k in range(nrhs):
                bound = abs_matvec_bound(A, W[k])
                assert np.all(np.abs(Y[k] - A @ W[k]) <= 1e-13 * bound), (p, n, call, k)
                assert np.all(np.abs(Y[k] - Yr[k]) <= 1e-13 * bound), (p, n, call, k)


def test_static_apply_allocates_no_device_memory():
    p, n, nrhs = 3, 20, 2
    W = inputs.uniform_rhs(3, p, n, seed=5, nrhs=nrhs)
    w = torch.as_tensor(W.ravel(), device="cuda")
    y = torch.zeros_like(w)
    cdl.cd_apply3d_static(p, n, 1.0, 0.5, w, y)  # first call: address look-up, module loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for _ in range(3):
        cdl.cd_apply3d_static(p, n, 1.0, 0.5, w, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == torch_bytes0


def test_static_apply_rejects_oversized_requests():
    p, n = 3, 70  # m = 71: one right-hand side needs more than the 48 MiB scratch
    N = cdl.cd_dofs(3, p, n)
    w = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(w)
    st = cdl.cd_apply3d_static(p, n, 1.0, 1.0, w, y, check=False)
    assert st == cdl.CD_EINVAL
    assert b"48 MiB" in cdl.load().cd_last_error()
