"""GPU tests of the serving runtime (iteration-level continuous batching, admission,
cancellation, timeouts)."""
import time

import numpy as np
import pytest

from gpu_helpers import oracle_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402
from paper_1805_10058_gb300 import inputs  # noqa: E402

SOLVE = dict(precision=cdl.CD_PREC_FP32_IR, precond=cdl.CD_PC_MG, rtol=1e-10)
# the server refines to half the requested tolerance (it returns x, not x + x_lo); a solve alone
# with that tolerance follows the same iterations
ALONE = dict(SOLVE, rtol=0.5e-10)


def _stream():
    rng = np.random.default_rng(7)
    shapes = [(2, 2, 20), (2, 3, 17), (3, 2, 6)]
    reqs = []
    for i in range(12):
        d, p, n = shapes[i % 3]
        nrhs = int(rng.integers(1, 4))
        betas = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), nrhs))
        b = inputs.uniform_rhs(d, p, n, seed=100 + i, nrhs=nrhs).ravel()
        reqs.append((d, p, n, np.ones(nrhs), betas, b))
    return reqs


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _stream()
    srv = cdl.Server(workers=3, max_batch=8, solve=SOLVE)
    tickets = [srv.submit(*r) for r in reqs]
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["mean_batch"] > 1.0  # same-shape solves shared the session steps
    for (d, p, n, al, be, b), (status, x, res) in zip(reqs, outs):
        assert status == cdl.CD_OK
        nrhs = len(al)
        # the same request alone, through cd_solve_host on a fresh solver
        s = cdl.Solver(d, p, n, max_batch=8, **ALONE)
        x1 = np.zeros_like(b)
        st1, res1 = s.cd_solve_host(b.copy(), x1, al, be)
        assert all(r["relres"] <= 1e-10 for r in res1)
        np.testing.assert_array_equal(x, x1)
        N = b.size // nrhs
        for k in range(nrhs):
            A = oracle_matrix(d, p, n, al[k], be[k])
            bk = b[k * N:(k + 1) * N]
            assert np.linalg.norm(bk - A @ x[k * N:(k + 1) * N]) <= 1.01e-10 * np.linalg.norm(bk)
            assert res[k]["iters_inner"] == res1[k]["iters_inner"]


def test_admission_under_a_small_budget_evicts_idle_solvers():
    reqs = _stream()[:6]
    # room for one of these small solvers at a time (~70 MB each by the admission estimate):
    # every new shape waits for or evicts the idle one
    srv = cdl.Server(workers=2, max_batch=4, hbm_budget=100 << 20, solve=SOLVE)
    tickets = [srv.submit(*r) for r in reqs]
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(o[0] == cdl.CD_OK for o in outs)
    assert st["bytes_in_use"] <= 100 << 20 and st["handles"] <= 1


def test_cancel_timeout_and_invalid_requests():
    d, p, n = 2, 2, 24
    b = inputs.uniform_rhs(d, p, n, seed=1).ravel()
    srv = cdl.Server(workers=1, max_batch=1, solve=SOLVE)
    tickets = [srv.submit(d, p, n, [1.0], [0.5], b) for _ in range(6)]
    assert srv.cancel(tickets[-1]) == cdl.CD_OK
    outs = [srv.wait(t) for t in tickets]
    assert outs[-1][0] == cdl.CD_CANCELLED
    assert all(o[0] == cdl.CD_OK for o in outs[:-1])
    with pytest.raises(cdl.CurlDivError):
        srv.submit(d, p, n, [1.0], [-1.0], b)
    with pytest.raises(cdl.CurlDivError):
        srv.submit(d, p, n, [1.0, 1.0], [1.0, 1.0], np.concatenate([b, b]))  # nrhs > max_batch
    srv.close()
    # a queue deadline: one worker, long queue, 1 ms limit -> some requests time out
    srv = cdl.Server(workers=1, max_batch=1, timeout_s=0.001, solve=SOLVE)
    tickets = [srv.submit(d, p, n, [1.0], [0.5], b) for _ in range(8)]
    outs = [srv.wait(t) for t in tickets]
    srv.close()
    sts = [o[0] for o in outs]
    assert cdl.CD_TIMEOUT in sts and all(s in (cdl.CD_OK, cdl.CD_TIMEOUT) for s in sts)


def test_requests_join_and_leave_between_krylov_chunks():
    """A request submitted while a long solve of the same shape is running is admitted into a
    free slot of the running session and finishes first (it does not wait for the long solve),
    and both results equal those of the same solves alone."""
    d, p, n = 2, 3, 96
    b_long = inputs.uniform_rhs(d, p, n, seed=41).ravel()
    b_short = inputs.uniform_rhs(d, p, n, seed=42).ravel()
    srv = cdl.Server(workers=1, max_batch=4, solve=SOLVE)
    t_long = srv.submit(d, p, n, [1.0], [1e4], b_long)  # many FP64-group iterations
    t0 = time.time()
    while srv.stats()["batches"] == 0 and time.time() - t0 < 60:  # the long solve is stepping
        time.sleep(0.002)
    assert srv.poll(t_long) is None
    t_short = srv.submit(d, p, n, [1.0], [1.0], b_short)  # a few dozen iterations
    out_short = srv.wait(t_short)
    assert srv.poll(t_long) is None  # still running when the short one is done
    out_long = srv.wait(t_long)
    srv.close()
    for (st, x, res), b, beta in ((out_short, b_short, 1.0), (out_long, b_long, 1e4)):
        assert st == cdl.CD_OK, res
        s = cdl.Solver(d, p, n, max_batch=4, **ALONE)
        x1 = np.zeros_like(b)
        st1, res1 = s.cd_solve_host(b.copy(), x1, [1.0], [beta])
        assert res1[0]["relres"] <= 1e-10
        np.testing.assert_array_equal(x, x1)
        assert res[0]["iters_inner"] == res1[0]["iters_inner"]
