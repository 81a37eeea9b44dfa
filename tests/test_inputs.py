"""The seeded input generators shared by the oracle side and the GPU side: reproducible,
of the library layout, and with the distributions the workloads state."""
import numpy as np

from paper_1805_10058_gb300 import inputs


def test_uniform_rhs_is_seeded_and_in_range():
    a = inputs.uniform_rhs(2, 3, 20, seed=4, nrhs=3)
    assert a.shape == (3, 2 * 21 ** 2)
    np.testing.assert_array_equal(a, inputs.uniform_rhs(2, 3, 20, seed=4, nrhs=3))
    assert not np.array_equal(a, inputs.uniform_rhs(2, 3, 20, seed=5, nrhs=3))
    assert a.min() >= -1.0 and a.max() <= 1.0
    assert abs(a.mean()) < 0.05 and abs(a.var() - 1.0 / 3.0) < 0.02  # uniform[-1, 1]
    b = inputs.uniform_rhs_seeds(3, 2, 6, [0, 7])
    assert b.shape == (2, 3 * 6 ** 3)
    np.testing.assert_array_equal(b[1], inputs.uniform_rhs(3, 2, 6, seed=7)[0])


def test_sweep_cases_cover_the_2d_sweep():
    cases = inputs.sweep_cases()
    assert len(cases) == 3 * 5 * 8 == 120
    assert {c[1] for c in cases} == {2, 3, 4}
    assert {c[4] for c in cases} == {1e-6, 1e-3, 1.0, 1e3, 1e6}
    assert all(c[0] == 2 and c[2] == 256 and c[3] == 1.0 for c in cases)


def test_loguniform_parameters():
    v = inputs.loguniform_params(seed=1, count=4000)
    assert v.min() >= 1e-6 and v.max() <= 1e6
    lg = np.log10(v)
    assert abs(lg.mean()) < 0.3 and abs(lg.std() - 12 / np.sqrt(12)) < 0.2  # uniform in log
    np.testing.assert_array_equal(v, inputs.loguniform_params(seed=1, count=4000))


def test_serving_stream_statistics():
    reqs = inputs.serving_stream(seed=0, count=2000, rate=200.0)
    assert len(reqs) == 2000
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 200.0) < 15.0  # Poisson arrivals, mean rate 200/s
    two = [r for r in reqs if r["d"] == 2]
    assert abs(len(two) / len(reqs) - 0.6) < 0.04  # 60% 2D, 40% 3D
    assert all(32 <= r["n"] <= 256 for r in two)
    assert all(16 <= r["n"] <= 96 for r in reqs if r["d"] == 3)
    assert {r["p"] for r in reqs} == {1, 2, 3, 4, 5}
    assert {r["nrhs"] for r in reqs} == {1, 2, 3, 4}
    assert all(1e-6 <= r["beta"] <= 1e6 and r["alpha"] == 1.0 for r in reqs)
    assert reqs == inputs.serving_stream(seed=0, count=2000, rate=200.0)
