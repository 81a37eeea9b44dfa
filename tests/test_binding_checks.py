"""Host-side argument checks of the Python binding (no GPU): a vector pair must hold the same
whole number (>= 1) of right-hand sides, device arguments must be contiguous CUDA tensors of the
right type, and per-solve parameters broadcast to the number of right-hand sides or fail.  A
short output vector would otherwise let the kernels write past its end."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1805_10058_gb300 import curldiv as cdl  # noqa: E402


def test_rhs_count_must_match_and_be_whole():
    N = 10
    assert cdl._nrhs(N, np.zeros(30), np.zeros(30), "x") == 3
    assert cdl._nrhs(N, torch.zeros(20), torch.zeros(20), "x") == 2
    for na, nb in ((0, 0), (5, 5), (25, 25), (30, 20), (20, 30)):
        with pytest.raises(ValueError):
            cdl._nrhs(N, np.zeros(na), np.zeros(nb), "x")


def test_device_arguments_must_be_contiguous_cuda_tensors_of_the_right_type():
    with pytest.raises(TypeError):
        cdl._dev(torch.zeros(4, dtype=torch.float64), "float64")  # host tensor
    with pytest.raises(TypeError):
        cdl._dev(np.zeros(4), "float64")  # not a tensor


def test_parameters_broadcast_to_the_rhs_count():
    (a, b), pa, pb = cdl._params(3, 1.0, [1e-6, 1.0, 1e6])
    np.testing.assert_array_equal(a, [1.0, 1.0, 1.0])
    np.testing.assert_array_equal(b, [1e-6, 1.0, 1e6])
    assert pa is not None and pb is not None
    (a, b), pa, pb = cdl._params(2, None, None)
    assert a is None and b is None and pa is None and pb is None
    with pytest.raises(ValueError):
        cdl._params(3, [1.0, 2.0], None)
