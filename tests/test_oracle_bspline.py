"""Pins for oracle/bspline.py against textbook values and the properties listed in Section 3.1."""
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import bspline


def test_cardinal_textbook_values():
    # hat function, quadratic and cubic cardinal B-spline values at the knots (de Boor)
    assert bspline.cardinal(1, 1) == 1
    assert bspline.cardinal(2, 1) == F(1, 2) and bspline.cardinal(2, F(3, 2)) == F(3, 4)
    assert [bspline.cardinal(3, k) for k in range(5)] == [0, F(1, 6), F(2, 3), F(1, 6), 0]
    # quintic: 1/120, 26/120, 66/120, 26/120, 1/120
    assert [bspline.cardinal(5, k) for k in range(1, 6)] == [F(1, 120), F(26, 120), F(66, 120),
                                                           F(26, 120), F(1, 120)]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 7])
def test_cardinal_partition_symmetry_support(p):
    for t in [F(0), F(1, 3), F(2, 7), F(1, 2)]:
        assert sum(bspline.cardinal(p, t + k) for k in range(-1, p + 2)) == 1
    for t in [F(1, 5), F(3, 2), F(p, 3)]:
        assert bspline.cardinal(p, t) == bspline.cardinal(p, p + 1 - t)
    assert bspline.cardinal(p, -F(1, 3)) == 0 and bspline.cardinal(p, p + 1) == 0


@pytest.mark.parametrize("p", [2, 3, 5])
def test_cardinal_derivative_matches_difference_quotient(p):
    t = F(7, 5)
    h = F(1, 10 ** 8)
    fd = (bspline.cardinal(p, t + h) - bspline.cardinal(p, t - h)) / (2 * h)
    assert abs(float(fd - bspline.cardinal(p, t, 1))) < 1e-12


@pytest.mark.parametrize("p,n", [(1, 5), (2, 7), (3, 9), (5, 11)])
def test_cox_de_boor_properties(p, n):
    x = np.linspace(0, 1, 1001)
    N = bspline.basis(p, n, x)
    assert N.shape == (x.size, n + p)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-14)  # partition of unity
    assert N.min() >= -1e-15
    # only N_1 and N_{n+p} are nonzero at the ends (eq:spline-boundary)
    assert np.all(np.abs(N[0, 1:]) < 1e-15) and abs(N[0, 0] - 1) < 1e-15
    assert np.all(np.abs(N[-1, :-1]) < 1e-15) and abs(N[-1, -1] - 1) < 1e-15
    # local support [xi_i, xi_{i+p+1}]
    xi = bspline.knot_vector(p, n)
    for i in range(n + p):
        outside = (x < xi[i]) | (x > xi[i + p + 1])
        assert np.all(N[outside, i] == 0)


@pytest.mark.parametrize("p,n", [(1, 6), (2, 7), (3, 9), (4, 10)])
def test_central_bsplines_are_shifted_cardinal(p, n):
    x = np.linspace(0, 1, 777)
    N = bspline.basis(p, n, x)
    G = bspline.basis_deriv(p, n, x)
    for i in range(p + 1, n + 1):  # paper's 1-based central indices
        t = n * x - i + p + 1
        np.testing.assert_allclose(N[:, i - 1], bspline.cardinal_float(p, t), atol=1e-13)
        # derivative: n phi_p'(t) = n (phi_{p-1}(t) - phi_{p-1}(t-1))
        dphi = n * (bspline.cardinal_float(p - 1, t) - bspline.cardinal_float(p - 1, t - 1))
        off_knots = np.abs(t - np.round(t)) > 1e-6
        np.testing.assert_allclose(G[off_knots, i - 1], dphi[off_knots], atol=1e-11)


@pytest.mark.parametrize("p,n", [(1, 4), (2, 5), (3, 6), (6, 8)])
def test_derivative_formula_against_finite_differences(p, n):
    rng = np.random.default_rng(3)
    x = rng.uniform(0.01, 0.99, 200)
    xi = np.arange(n + 1) / n
    x = x[np.min(np.abs(x[:, None] - xi[None, :]), 1) > 1e-4]
    h = 1e-6
    fd = (bspline.basis(p, n, x + h) - bspline.basis(p, n, x - h)) / (2 * h)
    np.testing.assert_allclose(bspline.basis_deriv(p, n, x), fd, atol=2e-6 * n ** 2)
