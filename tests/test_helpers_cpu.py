"""The row-by-row evaluation used by the full-size GPU checks agrees with the oracle's
sparse matrix (so the sampled full-size parity compares against the oracle)."""
import numpy as np
import pytest

from gpu_helpers import kron_rows, oracle_matrix


@pytest.mark.parametrize("d,p,n", [(2, 2, 7), (2, 4, 9), (3, 2, 4), (3, 3, 5)])
def test_kron_rows_equals_oracle_matvec(d, p, n):
    A = oracle_matrix(d, p, n, 1.0, 0.03)
    w = np.random.default_rng(0).uniform(-1, 1, A.shape[0])
    rows = np.arange(A.shape[0])
    out, bound = kron_rows(d, p, n, 1.0, 0.03, w, rows)
    np.testing.assert_allclose(out, A @ w, rtol=0, atol=1e-14 * bound.max())
    assert np.all(bound >= np.abs(out) - 1e-12)
