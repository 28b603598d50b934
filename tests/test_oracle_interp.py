"""Pins for the oracle's interpolative decomposition (Def. 3.1) against the SVD."""
import numpy as np
import pytest

from oracle import interp, qp_dense as qd
from paper_1301_1247_gb300 import inputs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_id_exact_on_low_rank(seed):
    rng = np.random.default_rng(seed)
    m, n, r = 60, 45, 11
    a = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ \
        (rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
    j, p, k = interp.row_id(a, 1e-12)
    assert k == r
    assert np.allclose(p[j, :], np.eye(k))
    assert np.linalg.norm(a - p @ a[j, :]) < 1e-11 * np.linalg.norm(a)


def test_id_error_bounded_by_svd_on_kernel_block():
    """For a well-separated Helmholtz interaction block the ID error is within
    sqrt(1 + k (m - k)) sigma_{k+1} (times a small factor) and k is at least the SVD rank."""
    omega = 20.0
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
    bd = qd.boundary(x, y, dx, dy)
    rows = np.arange(0, 40)
    cols = np.arange(150, 300)
    blk = qd.combined(bd.x[rows, None], bd.y[rows, None], bd.x[None, cols], bd.y[None, cols],
                      bd.nx[None, cols], bd.ny[None, cols], omega) * bd.w[None, cols]
    tol = 1e-10
    j, p, k = interp.row_id(blk, tol)
    s = np.linalg.svd(blk, compute_uv=False)
    svd_rank = int(np.sum(s > tol * s[0]))
    assert k >= svd_rank - 1
    err = np.linalg.norm(blk - p @ blk[j, :], 2)
    bound = np.sqrt(1 + k * (len(rows) - k)) * (s[k] if k < len(s) else 0.0)
    assert err <= 10 * bound + 1e-14 * s[0]
    assert err < 1e-8 * s[0]
