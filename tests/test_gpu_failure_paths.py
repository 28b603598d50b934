"""Error paths in the forms allowed on a shared GPU: nothing faults, traps or hangs.

* A bounded device wait runs out: the library's grid barrier with one CTA that never
  arrives gives up after a short limit, the call returns HBS_ERR_TIMEOUT, and the context
  stays usable.
* A rank overflow: an injected rank cap makes the interpolative decompositions stop short
  of the tolerance, and the calls return HBS_ERR_RANK.
* A singular block: the per-node inversion (Sec. 4) meets an exactly zero pivot and returns
  HBS_WARN_ILLCOND (a guided mode makes the Schur system singular in the same way, Remark 2.1).
* A device allocation failure, injected on the host: HBS_ERR_OOM, then normal service.
"""
import math

import numpy as np
import pytest

from oracle import qp_dense as qd
from oracle import readings as rd
from paper_1301_1247_gb300 import inputs

from gpu_util import dev, relerr, require_lib

pytestmark = pytest.mark.gpu


def _star_solve_matches_oracle(hbs):
    """A normal build and solve after a failure still agrees with the dense oracle."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
    th = -math.pi / 5
    h = hbs.Handle(x, y, dx, dy, 1.0, 10.0, 1e-12)
    _, c, d, _ = h.solve([th]).bragg(0)
    sol = qd.dense_solve(x, y, dx, dy, 10.0, 1.0, th, rd.options(x, y, 10.0, 1.0, th))
    assert relerr(np.concatenate([c, d]), qd.bragg_vector(sol)) < 1e-10


def test_barrier_wait_gives_up_and_context_survives():
    hbs = require_lib()
    st, passed = hbs.barrier_selftest(8, -1, 0.5)
    assert st == hbs.HBS_OK and passed == 8
    st, passed = hbs.barrier_selftest(8, 3, 0.05)
    assert st == hbs.HBS_ERR_TIMEOUT and passed == 0
    assert b"gave up" in hbs.lib().hbs_last_error()
    st, passed = hbs.barrier_selftest(16, -1, 0.5)
    assert st == hbs.HBS_OK and passed == 16
    _star_solve_matches_oracle(hbs)


def test_rank_cap_gives_err_rank():
    import torch
    hbs = require_lib()
    rng = np.random.default_rng(3)
    m, n, r = 80, 6000, 50
    mt = (rng.standard_normal((m, r)) * 10.0 ** (-np.arange(r) / 4.0)) @ rng.standard_normal((r, n))
    mt = mt.astype(np.complex128)
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    t = torch.zeros(m * n, dtype=torch.complex128, device="cuda")
    hbs.fault_inject(hbs.INJECT_RANK_CAP, 8)
    try:
        with pytest.raises(hbs.HbsError) as e:
            hbs.row_id(dev(np.asfortranarray(mt).ravel(order="F")), m, n, 1e-12, perm, t)
        assert e.value.status == hbs.HBS_ERR_RANK
        x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
        with pytest.raises(hbs.HbsError) as e:
            hbs.Handle(x, y, dx, dy, 1.0, 10.0, 1e-12)
        assert e.value.status == hbs.HBS_ERR_RANK
    finally:
        hbs.fault_inject(hbs.INJECT_CLEAR)
    k = hbs.row_id(dev(np.asfortranarray(mt).ravel(order="F")), m, n, 1e-12, perm, t)
    assert 30 < k <= r
    _star_solve_matches_oracle(hbs)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("count,n", [(3, 150), (200, 40), (5, 512), (2, 1000)])
def test_batched_inverse_matches_numpy_and_flags_singular_blocks(count, n, precision, monkeypatch):
    """The per-node inversion kernels (multi-CTA for few blocks, one CTA per block for many)
    against numpy's inverse; then one block with a zero column gives HBS_WARN_ILLCOND.  With
    the autotuner exploring, consecutive calls of one shape run every multi-CTA variant in
    turn: the persistent Gauss-Jordan and the blocked one on clusters of 1, 2, 4 and 8 CTAs."""
    hbs = require_lib()
    monkeypatch.setenv("HBS_AUTOTUNE", "1")
    monkeypatch.setenv("HBS_TUNE_FILE", "")
    rng = np.random.default_rng(count + n)
    a = rng.standard_normal((count, n, n)) + 1j * rng.standard_normal((count, n, n))
    a += 4 * np.sqrt(n) * np.eye(n)[None]  # well conditioned, as the leaf blocks of A are
    ref = np.linalg.inv(a)
    for _ in range(5):
        buf = dev(np.ascontiguousarray(np.transpose(a, (0, 2, 1))).ravel())  # column-major blocks
        assert hbs.batched_inverse(buf, n, count, precision) == hbs.HBS_OK
        got = np.transpose(buf.cpu().numpy().reshape(count, n, n), (0, 2, 1))
        assert relerr(got, ref) < (1e-13 if precision == 0 else 1e-12)
    a[count // 2][:, n // 3] = 0.0
    a2 = np.concatenate([a, a])  # twice the blocks: a shape class of its own, explored afresh
    for _ in range(5):
        buf = dev(np.ascontiguousarray(np.transpose(a2, (0, 2, 1))).ravel())
        assert hbs.batched_inverse(buf, n, 2 * count, precision) == hbs.HBS_WARN_ILLCOND
        assert b"singular" in hbs.lib().hbs_last_error()


def test_injected_allocation_failure_gives_oom_then_normal_service():
    hbs = require_lib()
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
    for after in (0, 7, 60):
        hbs.fault_inject(hbs.INJECT_ALLOC_FAILURE, after)
        try:
            with pytest.raises(hbs.HbsError) as e:
                hbs.Handle(x, y, dx, dy, 1.0, 10.0, 1e-12).solve([-0.7])
            assert e.value.status == hbs.HBS_ERR_OOM, after
        finally:
            hbs.fault_inject(hbs.INJECT_CLEAR)
    _star_solve_matches_oracle(hbs)
