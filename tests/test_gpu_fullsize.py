"""Checks at the benchmark's full size (N = 100 000, omega = 60, 1000 angles), on outputs the
oracle can compute one by one and on properties that hold at any size."""
import math

import numpy as np
import pytest

from oracle import qp_dense as qd
from paper_1301_1247_gb300 import inputs

from gpu_util import dev, relerr, require_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    hbs = require_lib()
    w = inputs.workload_complicated_n100k()
    x, y, dx, dy = w["obstacle"].sample(w["N"])
    h = hbs.Handle(x, y, dx, dy, w["d"], w["omega"], 1e-12, hbs.default_options(precision=1))
    return hbs, w, (x, y, dx, dy), h


def test_fullsize_inverse_rows_against_oracle(full):
    """x = A^{-1} b with the compressed inverse; rows of A x evaluated one by one by the oracle
    (dense definition of each row) reproduce b."""
    import torch
    hbs, w, geom, h = full
    n = w["N"]
    rng = np.random.default_rng(11)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xb = torch.zeros((1, n), dtype=torch.complex128, device="cuda")
    h.apply_inverse(dev(b[None, :]), xb, 1)
    x = xb.cpu().numpy()[0]
    bd = qd.boundary(*geom)
    rows = np.concatenate([rng.integers(0, n, 12), [0, 1, n - 1, n // 2]])
    ax = qd.a_rows(bd, w["omega"], rows) @ x
    assert relerr(ax, b[rows]) < 1e-10


def test_fullsize_flux_and_fp64_plain_path(full):
    """All 1000 angles conserve flux to the discretization floor; one Bloch group agrees with
    the all-FP64 plain per-phase path (q + 2M + 2l applies) to 1e-10."""
    hbs, w, geom, h = full
    th = np.asarray(w["thetas"]).ravel()
    res = h.solve(th)
    flux = np.array([res.bragg(i)[3] for i in range(len(th))])
    assert np.all(np.isfinite(flux)) and flux.max() < 1e-8
    h64 = hbs.Handle(*geom, w["d"], w["omega"], 1e-12)
    group = np.asarray(w["thetas"])[3]
    ref = h64.solve_plain(group)
    fast = h.solve(group)
    for i in range(len(group)):
        _, c1, d1, _ = fast.bragg(i)
        _, c2, d2, _ = ref.bragg(i)
        assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-10


def test_fullsize_compressions_hold_off_sample(full):
    """The neighbour ID (skeleton chosen among every stride-th node) and the periodizer IDs
    (found on a point subsample) reconstruct their matrices on nodes they never saw."""
    hbs, w, geom, h = full
    info = h.info()
    assert 0 < info["nb_rank"] < info["nb_proxies"]
    assert info["nb_residual"] < 1e-10
    assert info["pid_residual"] < 1e-10
