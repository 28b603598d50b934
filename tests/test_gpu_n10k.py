"""Checks at the N = 10 000 workload (wiggly obstacle, omega = 30, 20 angles uniform in
(-pi/2, 0), tol 1e-12, all-FP64 build): outputs the oracle computes one by one, and
properties that hold at any size."""
import numpy as np
import pytest

from oracle import qp_dense as qd
from paper_1301_1247_gb300 import inputs

from gpu_util import dev, relerr, require_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n10k():
    hbs = require_lib()
    w = inputs.workload_wiggly_n10k()
    x, y, dx, dy = w["obstacle"].sample(w["N"])
    h = hbs.Handle(x, y, dx, dy, w["d"], w["omega"], 1e-12)
    return hbs, w, (x, y, dx, dy), h


def test_n10k_inverse_rows_against_oracle(n10k):
    """Rows of A (A^{-1} b), each evaluated densely by the oracle, reproduce b (Sec. 4)."""
    import torch
    hbs, w, geom, h = n10k
    n = w["N"]
    rng = np.random.default_rng(5)
    b = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    xb = torch.zeros((2, n), dtype=torch.complex128, device="cuda")
    h.apply_inverse(dev(b), xb, 2)
    x = xb.cpu().numpy()
    bd = qd.boundary(*geom)
    rows = np.concatenate([rng.integers(0, n, 10), [0, n - 1, n // 3]])
    a = qd.a_rows(bd, w["omega"], rows)
    for c in range(2):
        assert relerr(a @ x[c], b[c, rows]) < 1e-11


def test_n10k_flux_and_plain_path(n10k):
    """All 20 angles conserve flux to the N = 10^4 discretization floor, and the precomputed
    path agrees with the paper's per-phase path (q + 2M + 2l applies) to 1e-11."""
    hbs, w, geom, h = n10k
    th = np.asarray(w["thetas"]).ravel()
    fast = h.solve(th)
    plain = h.solve_plain(th)
    for i in range(len(th)):
        _, c1, d1, f1 = fast.bragg(i)
        _, c2, d2, f2 = plain.bragg(i)
        assert np.isfinite(f1) and f1 < 1e-6
        assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-11
    info = h.info()
    assert info["nb_residual"] < 1e-10 and info["pid_residual"] < 1e-10
