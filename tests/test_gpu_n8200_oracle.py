"""Bragg amplitudes at N = 8200 against the dense FP64 oracle (tests/golden/dense_n8200.txt,
written by make_dense_n8200.py from oracle/ alone), at omega = 60 and omega = 30.

At this size the production paths that the small parity cases never reach all run: the
neighbour ID picks its skeleton among every third node and fits the other rows by least
squares (Sec. 3.2, Def. 3.1), the periodizer IDs work on a point subsample, and the leaf
level holds 256 nodes, so the one-CTA-per-node QR and Gauss-Jordan kernels run beside the
persistent ones (Sec. 4).  Each case has two groups of three angles sharing a Bloch phase and
one angle exactly at a Wood's anomaly (Sec. 2.4).  The library's contour, sampling and
per-phase contour choice must equal the oracle's own readings."""
import importlib.util
import os

import numpy as np
import pytest

from paper_1301_1247_gb300 import inputs

from gpu_util import assert_library_readings, require_lib

pytestmark = pytest.mark.gpu

_HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_dense_n8200", os.path.join(_HERE, "golden", "make_dense_n8200.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)

CASES = {name: (make, omega) for name, make, omega, _, _ in golden.CASES}


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("name", ["complicated_w60", "wiggly_w30"])
def test_n8200_bragg_amplitudes_match_dense_oracle(name, precision):
    hbs = require_lib()
    ref = golden.load()[name]
    make, omega = CASES[name]
    x, y, dx, dy = make().sample(golden.N)
    assert ref["n"] == golden.N and ref["omega"] == omega
    # the regenerated geometry is the one the oracle solved (to the last few bits)
    assert abs(float(np.sum(x)) - ref["sum_x"]) < 1e-9 and abs(float(np.sum(y)) - ref["sum_y"]) < 1e-9
    h = hbs.Handle(x, y, dx, dy, golden.D, omega, 1e-12, hbs.default_options(precision=precision))
    info = h.info()
    assert_library_readings(info, x, y, omega, golden.D)
    assert info["levels"] >= 8  # 256 leaves: levels beyond 128 nodes run the one-CTA kernels
    assert info["nb_residual"] < 1e-11 and info["pid_residual"] < 1e-11
    thetas = np.array([a["theta"] for a in ref["angles"]])
    res = h.solve(thetas)
    worst = 0.0
    for i, a in enumerate(ref["angles"]):
        nw, t0 = res.angle_info(i)
        if a["margin"] > 1e-3:
            assert abs(t0 - a["t0"]) <= 1e-12 * max(1.0, a["t0"]), (i, t0, a["t0"])
            assert nw == a["nw"], (i, nw, a["nw"])
        orders, c, d, flux = res.bragg(i)
        assert list(orders) == a["orders"], i
        want = np.array([a["c"][n] for n in a["orders"]] + [a["d"][n] for n in a["orders"]])
        got = np.concatenate([c, d])
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        # every amplitude, not only the vector norm
        assert np.max(np.abs(got - want)) <= 1e-10 * np.linalg.norm(want), i
        assert err <= 1e-10, (i, err)
        assert abs(flux - a["flux"]) < 1e-9, (i, flux, a["flux"])
        worst = max(worst, err)
    # the Wood's angle (last) is at an exact anomaly and uses the shifted contour
    assert ref["angles"][-1]["nw"] >= 1 and res.angle_info(len(thetas) - 1)[0] >= 1
    print(f"{name} precision={precision}: worst relative Bragg error vs dense oracle {worst:.2e}")
