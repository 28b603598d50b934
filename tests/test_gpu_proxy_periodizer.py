"""The second periodizer on the GPU (hbs_solve_proxy: proxy points and wall discrepancies)
against its dense oracle (oracle/proxy_periodizer.py), against the dense Fourier-wall oracle
(Secs. 2.2-2.4), and against the library's own Fourier-wall solve: two periodizations of one
continuum problem agree to the FP64 bar, including exact Wood's anomalies, where only the
Fourier-wall scheme needs its shifted contour and extra rows."""
import importlib.util
import math
import os

import numpy as np
import pytest

from oracle import proxy_periodizer as pp
from oracle import qp_dense as qd
from oracle import readings as rd
from paper_1301_1247_gb300 import inputs

from gpu_util import relerr, require_lib

pytestmark = pytest.mark.gpu


def test_proxy_periodizer_star_matches_both_oracles_and_the_fourier_wall_solve():
    hbs = require_lib()
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
    omega = 10.0
    thetas = np.concatenate([[-math.pi / 5, -1.0, -2.5, -math.acos(1.0 - 2.0 * math.pi / omega)],
                             inputs.bloch_grouped_angles(4, omega, 1.0, 1, 3).ravel()])
    h = hbs.Handle(x, y, dx, dy, 1.0, omega, 1e-12)
    y0 = h.info()["y0"]
    rp_ = h.solve_proxy(thetas)
    rf_ = h.solve(thetas)
    blocks = qd.obstacle_blocks(x, y, dx, dy, omega, 1.0)
    for i, th in enumerate(thetas):
        orders, c, d, flux = rp_.bragg(i)
        got = np.concatenate([c, d])
        sp = pp.solve(x, y, dx, dy, omega, 1.0, th, blocks=blocks)
        cp, dp = pp.bragg_at(sp, omega, 1.0, th, y0)
        assert list(orders) == list(sp.orders)
        assert relerr(got, np.concatenate([cp, dp])) < 1e-10, (th, "proxy oracle")
        sf = qd.dense_solve(x, y, dx, dy, omega, 1.0, th, rd.options(x, y, omega, 1.0, th), blocks)
        assert relerr(got, qd.bragg_vector(sf)) < 1e-10, (th, "Fourier-wall oracle")
        _, c2, d2, _ = rf_.bragg(i)
        assert relerr(got, np.concatenate([c2, d2])) < 1e-10, (th, "Fourier-wall solve")
        assert abs(flux - sf.flux_error) < 1e-8
        assert rp_.angle_info(i) == (0, 0.0)


def test_proxy_periodizer_n8200_matches_the_dense_oracle():
    """omega = 30, N = 8200 (neighbour ID on candidates, the one-CTA leaf kernels): the proxy
    periodizer's amplitudes against the dense Fourier-wall oracle's stored values."""
    hbs = require_lib()
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_dense_n8200", os.path.join(here, "golden", "make_dense_n8200.py"))
    golden = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(golden)
    ref = golden.load()["wiggly_w30"]
    x, y, dx, dy = inputs.wiggly(0, 0.35, 20, 0.03).sample(golden.N)
    h = hbs.Handle(x, y, dx, dy, golden.D, 30.0, 1e-12)
    thetas = np.array([a["theta"] for a in ref["angles"]])
    res = h.solve_proxy(thetas)
    for i, a in enumerate(ref["angles"]):
        orders, c, d, _ = res.bragg(i)
        assert list(orders) == a["orders"]
        want = np.array([a["c"][n] for n in a["orders"]] + [a["d"][n] for n in a["orders"]])
        assert relerr(np.concatenate([c, d]), want) < 1e-10, i
