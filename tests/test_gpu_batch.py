"""Many gratings built at once (hbs_build_batch): every level of every tree in the same
launches.  Each solver of the batch must solve like the same solver built alone, and the
smallest one like the dense oracle."""
import math

import numpy as np
import pytest

from oracle import qp_dense as qd
from paper_1301_1247_gb300 import inputs

from gpu_util import assert_library_readings, oracle_options_checked, relerr, require_lib

pytestmark = pytest.mark.gpu


def test_batch_build_matches_individual_builds():
    hbs = require_lib()
    specs = [(inputs.star(0.3, 0.3, 5), 400, 10.0), (inputs.wiggly(1, 0.35, 20, 0.03), 1500, 25.0),
             (inputs.wiggly(2, 0.3, 40, 0.04), 5000, 40.0), (inputs.star(0.25, 0.2, 3), 800, 5.0)]
    geoms = [obs.sample(n) for obs, n, _ in specs]
    omegas = [om for _, _, om in specs]
    batch = hbs.build_batch(geoms, omegas, 1.0, 1e-12)
    th = inputs.uniform_angles(4, 8, -math.pi / 2 + 0.05, -0.1)
    for i, (g, om) in enumerate(zip(geoms, omegas)):
        alone = hbs.Handle(*g, 1.0, om, 1e-12)
        ib, ia = batch[i].info(), alone.info()
        for key in ("levels", "nb_rank", "m", "n_contours"):
            assert ib[key] == ia[key], (i, key)
        assert abs(ib["max_rank"] - ia["max_rank"]) <= 1
        rb, ra = batch[i].solve(th), alone.solve(th)
        for a in range(len(th)):
            _, c1, d1, _ = rb.bragg(a)
            _, c2, d2, _ = ra.bragg(a)
            assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-11, (i, a)
    # the N = 400 star against the dense oracle
    x, y, dx, dy = geoms[0]
    assert_library_readings(batch[0].info(), x, y, omegas[0])
    res = batch[0].solve(th[:2])
    for a in range(2):
        opts = oracle_options_checked(res, a, x, y, omegas[0], th[a])
        sol = qd.dense_solve(x, y, dx, dy, omegas[0], 1.0, th[a], opts)
        _, c, d, _ = res.bragg(a)
        assert relerr(np.concatenate([c, d]), qd.bragg_vector(sol)) < 1e-10


def test_batch_many_gratings():
    """256 gratings, N log-uniform in [400, 20000], omega in [5, 40], 8 angles each, built in
    one batch: flux balance for every angle (to the discretization floor of each grating:
    the smallest N at the largest omega have only ~35 points per wavelength), and three of
    them equal to separate builds."""
    hbs = require_lib()
    w = inputs.workload_batch()
    geoms = [x["obstacle"].sample(x["N"]) for x in w]
    batch = hbs.build_batch(geoms, [x["omega"] for x in w], 1.0, 1e-12)
    worst, worst_resolved = 0.0, 0.0
    for i, x in enumerate(w):
        r = batch[i].solve(x["thetas"])
        xs, ys = geoms[i][0], geoms[i][1]
        perim = float(np.sum(np.hypot(np.diff(np.append(xs, xs[0])), np.diff(np.append(ys, ys[0])))))
        ppw = x["N"] / (x["omega"] * perim / (2 * math.pi))
        for a in range(len(x["thetas"])):
            fe = r.bragg(a)[3]
            assert np.isfinite(fe)
            worst = max(worst, fe)
            if ppw >= 200:
                worst_resolved = max(worst_resolved, fe)
    assert worst < 1e-3, worst
    assert worst_resolved < 2e-7, worst_resolved
    for i in (0, 1, 255):
        x = w[i]
        alone = hbs.Handle(*geoms[i], 1.0, x["omega"], 1e-12)
        rb, ra = batch[i].solve(x["thetas"]), alone.solve(x["thetas"])
        for a in range(len(x["thetas"])):
            _, c1, d1, _ = rb.bragg(a)
            _, c2, d2, _ = ra.bragg(a)
            assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-11
