"""Parity of the transmission path (Sec. 5) through the C ABI with the dense oracle
(oracle/transmission.py): entries of the interlaced operator, Bragg amplitudes of the full
solve (FP64 and tensor-core precision, exact Wood's anomalies), the compressed inverse, the
paper's per-phase path, and index 1 (no scattering)."""
import math

import numpy as np
import pytest

from oracle import qp_dense as qd
from oracle import readings as rd
from oracle import transmission as tr
from paper_1301_1247_gb300 import inputs

from gpu_util import assert_library_readings, dev, oracle_options_checked, relerr, require_lib

pytestmark = pytest.mark.gpu

D = 1.0


def _handle(hbs, geom, omega, index, precision=0, tol=1e-12):
    x, y, dx, dy = geom
    h = hbs.Handle(x, y, dx, dy, D, omega, tol, hbs.default_options(index=index, precision=precision))
    assert h.unknowns == 2 * len(x)
    info = h.info()
    assert info["n"] == len(x) and info["index"] == index
    assert_library_readings(info, x, y, omega)
    return h


def _compare(res, geom, omega, index, thetas, tol, blocks=None):
    x, y, dx, dy = geom
    blocks = blocks or tr.obstacle_blocks(x, y, dx, dy, omega, index, D)
    worst = 0.0
    for i, th in enumerate(thetas):
        nw, _ = res.angle_info(i)
        sol = tr.dense_solve(x, y, dx, dy, omega, index, D, th, oracle_options_checked(res, i, x, y, omega, th),
                             blocks)
        orders, c, d, fe = res.bragg(i)
        assert list(orders) == list(sol.orders)
        assert nw == len(sol.wood_modes)
        e = relerr(np.concatenate([c, d]), qd.bragg_vector(sol))
        assert e < tol, (th, e)
        assert abs(fe - sol.flux_error) < 1e-9
        worst = max(worst, e)
    print(f"transmission parity: worst relative Bragg error {worst:.2e} over {len(thetas)} angles")
    return worst


@pytest.mark.parametrize("case", [("star", 300, 10.0, 1.5), ("wiggly", 2001, 30.0, 1.3)])
def test_kernel_block_entries(case):
    """Entries of the interlaced operator (identity plus kernel differences with KR6 weights)
    and of its images, element by element, including the node's own 2 x 2 block and the
    Kapur-Rokhlin band next to it."""
    import torch
    hbs = require_lib()
    name, n, omega, index = case
    obs = inputs.star(0.3, 0.3, 5) if name == "star" else inputs.wiggly(3, 0.3, 60, 0.05)
    x, y, dx, dy = obs.sample(n)
    bd = qd.boundary(x, y, dx, dy)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, 2 * n, 50), [0, 1, 2, 3, 2 * n - 1, n, n + 1]]))
    cols = np.unique(np.concatenate([rng.integers(0, 2 * n, 60),
                                     [0, 1, 2, 3, 4, 5, 10, 11, 12, 13, 2 * n - 1, 2 * n - 12, n + 2, n + 3]]))
    gx, gy, gdx, gdy = (dev(a) for a in (x, y, dx, dy))
    out = torch.zeros((len(cols), len(rows)), dtype=torch.complex128, device="cuda")
    r_d, c_d = dev(rows.astype(np.int64)), dev(cols.astype(np.int64))
    ref = tr.matrix_a(bd, omega, index)[np.ix_(rows, cols)]
    hbs.kernel_block_transmission(gx, gy, gdx, gdy, omega, index, 0, 0.0, r_d, c_d, out)
    got = out.cpu().numpy().T
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale
    for shift in (-1.0, 1.0):
        refi = tr.matrix_a_image(bd, omega, D, int(shift))[np.ix_(rows, cols)]
        hbs.kernel_block_transmission(gx, gy, gdx, gdy, omega, index, 1, shift, r_d, c_d, out)
        got = out.cpu().numpy().T
        assert np.max(np.abs(got - refi)) <= 1e-13 * np.abs(refi).max()


@pytest.mark.parametrize("precision", [0, 2])
def test_solve_matches_oracle_paper_star(precision):
    """The transmission example of Sec. 6.1 (f(t) = 0.35 + 0.105 cos 3t, omega = 10, n = 1.5):
    generic angles, normal incidence and the exact Wood's anomaly of Sec. 6.2, in FP64 and in
    the tensor-core precision mode."""
    hbs = require_lib()
    geom = inputs.paper_star().sample(400)
    omega, index = 10.0, 1.5
    h = _handle(hbs, geom, omega, index, precision)
    thetas = np.array([-math.pi / 5, -0.4, -1.0, -math.pi / 2, -2.5, -math.acos(1.0 - 2.0 * math.pi / omega)])
    res = h.solve(thetas)
    assert res.angle_info(len(thetas) - 1)[0] == 1
    _compare(res, geom, omega, index, thetas, 1e-10)


def test_index_one_scatters_nothing():
    """n = 1: the operator is the identity, and every Bragg amplitude vanishes."""
    hbs = require_lib()
    geom = inputs.paper_star().sample(300)
    h = _handle(hbs, geom, 10.0, 1.0)
    res = h.solve([-math.pi / 5, -1.3])
    for i in range(2):
        _, c, d, fe = res.bragg(i)
        assert max(np.abs(c).max(), np.abs(d).max()) < 1e-11
        assert fe < 1e-11


@pytest.mark.parametrize("precision", [0, 2])
def test_wiggly_n3000_matches_oracle(precision):
    """N = 3000 nodes (6000 unknowns) at omega = 30: neighbour-ID candidates on every second
    node, periodizer IDs on a node subsample, several Bloch groups and an exact Wood's
    anomaly, against the dense oracle."""
    hbs = require_lib()
    geom = inputs.wiggly(0, 0.35, 20, 0.03).sample(3000)
    omega, index = 30.0, 1.3
    h = _handle(hbs, geom, omega, index, precision)
    info = h.info()
    assert info["nb_residual"] > 0.0  # the candidate stride is active
    thetas = np.array([-0.7, -1.9, -math.acos(1.0 - 2.0 * math.pi * 2 / omega)])
    res = h.solve(thetas)
    assert res.angle_info(2)[0] >= 1
    x, y, dx, dy = geom
    _compare(res, geom, omega, index, thetas, 1e-10, tr.obstacle_blocks(x, y, dx, dy, omega, index, D))


def test_plain_path_and_compressed_inverse():
    """The paper's per-phase path agrees with the precomputed one, and the compressed inverse
    solves the oracle's transmission system: rows of A times A^{-1} b reproduce b."""
    import torch
    hbs = require_lib()
    geom = inputs.wiggly(1, 0.33, 12, 0.04).sample(1500)
    omega, index = 20.0, 1.5
    h = _handle(hbs, geom, omega, index)
    thetas = [-0.5, -1.2, -2.2]
    a, b = h.solve(thetas), h.solve_plain(thetas)
    for i in range(len(thetas)):
        _, ca, da, _ = a.bragg(i)
        _, cb, db, _ = b.bragg(i)
        assert relerr(np.concatenate([ca, da]), np.concatenate([cb, db])) < 1e-10
    x, y, dx, dy = geom
    n2 = h.unknowns
    rng = np.random.default_rng(11)
    rhs = rng.standard_normal((2, n2)) + 1j * rng.standard_normal((2, n2))
    bt = torch.from_numpy(rhs).cuda()
    xt = torch.zeros_like(bt)
    h.apply_inverse(bt, xt, 2)
    sol = xt.cpu().numpy()
    bd = qd.boundary(x, y, dx, dy)
    amat = tr.matrix_a(bd, omega, index)
    rows = np.unique(np.concatenate([rng.integers(0, n2, 200), [0, 1, n2 - 2, n2 - 1]]))
    for k in range(2):
        assert relerr(amat[rows] @ sol[k], rhs[k][rows]) < 1e-10


def test_batch_build_and_server():
    """Transmission solvers built in one batch (every tree level of every grating in the same
    launches) solve like separate builds, the smallest like the dense oracle, and the request
    server answers single angles on them with the same amplitudes."""
    hbs = require_lib()
    specs = [(inputs.paper_star(), 300, 10.0), (inputs.wiggly(1, 0.35, 20, 0.03), 1200, 25.0),
             (inputs.star(0.25, 0.2, 3), 600, 8.0)]
    geoms = [obs.sample(n) for obs, n, _ in specs]
    omegas = [om for _, _, om in specs]
    index = 1.4
    opts = hbs.default_options(index=index)
    batch = hbs.build_batch(geoms, omegas, D, 1e-12, opts)
    th = inputs.uniform_angles(5, 6, -math.pi / 2 + 0.05, -0.1)
    for i, (g, om) in enumerate(zip(geoms, omegas)):
        assert batch[i].unknowns == 2 * len(g[0])
        alone = hbs.Handle(*g, D, om, 1e-12, opts)
        rb, ra = batch[i].solve(th), alone.solve(th)
        for a in range(len(th)):
            _, c1, d1, _ = rb.bragg(a)
            _, c2, d2, _ = ra.bragg(a)
            assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-11, (i, a)
    _compare(batch[0].solve(th[:3]), geoms[0], omegas[0], index, th[:3], 1e-10)
    sv = hbs.Server(hbm_budget_bytes=0, slots=2, max_batch=16)
    try:
        gids = [sv.add(h) for h in batch]
        reqs = [(i, a, sv.submit(gids[i], float(th[a]))) for i in range(len(batch)) for a in range(len(th))]
        for i, a, rid in reqs:
            _, c, d, _ = sv.wait(rid, 120.0)
            _, c2, d2, _ = batch[i].solve([th[a]]).bragg(0)
            assert relerr(np.concatenate([c, d]), np.concatenate([c2, d2])) < 1e-11, (i, a)
    finally:
        sv.close()


def test_proxy_periodizer_matches_its_oracle_and_the_fourier_wall_solve():
    """The second periodizer (hbs_solve_proxy) on a transmission solver: its amplitudes match
    the oracle's box scheme for the pair (transmission.proxy_solve), the dense Fourier-wall
    transmission oracle and the library's Fourier-wall solve, including an exact Wood's
    anomaly."""
    from oracle import proxy_periodizer as pp
    hbs = require_lib()
    geom = inputs.paper_star().sample(400)
    x, y, dx, dy = geom
    omega, index = 10.0, 1.5
    h = _handle(hbs, geom, omega, index)
    y0 = h.info()["y0"]
    thetas = np.array([-math.pi / 5, -1.0, -2.5, -math.acos(1.0 - 2.0 * math.pi / omega)])
    rp_, rf_ = h.solve_proxy(thetas), h.solve(thetas)
    blocks = tr.obstacle_blocks(x, y, dx, dy, omega, index, D)
    for i, th in enumerate(thetas):
        orders, c, d, flux = rp_.bragg(i)
        got = np.concatenate([c, d])
        sp = tr.proxy_solve(x, y, dx, dy, omega, index, D, th, blocks=blocks)
        cp, dp = pp.bragg_at(sp, omega, D, th, y0)
        assert list(orders) == list(sp.orders)
        assert relerr(got, np.concatenate([cp, dp])) < 1e-10, (th, "proxy oracle")
        sf = tr.dense_solve(x, y, dx, dy, omega, index, D, th, rd.options(x, y, omega, D, th), blocks)
        assert relerr(got, qd.bragg_vector(sf)) < 1e-10, (th, "Fourier-wall oracle")
        _, c2, d2, _ = rf_.bragg(i)
        assert relerr(got, np.concatenate([c2, d2])) < 1e-10, (th, "Fourier-wall solve")
        assert abs(flux - sf.flux_error) < 1e-8
