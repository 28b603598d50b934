"""Pins for the transmission oracle (Sec. 5; oracle/transmission.py).

The operator is derived from the jump relations, so it is pinned by what the mathematics
fixes without it: the dielectric disc in closed form (Mie series), the identity and zero
scattering at index 1, the combined layer as a special case of the pair, finite differences
of the normal derivatives, quasi-periodicity at the walls, the flux balance, mirror
symmetry, and the second periodizer."""
import math

import numpy as np
import pytest

from oracle import proxy_periodizer as pp
from oracle import qp_dense as qd
from oracle import readings as rd
from oracle import transmission as tr
from paper_1301_1247_gb300 import inputs

D = 1.0


def _disc(n, a=0.35):
    t = 2.0 * np.pi * np.arange(n) / n
    return a * np.cos(t), a * np.sin(t), -a * np.sin(t), a * np.cos(t)


def _paper_star(n):
    # Sec. 6.1: f(t) = 0.35 + 0.105 cos 3t, the transmission example uses n = 1.5, omega = 10
    return inputs.paper_star().sample(n)


def test_dielectric_disc_matches_the_mie_series_at_sixth_order():
    """Scattered field outside and total field inside an isolated disc against the closed
    form; the error falls at the Kapur-Rokhlin rate.  A wrong sign or a missing kernel
    difference anywhere in the 2 x 2 operator breaks it."""
    om, idx, th = 10.0, 1.5, -math.pi / 5
    out_pts = (np.array([0.6, -0.5, 0.0, 0.9]), np.array([0.1, 0.4, -0.7, 0.3]))
    in_pts = (np.array([0.1, -0.15, 0.0]), np.array([0.05, 0.1, -0.2]))
    errs = []
    for n in (256, 512):
        bd, sg, ta = tr.free_solve(*_disc(n), om, idx, th)
        e = []
        for (px, py), k in ((out_pts, om), (in_pts, idx * om)):
            u = tr.free_field(bd, sg, ta, k, px, py)
            ex = tr.mie_disc(0.35, om, idx, th, px, py)
            e.append(np.max(np.abs(u - ex)) / np.max(np.abs(ex)))
        errs.append(max(e))
    assert errs[1] < 1e-7
    assert errs[0] / errs[1] > 40


@pytest.mark.filterwarnings("ignore::scipy.linalg.LinAlgWarning")
def test_index_one_is_the_identity_and_scatters_nothing():
    """With n = 1 both sides share one wavenumber: every kernel difference vanishes, A = I,
    and the densities are the Green's-identity data of u_inc, whose images and wall
    potentials cancel outside: every Bragg amplitude is zero.  At an exact Wood's anomaly the
    grazing order (k_n = 0) is the exception: without an obstacle the grazing plane wave
    itself solves the homogeneous problem, so its amplitude is not determined (the system is
    singular there); it carries no flux, and every other order still vanishes."""
    x, y, dx, dy = _paper_star(300)
    bd = qd.boundary(x, y, dx, dy)
    assert np.array_equal(tr.matrix_a(bd, 10.0, 1.0), np.eye(600))
    for th in (-math.pi / 5, -math.acos(1.0 - 2.0 * math.pi / 10.0)):
        s = tr.dense_solve(x, y, dx, dy, 10.0, 1.0, D, th, rd.options(x, y, 10.0, D, th))
        keep = ~np.isin(s.orders, s.wood_modes)
        assert max(np.max(np.abs(s.c[keep])), np.max(np.abs(s.d[keep]))) < 1e-12
        assert s.flux_error < 1e-12


def test_pair_with_combined_densities_is_the_combined_layer():
    """s = -i eta (sigma = -i w eta), tau = eta makes w S s + D tau the Dirichlet combined
    layer, so the pair's outside rows reduce to the (separately pinned) Dirichlet oracle's."""
    om = 10.0
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(200)
    bd = qd.boundary(x, y, dx, dy)
    rng = np.random.default_rng(5)
    eta = rng.standard_normal(bd.n) + 1j * rng.standard_normal(bd.n)
    pair = tr.interlace_rows(-1j * eta, eta)

    def close(a, b):
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)

    for j in (-1, 1):
        close((tr.matrix_a_image(bd, om, D, j) @ pair)[1::2], qd.matrix_a_image(bd, om, D, j) @ eta)
    ct = qd.contour(120, 0.4, 2.0, 2.0)
    alpha = np.exp(0.7j)
    xs, ys = qd.sample_points(D, 17), np.full(17, 0.9)
    for der in (None, "x", "y"):
        pe, px = tr.eval_rows(xs, ys, bd, ct, om, D, alpha, 1, der)
        de, dxi = qd.eval_rows(xs, ys, bd, ct, om, D, alpha, 1, der)
        close(pe @ pair, de @ eta)
        assert np.array_equal(px, dxi)
    for x0, sh in ((-0.5 * D, D), (0.5 * D, -D)):
        close(tr.wall_fourier_rows_pair(bd.x + sh, bd.y, bd.nx, bd.ny, bd.w, ct, om, x0) @ pair,
              qd.wall_fourier_rows(bd.x + sh, bd.y, bd.nx, bd.ny, bd.w, ct, om, x0) @ eta)
    bl, br = tr.matrix_b_parts(bd, ct, om, D)
    dl, dr = qd.matrix_b_parts(bd, ct, om, D)
    assert np.array_equal(bl[1::2], dl) and np.array_equal(br[1::2], dr)


def test_sigma_rows_are_minus_normal_derivatives():
    """The sigma rows of the image blocks, of B and of the right-hand side equal minus a
    centred finite difference of the field along the normal, divided by w."""
    om = 10.0
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(160)
    bd = qd.boundary(x, y, dx, dy)
    h = 1e-5
    rng = np.random.default_rng(7)
    eta = rng.standard_normal(2 * bd.n) + 1j * rng.standard_normal(2 * bd.n)
    ct = qd.contour(120, 0.4, 2.0, 2.0)
    xi = rng.standard_normal(2 * ct.m) + 1j * rng.standard_normal(2 * ct.m)
    alpha = np.exp(0.3j)
    up = (bd.x + h * bd.nx, bd.y + h * bd.ny)
    dn = (bd.x - h * bd.nx, bd.y - h * bd.ny)

    # images +-1 only (P = 1 rows minus the obstacle's own term)
    def img_field(pts):
        e, _ = tr.eval_rows(pts[0], pts[1], bd, ct, om, D, alpha, 1)
        e0, _ = tr.eval_rows(pts[0], pts[1], bd, ct, om, D, alpha, 0)
        return (e - e0) @ eta

    fd = -(img_field(up) - img_field(dn)) / (2 * h) / om
    rows = (alpha * tr.matrix_a_image(bd, om, D, 1) + tr.matrix_a_image(bd, om, D, -1) / alpha) @ eta
    assert np.linalg.norm(rows[0::2] - fd) < 1e-6 * np.linalg.norm(fd)

    def wall_field(pts):
        return tr.eval_rows(pts[0], pts[1], bd, ct, om, D, alpha, 0)[1] @ xi

    fd = -(wall_field(up) - wall_field(dn)) / (2 * h) / om
    bl, br = tr.matrix_b_parts(bd, ct, om, D)
    assert np.linalg.norm(((bl + alpha * br) @ xi)[0::2] - fd) < 1e-6 * np.linalg.norm(fd)

    th = -0.9
    inc = lambda p: np.exp(1j * om * (math.cos(th) * p[0] + math.sin(th) * p[1]))
    rhs = tr.incident_rhs(bd, om, th)
    assert np.linalg.norm(rhs[0::2] - (inc(up) - inc(dn)) / (2 * h) / om) < 1e-6
    assert np.max(np.abs(rhs[1::2] + inc((bd.x, bd.y)))) < 1e-14


def test_wall_quasi_periodicity_and_flux_balance():
    """The solved outside field, summed directly at points of the walls, is quasi-periodic,
    and the lossless grating conserves flux, converging at the Kapur-Rokhlin rate."""
    om, idx, th = 10.0, 1.5, -math.pi / 5
    errs = []
    for n in (300, 600):
        x, y, dx, dy = _paper_star(n)
        o = rd.options(x, y, om, D, th)
        s = tr.dense_solve(x, y, dx, dy, om, idx, D, th, o)
        errs.append(s.flux_error)
    bd = qd.boundary(x, y, dx, dy)
    ct = qd.contour(o.m, o.h, o.c, o.w, o.t0)
    yy = np.linspace(-1.0, 1.0, 41)
    for der in (None, "x"):
        el, xl = tr.eval_rows(np.full_like(yy, -0.5), yy, bd, ct, om, D, s.alpha, 1, der)
        er, xr = tr.eval_rows(np.full_like(yy, 0.5), yy, bd, ct, om, D, s.alpha, 1, der)
        ul, ur = el @ s.eta + xl @ s.xi, er @ s.eta + xr @ s.xi
        assert np.max(np.abs(ul - ur / s.alpha)) < 1e-11 * np.max(np.abs(ul))
    # measured: 4.8e-6 (N = 300), 1.1e-7 (600), 1.3e-9 (1200)
    assert errs[1] < 2e-7
    assert errs[0] / errs[1] > 30


def test_mirror_symmetry_normal_incidence():
    obs = inputs.star(0.3, 0.25, 4)
    x, y, dx, dy = obs.sample(320)
    th = -math.pi / 2
    s = tr.dense_solve(x, y, dx, dy, 10.0, 1.5, D, th, rd.options(x, y, 10.0, D, th))
    assert list(s.orders) == list(-s.orders[::-1])
    assert np.allclose(s.c, s.c[::-1], atol=1e-12, rtol=0)
    assert np.allclose(s.d, s.d[::-1], atol=1e-12, rtol=0)


@pytest.mark.parametrize("obs,n,om,idx,thetas", [
    (inputs.star(0.3, 0.3, 5), 400, 10.0, 1.5,
     [-math.pi / 5, -1.0, -2.5, -math.acos(1.0 - 2.0 * math.pi / 10.0)]),
    (inputs.wiggly(0, 0.35, 20, 0.03), 1000, 30.0, 1.3, [-0.7, -math.acos(1.0 - 2.0 * math.pi * 2 / 30.0)]),
])
def test_second_periodizer_and_both_contours_agree(obs, n, om, idx, thetas):
    """The box scheme (proxy points, wall discrepancies) and the Fourier-wall scheme on its
    standard and its shifted contour solve one continuum problem: equal Bragg amplitudes.
    This checks B, C~ and the Wood's rows of the pair independently of their derivation."""
    x, y, dx, dy = obs.sample(n)
    blocks = tr.obstacle_blocks(x, y, dx, dy, om, idx, D)
    shift = rd.discretization(x, y, om, D).shift
    for th in thetas:
        f = tr.dense_solve(x, y, dx, dy, om, idx, D, th, rd.options(x, y, om, D, th), blocks)
        vf = qd.bragg_vector(f)
        p = tr.proxy_solve(x, y, dx, dy, om, idx, D, th, blocks=blocks)
        assert p.residual < 1e-11
        c, d = pp.bragg_at(p, om, D, th, f.y0)
        assert np.linalg.norm(np.concatenate([c, d]) - vf) < 1e-10 * np.linalg.norm(vf), th
        if not len(f.wood_modes):
            for t0 in (0.0, shift):
                g = tr.dense_solve(x, y, dx, dy, om, idx, D, th, rd.options(x, y, om, D, th, t0=t0), blocks)
                assert np.linalg.norm(qd.bragg_vector(g) - vf) < 1e-10 * np.linalg.norm(vf), (th, t0)
