"""The oracle's second periodizing scheme (proxy points and wall discrepancies,
oracle/proxy_periodizer.py) against the Fourier-wall scheme of Secs. 2.2-2.4: two
discretizations of one continuum problem must give the same Bragg amplitudes.  A mistake in
either scheme's wall operators (Q, C~, the contour, the Wood's rows, the image telescoping)
breaks the agreement."""
import math

import numpy as np
import pytest

from oracle import proxy_periodizer as pp
from oracle import qp_dense as qd
from oracle import readings as rd
from paper_1301_1247_gb300 import inputs


def _compare(obs, n, omega, thetas, tol):
    x, y, dx, dy = obs.sample(n)
    blocks = qd.obstacle_blocks(x, y, dx, dy, omega, 1.0)
    for th in thetas:
        s = pp.solve(x, y, dx, dy, omega, 1.0, th, blocks=blocks)
        f = qd.dense_solve(x, y, dx, dy, omega, 1.0, th, rd.options(x, y, omega, 1.0, th), blocks)
        assert list(s.orders) == list(f.orders)
        c, d = pp.bragg_at(s, omega, 1.0, th, f.y0)
        v, vf = np.concatenate([c, d]), qd.bragg_vector(f)
        assert s.residual < 1e-11, (th, s.residual)
        assert np.linalg.norm(v - vf) / np.linalg.norm(vf) < tol, th


def test_proxy_and_fourier_wall_schemes_agree_on_the_star():
    """omega = 10, N = 400: generic angles, normal incidence and the Wood's anomaly of Sec. 6.2
    (where the Fourier-wall scheme needs its shifted contour and extra row; the box scheme
    needs nothing special)."""
    _compare(inputs.star(0.3, 0.3, 5), 400, 10.0,
             [-math.pi / 5, -1.0, -2.5, -math.pi / 2, -math.acos(1.0 - 2.0 * math.pi / 10.0)], 1e-12)


def test_proxy_and_fourier_wall_schemes_agree_on_a_wiggly_obstacle():
    _compare(inputs.wiggly(0, 0.35, 20, 0.03), 1200, 30.0,
             [-0.7, -2.0, -math.acos(1.0 - 2.0 * math.pi * 2 / 30.0)], 1e-11)


def test_proxy_scheme_sizes_are_converged():
    """More proxies, more Rayleigh-Bloch modes and a taller box leave the amplitudes unchanged
    (after referring them to one height)."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(400)
    omega, th = 10.0, -0.8
    blocks = qd.obstacle_blocks(x, y, dx, dy, omega, 1.0)
    ref = np.concatenate(pp.bragg_at(pp.solve(x, y, dx, dy, omega, 1.0, th, blocks=blocks), omega, 1.0, th, 0.7))
    for o in (pp.ProxyOptions(m_proxy=160), pp.ProxyOptions(k_modes=80), pp.ProxyOptions(h=0.55)):
        v = np.concatenate(pp.bragg_at(pp.solve(x, y, dx, dy, omega, 1.0, th, o, blocks), omega, 1.0, th, 0.7))
        assert np.linalg.norm(v - ref) / np.linalg.norm(ref) < 1e-12, o


def test_proxy_scheme_conserves_flux():
    """Lossless Dirichlet grating: the outgoing propagating orders carry the incident flux,
    from the a_n, b_n directly (the incident wave's own term in the order 0 below)."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(600)
    omega, th = 10.0, -0.9
    s = pp.solve(x, y, dx, dy, omega, 1.0, th)
    kn = qd.k_n(omega, qd.kappa_n(omega, 1.0, th, s.orders)).real
    k0 = omega * abs(math.sin(th))
    inc = np.where(s.orders == 0, np.exp(1j * k0 * s.h), 0.0)
    flux = float(np.sum((kn / k0) * (np.abs(s.c) ** 2 + np.abs(s.d + inc) ** 2)))
    assert abs(flux - 1.0) < 1e-6
