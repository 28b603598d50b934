"""Pins for the oracle's own discretization choices (oracle/readings.py): the Sommerfeld
contour and its size (Sec. 2.3), the Wood's-anomaly contour and the per-phase choice between
the two (Sec. 2.4), and the Bragg sampling (Remark 2.2).  None of these values comes from the
library; the GPU tests assert that the library makes the same choices."""
import math

import numpy as np

from oracle import qp_dense as qd
from oracle import readings as rd
from paper_1301_1247_gb300 import inputs

D = 1.0


def test_wood_shift_is_half_the_smallest_anomaly_wavenumber():
    """omega = 10, d = 1, worked by hand: at an anomaly kappa_n = +-10 and the other orders
    sit at +-10 - 2 pi j.  j = 1, 2, 3 give kappa = 3.717, -2.566, -8.850 and
    k = 9.2836, 9.6652, 4.6566 (j >= 4 is evanescent), so T = 4.6566 / 2."""
    assert abs(rd.wood_shift(10.0, D) - 2.32830) < 1e-4
    # brute force over every exact anomaly angle: all real k_n > 0 stay >= 2T, and one equals it
    for omega in (10.0, 23.7, 30.0, 60.0):
        t_shift = rd.wood_shift(omega, D)
        smallest = math.inf
        for n_an in range(1, int(2 * omega / (2 * math.pi)) + 1):
            th = -math.acos(1.0 - 2.0 * math.pi * n_an / (omega * D))
            ns = qd.mode_range(omega, D, th, extra=3)
            kn = qd.k_n(omega, qd.kappa_n(omega, D, th, ns))
            pos = [k.real for k in kn if k.imag == 0.0 and k.real > 0.0]
            smallest = min(smallest, min(pos))
        assert abs(smallest - 2.0 * t_shift) < 1e-9 * omega


def test_contour_size_formula_on_a_circle():
    """A circle of radius 0.4 at omega = 10: gaps 0.1 and 1.1, s_min = 37 / 1.2 = 30.833, and
    K = sqrt(100 + 950.69) + 4 + T = 36.414 + 2.328 = 38.743 by hand, so M = ceil(2K/0.2) = 388;
    S = max(32, 2 ceil(10 / 2 pi) + 44) = 48 and y0 = 0.4 + 1/4."""
    t = 2 * math.pi * np.arange(512) / 512
    disc = rd.discretization(0.4 * np.cos(t), 0.4 * np.sin(t), 10.0, D)
    assert abs(disc.k_reach - 38.7427) < 1e-3
    assert disc.m == 388
    assert disc.n_samples == 48 and abs(disc.y0 - 0.65) < 1e-12


def test_pole_distance_by_brute_force():
    """The refined distance equals a dense scan of the contour (1e6 points) to 1e-7, and is 0
    for a pole on the contour."""
    for p, t0 in ((complex(3.1, 0.0), 0.0), (complex(0.0, 1.5), 0.0), (complex(2.5, 0.0), 2.33),
                  (complex(0.0, 1.94), 4.25), (complex(-7.0, 0.3), 2.33)):
        ts = np.linspace(p.real - 10, p.real + 10, 1_000_001)
        u = (ts - t0) / rd.CONTOUR_W
        k = ts - 1j * rd.CONTOUR_C * np.tanh(u)
        dk = np.hypot(1.0, (rd.CONTOUR_C / rd.CONTOUR_W) / np.cosh(u) ** 2)
        assert abs(rd.pole_distance(p, t0) - np.min(np.abs(k - p) / dk)) < 1e-7
    on = complex(1.3, -rd.CONTOUR_C * math.tanh(1.3 / rd.CONTOUR_W))
    assert rd.pole_distance(on, 0.0) < 1e-9


def test_contour_choice_keeps_every_pole_away():
    """Over many angles, exact anomalies included, the chosen contour keeps all poles at least
    0.6 away in t (quadrature error ~exp(-2 pi 0.6 / 0.2) ~ 1e-8 at worst, far less in
    practice), and at the paper's Wood's angle (Sec. 6.2) the shifted contour is chosen."""
    for omega in (10.0, 30.0, 60.0):
        disc = rd.discretization(*inputs.star(0.3, 0.3, 5).sample(256)[:2], omega, D)
        ths = list(-np.linspace(0.02, math.pi - 0.02, 60))
        ths += [-math.acos(1.0 - 2.0 * math.pi * n / (omega * D)) for n in (1, 2)]
        for th in ths:
            t0, _ = rd.choose_t0(omega, D, th, disc)
            dist = rd.contour_distances(omega, D, th, disc)
            chosen = dist[1] if (t0 > 0 and len(dist) > 1) else dist[0]
            assert chosen >= 0.6, (omega, th, dist)
    disc = rd.discretization(*inputs.star(0.3, 0.3, 5).sample(256)[:2], 10.0, D)
    th_w = -math.acos(1.0 - 2.0 * math.pi / 10.0)
    assert rd.choose_t0(10.0, D, th_w, disc)[0] == disc.shift > 0


def test_contour_size_is_converged():
    """With the reading's K and M the Bragg amplitudes already agree with a contour reaching
    30 % farther (same h): truncating the contour at K costs nothing measurable."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(300)
    omega, th = 10.0, -math.pi / 5
    blocks = qd.obstacle_blocks(x, y, dx, dy, omega, D)
    o = rd.options(x, y, omega, D, th)
    a = qd.dense_solve(x, y, dx, dy, omega, D, th, o, blocks)
    o.m = int(1.3 * o.m)
    b = qd.dense_solve(x, y, dx, dy, omega, D, th, o, blocks)
    va, vb = qd.bragg_vector(a), qd.bragg_vector(b)
    assert np.linalg.norm(va - vb) / np.linalg.norm(va) < 1e-12


def test_bragg_results_independent_of_samples_and_y0():
    """Remark 2.2: the amplitudes are coefficients of the exact Rayleigh-Bloch expansion, so
    they do not depend on where (y0) or how densely (S) the field is sampled, once S exceeds the
    band of modes the field holds at y0.  Also at a Wood's anomaly, where the extra row samples
    the field at -y0."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(300)
    omega = 10.0
    blocks = qd.obstacle_blocks(x, y, dx, dy, omega, D)
    for th in (-math.pi / 5, -math.acos(1.0 - 2.0 * math.pi / omega)):
        base = rd.options(x, y, omega, D, th)
        ref = qd.bragg_vector(qd.dense_solve(x, y, dx, dy, omega, D, th, base, blocks))
        for n_s, dy0 in ((base.n_samples + 24, 0.0), (base.n_samples, 0.15), (2 * base.n_samples, 0.3)):
            o = rd.options(x, y, omega, D, th)
            o.n_samples, o.y0 = n_s, o.y0 + dy0
            s = qd.dense_solve(x, y, dx, dy, omega, D, th, o, blocks)
            v = qd.bragg_vector(s)
            # d_n is measured at -y0, the incident wave's phase reference; c_n at +y0.  Both
            # are amplitudes of modes normalised at y = 0 in the paper's expansion, so moving
            # y0 rescales mode n by exp(i k_n dy0): undo that before comparing.
            kn = qd.k_n(omega, qd.kappa_n(omega, D, th, s.orders))
            ph = np.concatenate([np.exp(-1j * kn * dy0), np.exp(-1j * kn * dy0)])
            assert np.linalg.norm(v * ph - ref) / np.linalg.norm(ref) < 1e-13, (th, n_s, dy0)
