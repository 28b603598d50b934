"""The discretization choices the paper leaves open, computed on the oracle side.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The library makes the
same choices in its own code; the tests compare the two instead of feeding the
library's values to the oracle.

Readings (the paper is silent or defers to a reference that is not at hand):

* Sommerfeld contour (Sec. 2.3).  k(t) = t - i c tanh((t - t0)/w) with c = w = 2,
  trapezoid spacing h = 0.2 in t, M nodes symmetric about t0.  The integrands of
  the wall potentials decay like exp(-|Im s| gap) along the contour, where the
  gap is the distance between the sources and the wall they are evaluated on:
  gap_B = d/2 - max|x| for the wall potentials on the obstacle (B), and
  gap_C = 3d/2 - max|x| for the images +-1 on the walls (C~).  With
  s_min = 37/(gap_B + gap_C) (so that exp(-s_min (gap_B + gap_C)) ~ 1e-16) the
  contour reaches K = sqrt(omega^2 + s_min^2) + 2 w (plus the shift T below
  when a second contour exists) and M = ceil(2 K / h).
* Wood's anomalies (Sec. 2.4).  A second contour crosses the real axis at
  t0 = T, half the smallest positive k_n that occurs at an exact anomaly.  A
  group of angles sharing a Bloch phase uses the contour that stays farther, in
  the trapezoid variable t, from all poles +-k_n of the wall integrands (the
  quadrature error near a pole at t-distance delta is ~exp(-2 pi delta / h)).
  The poles counted are +-k_n of the propagating orders and four more on each
  side; real poles with |k_n| > T + 6 are left out (both contours run at depth
  ~c there, so they rank the two alike).  Distances beyond 3 count as 3: either
  contour is then exact to rounding, and on a tie the standard one (t0 = 0) is
  kept.
* Bragg sampling (Remark 2.2, "typically 20" samples).  S = max(32, 2 ceil(omega d / 2 pi) + 44)
  equispaced samples on each line y = +-y0, y0 = max|y| + d/4.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.optimize

from . import qp_dense as qd

CONTOUR_C = 2.0
CONTOUR_W = 2.0
CONTOUR_H = 0.2
DISTANCE_CAP = 3.0


@dataclasses.dataclass
class Discretization:
    m: int          # contour nodes
    h: float        # trapezoid spacing in t
    c: float        # contour depth
    w: float        # contour bend width
    k_reach: float  # K: the contour covers Re k in about [-K, K]
    shift: float    # T: crossing point of the second contour (0 if none)
    n_samples: int  # S
    y0: float


def wood_shift(omega: float, d: float) -> float:
    """T = half the smallest positive k_n arising at an exact Rayleigh-Wood anomaly.

    At an anomaly some order has kappa = +-omega; then every order m has
    kappa_m = +-omega + 2 pi j / d for an integer j, and
    k_m = sqrt(omega^2 - kappa_m^2).  The two signs give the same set of k_m."""
    ks = []
    j = 1
    while True:
        kap = -omega + 2.0 * math.pi * j / d
        if kap >= omega:
            break
        v = omega * omega - kap * kap
        if v > 1e-12:
            ks.append(math.sqrt(v))
        j += 1
    return 0.5 * (min(ks) if ks else omega)


def discretization(x, y, omega: float, d: float) -> Discretization:
    """Contour, Bragg sampling and y0 for one obstacle (readings in the module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    xmax = float(np.max(np.abs(x)))
    gap_b = 0.5 * d - xmax
    gap_c = 1.5 * d - xmax
    s_min = 37.0 / (gap_b + gap_c)
    shift = wood_shift(omega, d)
    k_reach = math.sqrt(omega * omega + s_min * s_min) + 2.0 * CONTOUR_W
    if shift > 0.0:
        k_reach += shift
    m = int(math.ceil(2.0 * k_reach / CONTOUR_H))
    n_samples = max(32, 2 * int(math.ceil(omega * d / (2.0 * math.pi))) + 44)
    y0 = float(np.max(np.abs(y))) + 0.25 * d
    return Discretization(m, CONTOUR_H, CONTOUR_C, CONTOUR_W, k_reach, shift, n_samples, y0)


def pole_distance(p: complex, t0: float, c: float = CONTOUR_C, w: float = CONTOUR_W) -> float:
    """min over real t of |k(t) - p| / |k'(t)|, k(t) = t - i c tanh((t - t0)/w): the distance
    from the pole p to the contour measured in the trapezoid variable.  A coarse scan finds the
    basin, a bounded scalar minimisation refines it."""
    def f(t):
        u = (t - t0) / w
        k = t - 1j * c * math.tanh(u)
        dk = math.hypot(1.0, (c / w) / math.cosh(u) ** 2)
        return abs(k - p) / dk

    ts = np.linspace(p.real - 8.0, p.real + 8.0, 1601)
    us = (ts - t0) / w
    vals = np.abs(ts - 1j * c * np.tanh(us) - p) / np.hypot(1.0, (c / w) / np.cosh(us) ** 2)
    i = int(np.argmin(vals))
    lo, hi = ts[max(i - 1, 0)], ts[min(i + 1, len(ts) - 1)]
    r = scipy.optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12})
    return float(min(r.fun, vals[i]))


def contour_distances(omega: float, d: float, theta: float, disc: Discretization):
    """Capped distances of all poles +-k_n to the standard contour and to the shifted one."""
    # one order more on each side than the four named in the reading: those extra poles
    # are evanescent with |Im k_n| > 3 + c, beyond the cap, so they change nothing
    ns = qd.mode_range(omega, d, theta, extra=5)
    kn = qd.k_n(omega, qd.kappa_n(omega, d, theta, ns))
    kn = [complex(k) for k in kn if not (k.imag == 0.0 and abs(k.real) > disc.shift + 6.0)]
    out = []
    for t0 in ((0.0, disc.shift) if disc.shift > 0.0 else (0.0,)):
        best = DISTANCE_CAP
        for k in kn:
            for p in (k, -k):
                best = min(best, pole_distance(p, t0, disc.c, disc.w))
        out.append(best)
    return out


def choose_t0(omega: float, d: float, theta: float, disc: Discretization):
    """Crossing point of the contour used for the Bloch phase of `theta`, and the margin
    |dist_shifted - dist_standard| of the decision (a near tie means both contours are fine;
    inf when the choice cannot tie)."""
    dist = contour_distances(omega, d, theta, disc)
    if len(dist) == 1 or min(dist) >= DISTANCE_CAP:
        return 0.0, math.inf  # one contour, or both at the cap: the standard one, no tie
    t0 = disc.shift if dist[1] > dist[0] else 0.0
    return t0, abs(dist[1] - dist[0])


def options(x, y, omega: float, d: float, theta: float, t0: float | None = None) -> qd.Options:
    """qp_dense.Options for one angle from the readings (t0 chosen here unless given)."""
    disc = discretization(x, y, omega, d)
    if t0 is None:
        t0, _ = choose_t0(omega, d, theta, disc)
    return qd.Options(m=disc.m, h=disc.h, c=disc.c, w=disc.w, t0=t0, n_samples=disc.n_samples, y0=disc.y0)
