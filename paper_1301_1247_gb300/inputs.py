"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver itself: it only turns a seed and
a few shape parameters into obstacle boundary samples z(t_j), z'(t_j) and sets
of incident angles.  Both the CUDA library and the CPU oracle take these arrays
as their inputs.

Obstacles are radial curves z(t) = (r(t) cos t, r(t) sin t), t in [0, 2pi),
traversed counter-clockwise, sampled at the N equispaced parameter values
t_j = 2 pi j / N of the periodic trapezoid rule (Sec. 2.3).  The paper's own
examples are of this form: the star f(t) = 0.35 + 0.105 cos 3t (Sec. 6.1) and a
random radial Fourier series (Sec. 6.2), whose coefficients it does not print,
so seeded stand-ins are drawn here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class RadialObstacle:
    """r(t) = r0 * (1 + sum_j a_j cos(j t + phi_j))."""

    r0: float
    modes: tuple  # tuple of (j, a_j, phi_j)

    def radius(self, t: np.ndarray) -> np.ndarray:
        r = np.ones_like(t)
        for j, a, p in self.modes:
            r = r + a * np.cos(j * t + p)
        return self.r0 * r

    def dradius(self, t: np.ndarray) -> np.ndarray:
        dr = np.zeros_like(t)
        for j, a, p in self.modes:
            dr = dr - a * j * np.sin(j * t + p)
        return self.r0 * dr

    def sample(self, n: int):
        """Return (x, y, dx, dy) at t_j = 2 pi j / n, float64 arrays of length n."""
        t = 2.0 * math.pi * np.arange(n, dtype=np.float64) / n
        r = self.radius(t)
        dr = self.dradius(t)
        c, s = np.cos(t), np.sin(t)
        x = r * c
        y = r * s
        dx = dr * c - r * s
        dy = dr * s + r * c
        return (np.ascontiguousarray(x), np.ascontiguousarray(y),
                np.ascontiguousarray(dx), np.ascontiguousarray(dy))

    def extent(self, n_fine: int = 20000):
        t = 2.0 * math.pi * np.arange(n_fine) / n_fine
        r = self.radius(t)
        return (float(np.max(np.abs(r * np.cos(t)))), float(np.max(np.abs(r * np.sin(t)))),
                float(np.min(r)), float(np.max(r)))


def star(r0: float = 0.3, eps: float = 0.3, m: int = 5) -> RadialObstacle:
    """Smooth star r(t) = r0 (1 + eps cos m t)."""
    return RadialObstacle(r0, ((m, eps, 0.0),))


def paper_star() -> RadialObstacle:
    """The star of the scaling experiment, f(t) = 0.35 + 0.105 cos 3t (Sec. 6.1)."""
    return RadialObstacle(0.35, ((3, 0.3, 0.0),))


def wiggly(seed: int, r0: float, n_modes: int, amp: float, d: float = 1.0,
           max_radius_frac: float = 0.42, min_radius_frac: float = 0.2) -> RadialObstacle:
    """Seeded random radial Fourier series r0 (1 + sum_{j=1}^{n_modes} a_j cos(j t + phi_j)).

    a_j ~ U(0, amp) and phi_j ~ U(0, 2 pi) from numpy default_rng(seed).  The
    paper requires the obstacle to stay inside the unit cell without touching
    its walls (Sec. 2.1); the draw is deterministically rescaled (all a_j
    multiplied by 0.8 until it fits) so that max r <= max_radius_frac * d and
    min r >= min_radius_frac * r0.
    """
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, amp, size=n_modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    for _ in range(200):
        obs = RadialObstacle(r0, tuple((j + 1, float(a[j]), float(phi[j])) for j in range(n_modes)))
        _, _, rmin, rmax = obs.extent()
        if rmax <= max_radius_frac * d and rmin >= min_radius_frac * r0:
            return obs
        a = a * 0.8
    raise RuntimeError("could not rescale obstacle into the unit cell")


def bloch_grouped_angles(seed: int, omega: float, d: float, n_groups: int, q: int) -> np.ndarray:
    """Incident angles in groups of q sharing one Bloch phase alpha = exp(i omega d cos theta).

    Within a group cos(theta_m) = c + 2 pi m / (omega d), m = 0..q-1 (Remark 3.1,
    Sec. 6.2); the group offsets c are drawn from default_rng(seed) so that all
    cos(theta) lie in (-1, 1).  Returns an (n_groups, q) array of theta in (-pi, 0).
    """
    step = 2.0 * math.pi / (omega * d)
    hi = 1.0 - (q - 1) * step
    if hi <= -1.0:
        raise ValueError("q angles sharing alpha do not fit in (-1, 1)")
    rng = np.random.default_rng(seed)
    lo_margin = 1e-3
    c = rng.uniform(-1.0 + lo_margin, hi - lo_margin, size=n_groups)
    cos_t = c[:, None] + step * np.arange(q)[None, :]
    return -np.arccos(cos_t)


def uniform_angles(seed: int, n: int, lo: float = -math.pi / 2, hi: float = 0.0) -> np.ndarray:
    """n angles uniform in (lo, hi) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


# Named workloads.  Each returns (obstacle, omega, d, N) plus its angle set.

def workload_star_n400():
    """Star r = 0.3(1 + 0.3 cos 5t), d = 1, omega = 10, N = 400, theta = -pi/5."""
    return dict(obstacle=star(0.3, 0.3, 5), omega=10.0, d=1.0, N=400,
                thetas=np.array([-math.pi / 5]))


def workload_wiggly_n10k(seed: int = 0):
    """Wiggly r = 0.35(1 + sum_{j<=20} a_j cos(j t + phi_j)), a_j ~ U(0, 0.03), omega = 30,
    N = 10 000, 20 angles uniform in (-pi/2, 0)."""
    return dict(obstacle=wiggly(seed, 0.35, 20, 0.03), omega=30.0, d=1.0, N=10000,
                thetas=uniform_angles(seed + 1, 20))


def workload_complicated_n100k(seed: int = 0, n_groups: int = 100, q: int = 10):
    """Complicated obstacle: r0 = 0.3 with 60 modes of amplitude <= 0.05, omega = 60,
    N = 100 000, 1000 angles in 100 groups of 10 sharing a Bloch phase."""
    return dict(obstacle=wiggly(seed, 0.3, 60, 0.05), omega=60.0, d=1.0, N=100000,
                thetas=bloch_grouped_angles(seed + 1, 60.0, 1.0, n_groups, q))


def workload_transmission_n10k(seed: int = 0, n_groups: int = 100, q: int = 9):
    """Transmission grating (Sec. 6.3: the complicated obstacle of Sec. 6.2 with dielectric
    obstacles): r0 = 0.3 with 60 modes of amplitude <= 0.05, omega = 30, refractive index
    1.5, N = 10 000 nodes (20 000 unknowns), 900 angles in 100 groups of 9 sharing a Bloch
    phase."""
    return dict(obstacle=wiggly(seed, 0.3, 60, 0.05), omega=30.0, d=1.0, N=10000, index=1.5,
                thetas=bloch_grouped_angles(seed + 1, 30.0, 1.0, n_groups, q))


def workload_batch(seed: int = 0, count: int = 256, n_lo: int = 400, n_hi: int = 20000, w_lo: float = 5.0,
                   w_hi: float = 40.0, n_angles: int = 8):
    """Many independent gratings: alternating star and wiggly obstacles with N log-uniform in
    [n_lo, n_hi] (rounded to a multiple of 8), omega uniform in [w_lo, w_hi] and n_angles
    incident angles uniform in (-pi/2 + 0.02, -0.1) each (away from grazing incidence).  Returns a list of dicts (obstacle, N, omega,
    d, thetas)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))) / 8.0)) * 8
        omega = float(rng.uniform(w_lo, w_hi))
        if i % 2 == 0:
            obs = star(float(rng.uniform(0.2, 0.3)), float(rng.uniform(0.1, 0.3)), int(rng.integers(3, 7)))
        else:
            obs = wiggly(int(rng.integers(0, 1 << 30)), 0.3, 20, 0.03)
        th = rng.uniform(-math.pi / 2 + 0.02, -0.1, n_angles)
        out.append(dict(obstacle=obs, N=n, omega=omega, d=1.0, thetas=th))
    return out


def workload_serving(seed: int = 0, count: int = 32, n_lo: int = 2000, n_hi: int = 100000, w_lo: float = 10.0,
                     w_hi: float = 60.0):
    """Resident geometries for the request loop: alternating wiggly and star obstacles with N
    log-uniform in [n_lo, n_hi] (rounded to a multiple of 8) and omega uniform in [w_lo, w_hi].
    Returns a list of dicts (obstacle, N, omega, d)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))) / 8.0)) * 8
        omega = float(rng.uniform(w_lo, w_hi))
        if i % 2 == 0:
            obs = wiggly(int(rng.integers(0, 1 << 30)), 0.3, 40, 0.04)
        else:
            obs = star(float(rng.uniform(0.2, 0.3)), float(rng.uniform(0.1, 0.3)), int(rng.integers(3, 7)))
        out.append(dict(obstacle=obs, N=n, omega=omega, d=1.0))
    return out


def request_stream(seed: int, count: int, rate_per_s: float, omegas, d: float = 1.0, wood_frac: float = 0.1):
    """A Poisson stream of single-angle requests over the geometries with wavenumbers `omegas`:
    arrival times (s, exponential gaps of mean 1/rate), geometry index (uniform), and angle:
    uniform in (-pi + 0.05, -0.05), except a fraction wood_frac placed exactly at a
    Rayleigh-Wood anomaly of the geometry, cos(theta) = 1 - 2 pi n / (omega d).  Returns
    (times, geometry indices, angles) as numpy arrays."""
    rng = np.random.default_rng(seed)
    times = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    gi = rng.integers(0, len(omegas), size=count)
    th = rng.uniform(-math.pi + 0.05, -0.05, size=count)
    for i in np.flatnonzero(rng.random(count) < wood_frac):
        om = float(omegas[gi[i]])
        orders = [n for n in range(1, 64) if 1.0 - 2.0 * math.pi * n / (om * d) > -1.0]
        n = int(rng.choice(orders))
        th[i] = -math.acos(1.0 - 2.0 * math.pi * n / (om * d))
    return times, gi, th
