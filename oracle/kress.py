"""Kress's spectral quadrature for the combined-field matrix A (oracle side; test infrastructure).

A second, independent discretization of the same boundary integral operator
A = I/2 + D - i w S of Secs. 2.2-2.3, used only to pin the Kapur-Rokhlin (KR6)
discretization that the paper and the library use: both must give the same Bragg
amplitudes once converged in N.

On N = 2n equispaced parameter points t_j = pi j / n, the kernel of A in the parameter,
K(t, tau) = [dG/dn_y - i w G](z(t), z(tau)) |z'(tau)|, is split as
    K(t, tau) = K1(t, tau) log(4 sin^2((t - tau)/2)) + K2(t, tau)
with K1, K2 smooth (Bessel's J0, J1 carry the logarithms of Y0, Y1):
    G part:   M1 = -(1/4pi) J0(w r) |z'|,
              M2(t, t) = [i/4 - (gamma + log(w |z'(t)| / 2)) / 2pi] |z'(t)|
    dG/dn_y:  L1 = -(w/4pi) J1(w r) [(x1 - y1) z2'(tau) - (x2 - y2) z1'(tau)] / r,  L1(t, t) = 0,
              L2(t, t) = (z1'' z2' - z2'' z1')(t) / (4 pi |z'(t)|^2)
and the log part is integrated exactly against trigonometric interpolation (Kress's weights)
    R_j(t) = -(2 pi / n) sum_{m=1}^{n-1} cos(m (t - t_j)) / m - (pi / n^2) cos(n (t - t_j)),
the smooth part by the trapezoid rule:
    A_ij = delta_ij / 2 + R_j(t_i) K1(t_i, t_j) + (pi / n) K2(t_i, t_j).
z'' is obtained from the samples of z' by spectral differentiation.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

EULER_GAMMA = 0.57721566490153286061


def kress_weights(n_points: int) -> np.ndarray:
    """R(t_i - t_j) as a function of the index difference k = i - j (mod N), length N."""
    if n_points % 2:
        raise ValueError("Kress's rule needs an even number of points")
    n = n_points // 2
    k = np.arange(n_points)
    dt = math.pi * k / n
    m = np.arange(1, n)
    r = -(2.0 * math.pi / n) * np.sum(np.cos(np.outer(dt, m)) / m[None, :], axis=1)
    return r - (math.pi / n ** 2) * np.cos(n * dt)


def spectral_derivative(f: np.ndarray) -> np.ndarray:
    """d/dt of a 2 pi-periodic function sampled at t_j = 2 pi j / N (Nyquist mode dropped)."""
    n = len(f)
    k = np.fft.fftfreq(n, d=1.0 / n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return np.real(np.fft.ifft(1j * k * np.fft.fft(f)))


def matrix_a(x, y, dx, dy, omega: float) -> np.ndarray:
    """A = I/2 + D - i w S on the N nodes by Kress's quadrature (module docstring)."""
    x, y, dx, dy = (np.asarray(a, dtype=np.float64) for a in (x, y, dx, dy))
    npts = len(x)
    ddx, ddy = spectral_derivative(dx), spectral_derivative(dy)
    speed = np.hypot(dx, dy)
    idx = np.arange(npts)
    diff = (idx[:, None] - idx[None, :]) % npts
    t = 2.0 * math.pi * idx / npts
    logs = np.zeros((npts, npts))
    off = diff != 0
    logs[off] = np.log(4.0 * np.sin(0.5 * (t[:, None] - t[None, :])[off]) ** 2)
    d1 = x[:, None] - x[None, :]
    d2 = y[:, None] - y[None, :]
    r = np.hypot(d1, d2)
    r[~off] = 1.0
    z = omega * r
    j0, j1 = scipy.special.j0(z), scipy.special.j1(z)
    h0, h1 = scipy.special.hankel1(0, z), scipy.special.hankel1(1, z)
    cross = d1 * dy[None, :] - d2 * dx[None, :]          # (x - y) . n_y |z'(tau)|
    m1 = -j0 * speed[None, :] / (4.0 * math.pi)
    m_full = 0.25j * h0 * speed[None, :]
    l1 = -(omega / (4.0 * math.pi)) * j1 * cross / r
    l_full = 0.25j * omega * h1 * cross / r
    m2 = m_full - m1 * logs
    l2 = l_full - l1 * logs
    dg = ~off
    m1[dg] = -speed / (4.0 * math.pi)
    m2[dg] = (0.25j - (EULER_GAMMA + np.log(0.5 * omega * speed)) / (2.0 * math.pi)) * speed
    l1[dg] = 0.0
    l2[dg] = (ddx * dy - ddy * dx) / (4.0 * math.pi * speed ** 2)
    k1 = l1 - 1j * omega * m1
    k2 = l2 - 1j * omega * m2
    a = kress_weights(npts)[diff] * k1 + (2.0 * math.pi / npts) * k2
    a[idx, idx] += 0.5
    return a
