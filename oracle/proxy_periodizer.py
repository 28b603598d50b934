"""A second periodizing scheme: proxy points and wall discrepancies (oracle side; test
infrastructure).

The paper periodizes with Sommerfeld-contour wall potentials (Secs. 2.2-2.4) and names no
other scheme; its conclusion (Sec. 7) points to a cited one for wall-crossing gratings.
This module solves the same quasi-periodic Dirichlet problem with a different
representation of the far images, so that the two schemes' Bragg amplitudes pin each
other: they discretize one continuum problem two ways.

Reading used here (the box scheme of the proxy-point method family):

* Box.  The unit cell is cut to the rectangle |x| <= d/2, |y| <= h, h = max|y| + d/8 on
  the obstacle.  Inside it the scattered field is
      u = sum_{|j| <= 1} alpha^j (D - i w S)_{dOmega + j d} eta  +  sum_p c_p phi_p,
  where phi_p = dG/dn_p - i w G is a combined-field source at proxy point z_p on a circle
  of radius R_p = max(0.75 d, 1.4 * half-diagonal of the box) around the cell centre (outward
  normal n_p), M_p = max(100, 2 ceil(w R_p) + 60) points.  The proxies stand for all
  images |j| >= 2 (and anything else outside the box).
* Equations, all in the least-squares sense (the system is consistent):
  - on dOmega: u = -u_inc (N rows: A~ eta + Phi c with A~ = A + alpha A_1 + alpha^{-1} A_{-1});
  - on the walls at M_w = 40 Gauss-Legendre heights y_k in [-h, h]: the discrepancies
    u(-d/2, y_k) - alpha^{-1} u(d/2, y_k) = 0 and the same for u_x.  The images telescope:
    their part is alpha Phi_1(L) - alpha^{-2} Phi_{-1}(R) (Sec. 2.4's reading R4);
  - on the lines y = +h and y = -h at M_t equispaced x_k = -d/2 + (k + 1/2) d/M_t, the
    field and its y-derivative equal those of outgoing Rayleigh-Bloch expansions
    sum_{|n| <= K} a_n e^{i(kappa_n x + k_n (y - h))} above and
    sum b_n e^{i(kappa_n x - k_n (y + h))} below, K = ceil(w d / pi) + 40 (every propagating
    order of any angle and 40 evanescent ones, which have decayed by exp(-2 pi 40 / 8) ~ 1e-14
    from the obstacle to the lines), M_t = 2 (2K + 1) + 8.
* The Bragg amplitudes are a_n and b_n of the propagating orders, referred to y = +-h; at
  another height y0 they are a_n e^{i k_n (y0 - h)} and b_n e^{i k_n (y0 - h)}.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg

from . import qp_dense as qd


@dataclasses.dataclass
class ProxyOptions:
    h: float | None = None          # box half-height (default max|y| + d/8)
    r_proxy: float | None = None    # proxy circle radius
    m_proxy: int | None = None
    m_wall: int = 40
    k_modes: int | None = None
    m_line: int | None = None


@dataclasses.dataclass
class ProxySolution:
    orders: np.ndarray
    a: np.ndarray        # all 2K+1 coefficients above
    b: np.ndarray        # below
    modes: np.ndarray    # n = -K..K
    c: np.ndarray        # propagating a_n, referred to y = +h
    d: np.ndarray        # propagating b_n, referred to y = -h
    h: float
    residual: float      # relative least-squares residual


def resolved(x, y, omega, d, theta, o: ProxyOptions):
    """The scheme's sizes for one obstacle (the reading in the module docstring)."""
    h = o.h if o.h is not None else float(np.max(np.abs(y))) + d / 8.0
    half_diag = math.hypot(0.5 * d, h)
    rp = o.r_proxy if o.r_proxy is not None else max(0.75 * d, 1.4 * half_diag)
    mp = o.m_proxy if o.m_proxy is not None else max(100, 2 * int(math.ceil(omega * rp)) + 60)
    # every propagating order of any angle, |n| <= omega d / pi, and 40 evanescent ones beyond:
    # the obstacle sits d/8 below the lines, so mode n decays like exp(-2 pi |n| / 8) there
    kk = o.k_modes if o.k_modes is not None else int(math.ceil(omega * d / math.pi)) + 40
    mt = o.m_line if o.m_line is not None else 2 * (2 * kk + 1) + 8
    return h, rp, mp, kk, mt


def _proxy_field(tx, ty, px, py, pnx, pny, omega, deriv=None):
    """phi_p and its target derivatives at targets (rows) for proxies (columns)."""
    if deriv is None:
        return qd.combined(tx[:, None], ty[:, None], px[None, :], py[None, :], pnx[None, :], pny[None, :], omega)
    gx, gy = qd.combined_grad(tx[:, None], ty[:, None], px[None, :], py[None, :], pnx[None, :], pny[None, :], omega)
    return gx if deriv == "x" else gy


def _image_field(tx, ty, bd, omega, d, j, deriv=None):
    """Field at targets of the image j d of the combined-field layer (rows x N), trapezoid weights."""
    sx = bd.x[None, :] + j * d
    if deriv is None:
        k = qd.combined(tx[:, None], ty[:, None], sx, bd.y[None, :], bd.nx[None, :], bd.ny[None, :], omega)
    else:
        gx, gy = qd.combined_grad(tx[:, None], ty[:, None], sx, bd.y[None, :], bd.nx[None, :], bd.ny[None, :], omega)
        k = gx if deriv == "x" else gy
    return k * bd.w[None, :]


def solve(x, y, dx, dy, omega: float, d: float, theta: float, o: ProxyOptions | None = None,
          blocks=None) -> ProxySolution:
    """Fill the rectangular system of the reading above densely and solve it by LAPACK least
    squares; `blocks` = qp_dense.obstacle_blocks(...) of the same obstacle, or None."""
    o = o or ProxyOptions()
    bd = qd.boundary(x, y, dx, dy)
    alpha = np.exp(1j * omega * d * math.cos(theta))
    h, rp, mp, kk, mt = resolved(x, y, omega, d, theta, o)
    n = bd.n
    ang = 2.0 * math.pi * np.arange(mp) / mp
    px, py = rp * np.cos(ang), rp * np.sin(ang)
    pnx, pny = np.cos(ang), np.sin(ang)
    modes = np.arange(-kk, kk + 1)
    kap = qd.kappa_n(omega, d, theta, modes)
    kn = qd.k_n(omega, kap)

    a0, imgs = blocks if blocks is not None else qd.obstacle_blocks(x, y, dx, dy, omega, d)
    at = a0 + alpha * imgs[1] + imgs[-1] / alpha

    gy_nodes, _ = np.polynomial.legendre.leggauss(o.m_wall)
    yw = h * gy_nodes
    xl, xr = np.full_like(yw, -0.5 * d), np.full_like(yw, 0.5 * d)
    xt = -0.5 * d + (np.arange(mt) + 0.5) * d / mt

    nu = 2 * kk + 1
    ncol = n + mp + 2 * nu
    rows = []
    # dOmega
    r0 = np.zeros((n, ncol), dtype=np.complex128)
    r0[:, :n] = at
    r0[:, n:n + mp] = _proxy_field(bd.x, bd.y, px, py, pnx, pny, omega)
    rows.append(r0)
    # wall discrepancies of u and u_x
    for der in (None, "x"):
        r = np.zeros((o.m_wall, ncol), dtype=np.complex128)
        r[:, :n] = alpha * _image_field(xl, yw, bd, omega, d, 1, der) - _image_field(xr, yw, bd, omega, d, -1, der) / alpha ** 2
        r[:, n:n + mp] = (_proxy_field(xl, yw, px, py, pnx, pny, omega, der)
                          - _proxy_field(xr, yw, px, py, pnx, pny, omega, der) / alpha)
        rows.append(r)
    # matching on y = +h (a) and y = -h (b): u and u_y
    for sgn, off in ((1.0, n + mp), (-1.0, n + mp + nu)):
        yy = np.full_like(xt, sgn * h)
        ex = np.exp(1j * np.outer(xt, kap))
        for der in (None, "y"):
            r = np.zeros((mt, ncol), dtype=np.complex128)
            for j in (-1, 0, 1):
                r[:, :n] += (alpha ** j) * _image_field(xt, yy, bd, omega, d, j, der)
            r[:, n:n + mp] = _proxy_field(xt, yy, px, py, pnx, pny, omega, der)
            r[:, off:off + nu] = -(ex if der is None else ex * (1j * sgn * kn)[None, :])
            rows.append(r)
    big = np.vstack(rows)
    rhs = np.zeros(big.shape[0], dtype=np.complex128)
    rhs[:n] = -np.exp(1j * omega * (math.cos(theta) * bd.x + math.sin(theta) * bd.y))
    # equilibrate columns (proxy and mode columns differ in scale from the density's)
    scale = 1.0 / np.maximum(np.linalg.norm(big, axis=0), 1e-300)
    sol, *_ = scipy.linalg.lstsq(big * scale[None, :], rhs, lapack_driver="gelsd")
    sol = sol * scale
    res = float(np.linalg.norm(big @ sol - rhs) / np.linalg.norm(rhs))
    a = sol[n + mp:n + mp + nu]
    b = sol[n + mp + nu:]
    orders = qd.mode_range(omega, d, theta)
    sel = orders + kk
    return ProxySolution(orders, a, b, modes, a[sel], b[sel], h, res)


def bragg_at(sol: ProxySolution, omega, d, theta, y0):
    """(c_n, d_n) of the propagating orders referred to y = +-y0 (the Fourier-wall scheme's
    convention, Remark 2.2): a_n e^{i k_n (y0 - h)}, b_n e^{i k_n (y0 - h)}."""
    kn = qd.k_n(omega, qd.kappa_n(omega, d, theta, sol.orders)).real
    ph = np.exp(1j * kn * (y0 - sol.h))
    return sol.c * ph, sol.d * ph
