"""Dense FP64 oracle for the quasi-periodic Dirichlet grating problem.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg call
it.  It shares no code with the CUDA path.

What it computes is the plain definition of the discrete problem: the
extended Nystrom system of Eq. (block2),

    [ A~  B ] [eta]   [b]
    [ C~  Q ] [xi ] = [0],     A~ = A + alpha A_1 + alpha^{-1} A_{-1}   (P = 1),

filled densely with exact neighbour blocks A_{+-1} (no interpolative
decomposition, no hierarchical compression), optionally extended by one
unknown and one row per Rayleigh-Bloch mode whose pole the Sommerfeld contour
was moved across (Sec. 2.4, Wood's anomalies), solved with LAPACK zgesv
(scipy.linalg.solve), followed by Bragg-amplitude extraction (Remarks 2.2,
2.3) and the flux balance (Sec. 6, error-measure remark).

Where the paper is silent, garbled or inconsistent this module takes the
following readings (each is also listed with its pin in the design notes):

* Eq. for A_nm (Sec. 2.3) omits the identity term of A = I/2 + D - i w S
  (Sec. 2.2); the 1/2 is added on the diagonal.  Normals point out of the
  obstacle (counter-clockwise parametrisation); R_{|n-m|} uses the circular
  index distance.
* The printed Q (Eq. Q) is not what the stated representation (urep) and wall
  conditions (f), (fn) give: re-deriving the Fourier coefficients of the wall
  potentials on L and R yields, per contour node k with s = sqrt(w^2 - k^2),
  e = exp(i s d), rows [f; fn] and columns [mu; nu]:
        [ e i (a - 1/a) / (2 s)       1 - e (a + 1/a) / 2 ]
        [ -1 + e (a + 1/a) / 2        e i s (a - 1/a) / 2 ]
  whose determinant (1 - e a)(1 - e / a) vanishes exactly at the Rayleigh-Bloch
  poles k = +-k_n named in Sec. 2.4.  This form is used.
* C~ (Sec. 2.4) names image -(P+1) at wall R; with P = 0 that does not reduce
  to Eq. (C).  Translating the images shows the discrepancy of the image sum is
  alpha^P Phi_P(L) - alpha^{-(P+1)} Phi_{-P}(R); that is used.
* Sommerfeld contour (Sec. 2.3, details deferred to a missing reference):
  k(t) = t - i c tanh((t - t0)/w), trapezoid rule in t with spacing h on
  M nodes symmetric about t0, sqrt(w^2 - k^2) = sqrt(w - k) sqrt(w + k).
* Wood's anomalies (Sec. 2.4): moving the crossing point to t0 > 0 flips the
  poles +k_n lying between the two contours; per flipped mode one unknown
  multiplies the plane wave exp(i(kappa_n x + k_n y)) (exactly quasi-periodic,
  so it adds nothing to the wall rows) and one row demands that the mode have
  no incoming part below the grating: i k_n u^_n + (u_y)^_n = 0 at y = -y0.
* Bragg extraction: u, u_y are sampled at S_s points x_s = -d/2 + (s + 1/2) d/S_s
  on y = +-y0 and transformed by the DFT; c_n, d_n are the mode-n coefficients
  of u at +y0 and -y0.
* Flux balance for unit incident amplitude (the cited Eq. 4.2 is missing):
  sum_n (k_n / k_0) (|c_n|^2 + |d_n + delta_{n0} exp(i k_0 y0)|^2) = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.special

from . import kr6


# --------------------------------------------------------------------------
# Geometry and quadrature (Sec. 2.3)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Boundary:
    x: np.ndarray
    y: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    speed: np.ndarray
    w: np.ndarray  # trapezoid weights (2 pi / N) |z'(t_j)|

    @property
    def n(self) -> int:
        return len(self.x)


def boundary(x, y, dx, dy) -> Boundary:
    """Nodes y_j = z(2 pi j/N), outward normals (counter-clockwise curve), speeds and
    periodic trapezoid weights (Sec. 2.3)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    sp = np.hypot(dx, dy)
    n = len(x)
    return Boundary(x, y, dy / sp, -dx / sp, sp, (2.0 * math.pi / n) * sp)


# --------------------------------------------------------------------------
# Kernels (Eqs. S, D, G)
# --------------------------------------------------------------------------

def green(tx, ty, sx, sy, omega):
    """G(x, y) = (i/4) H0^(1)(omega |x - y|) for target/source arrays (broadcast)."""
    r = np.hypot(tx - sx, ty - sy)
    return 0.25j * scipy.special.hankel1(0, omega * r)


def combined(tx, ty, sx, sy, snx, sny, omega):
    """Combined-field kernel dG/dn_y - i omega G of the representation (urep)."""
    ddx = tx - sx
    ddy = ty - sy
    r = np.hypot(ddx, ddy)
    h0 = scipy.special.hankel1(0, omega * r)
    h1 = scipy.special.hankel1(1, omega * r)
    dgdn = 0.25j * omega * h1 * (ddx * snx + ddy * sny) / r
    return dgdn - 1j * omega * 0.25j * h0


def combined_grad(tx, ty, sx, sy, snx, sny, omega):
    """Gradient with respect to the target point of the combined kernel.

    With f(r) = (i/4) H0(omega r): f' = -(i omega/4) H1, f'' = -(i omega^2/4)(H0 - H1/(omega r)).
    G = f(r), dG/dn_y = -(f'/r) d.n (d = x - y), so
      d/dx_i [dG/dn_y] = -g'(r) (d_i/r)(d.n) - g(r) n_i,   g = f'/r,  g' = (f'' - f'/r)/r,
      d/dx_i [G]        = g(r) d_i.
    """
    ddx = tx - sx
    ddy = ty - sy
    r = np.hypot(ddx, ddy)
    z = omega * r
    h0 = scipy.special.hankel1(0, z)
    h1 = scipy.special.hankel1(1, z)
    f1 = -0.25j * omega * h1
    f2 = -0.25j * omega * omega * (h0 - h1 / z)
    g = f1 / r
    gp = (f2 - f1 / r) / r
    dn = ddx * snx + ddy * sny
    kx = -gp * (ddx / r) * dn - g * snx - 1j * omega * g * ddx
    ky = -gp * (ddy / r) * dn - g * sny - 1j * omega * g * ddy
    return kx, ky


# --------------------------------------------------------------------------
# The N x N blocks (Sec. 2.3, Sec. 2.4)
# --------------------------------------------------------------------------

def matrix_a(bd: Boundary, omega: float) -> np.ndarray:
    """A_nm = delta_nm/2 + (2 pi/N) R_{|n-m|} [dG/dn_y - i w G](y_n, y_m) |z'(t_m)| (Sec. 2.3)."""
    n = bd.n
    idx = np.arange(n)
    dist = np.abs(idx[:, None] - idx[None, :])
    dist = np.minimum(dist, n - dist)
    rw = kr6.weights(n)[dist]
    with np.errstate(divide="ignore", invalid="ignore"):
        k = combined(bd.x[:, None], bd.y[:, None], bd.x[None, :], bd.y[None, :],
                     bd.nx[None, :], bd.ny[None, :], omega)
    k[idx, idx] = 0.0
    a = rw * k * bd.w[None, :]
    a[idx, idx] += 0.5
    return a


def matrix_a_image(bd: Boundary, omega: float, d: float, j: int) -> np.ndarray:
    """A_j: effect on the obstacle of the image obstacle shifted by j d (Sec. 2.4), plain
    trapezoid weights (the image is well separated)."""
    return combined(bd.x[:, None], bd.y[:, None], bd.x[None, :] + j * d, bd.y[None, :],
                    bd.nx[None, :], bd.ny[None, :], omega) * bd.w[None, :]


# --------------------------------------------------------------------------
# Sommerfeld contour (Sec. 2.3)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Contour:
    k: np.ndarray   # complex nodes
    wk: np.ndarray  # complex weights dk
    t0: float
    c: float
    w: float
    h: float

    @property
    def m(self) -> int:
        return len(self.k)


def contour(m: int, h: float, c: float = 1.0, w: float = 1.0, t0: float = 0.0) -> Contour:
    """k(t) = t - i c tanh((t - t0)/w); trapezoid nodes t = t0 + (j - (m-1)/2) h."""
    t = t0 + (np.arange(m) - 0.5 * (m - 1)) * h
    u = (t - t0) / w
    k = t - 1j * c * np.tanh(u)
    wk = h * (1.0 - 1j * (c / w) / np.cosh(u) ** 2)
    return Contour(k, wk, t0, c, w, h)


def sqrt_branch(omega, k):
    """sqrt(omega^2 - k^2) with cuts (-inf,-omega) u (omega,inf): non-negative real or
    positive imaginary on the real axis (Sec. 2.2)."""
    return np.sqrt(omega - k) * np.sqrt(omega + k)


# --------------------------------------------------------------------------
# Periodizing blocks B, C~, Q (Eqs. B, C, Q; Sec. 2.4)
# --------------------------------------------------------------------------

def wall_field_rows(tx, ty, ct: Contour, omega, d, deriv=None):
    """Field at targets (tx, ty) inside the unit cell of unit Fourier densities at each
    contour node, for the four wall potentials (Eqs. Sh, Dh):

    returns SL, SR, DL, DR (targets x M), already multiplied by the contour weights.
    deriv in (None, 'x', 'y') selects u, u_x or u_y.  Inside the cell
    sign(x - x_L) = +1 and sign(x - x_R) = -1.
    """
    tx = np.asarray(tx, dtype=np.float64)[:, None]
    ty = np.asarray(ty, dtype=np.float64)[:, None]
    k = ct.k[None, :]
    s = sqrt_branch(omega, k)
    el = np.exp(1j * k * ty) * np.exp(1j * s * (tx + 0.5 * d))
    er = np.exp(1j * k * ty) * np.exp(1j * s * (0.5 * d - tx))
    sl = 0.5j * el / s
    sr = 0.5j * er / s
    dl = 0.5 * el
    dr = -0.5 * er
    if deriv == "y":
        sl, sr, dl, dr = (1j * k * v for v in (sl, sr, dl, dr))
    elif deriv == "x":
        # d/dx exp(i s |x - x0|) = i s sign(x - x0) exp(...)
        sl, dl = 1j * s * sl, 1j * s * dl
        sr, dr = -1j * s * sr, -1j * s * dr
    wk = ct.wk[None, :]
    return sl * wk, sr * wk, dl * wk, dr * wk


def matrix_b_parts(bd: Boundary, ct: Contour, omega, d):
    """B = B_L + alpha B_R (Eq. B) with B_X = [S^_{dOmega,X} | D^_{dOmega,X}] (N x 2M)."""
    sl, sr, dl, dr = wall_field_rows(bd.x, bd.y, ct, omega, d)
    return np.hstack([sl, dl]), np.hstack([sr, dr])


def wall_fourier_parts(sx, sy, snx, sny, ct: Contour, omega, x0):
    """Fourier transforms at the contour nodes (M x sources) of the wall data of a
    single-layer source (value S^, x-derivative D*^) and of a double-layer source (value
    D^, x-derivative T^) at (sx, sy) with normal (snx, sny), for the wall at x = x0
    (Sec. 2.2)."""
    k = ct.k[:, None]
    s = sqrt_branch(omega, k)
    sg = np.sign(sx - x0)[None, :]
    base = np.exp(-1j * k * sy[None, :]) * np.exp(1j * s * np.abs(sx - x0)[None, :]) / (4.0 * math.pi)
    s_hat = 1j * base / s
    d_hat = base * (-sg * snx[None, :] + (k / s) * sny[None, :])
    dstar_hat = base * sg
    t_hat = 1j * base * (s * snx[None, :] - k * sg * sny[None, :])
    return s_hat, d_hat, dstar_hat, t_hat


def wall_fourier_rows(sx, sy, snx, sny, sw, ct: Contour, omega, x0):
    """Fourier transform at the contour nodes of the wall discrepancy rows produced by
    combined-field sources (sx, sy) (Sec. 2.2, operators S^, D^, D*^, T^):

    f-row  = D^ - i w S^,   fn-row = T^ - i w D*^,  each 2M x N after stacking [f; fn],
    multiplied by the source weights sw.
    """
    s_hat, d_hat, dstar_hat, t_hat = wall_fourier_parts(sx, sy, snx, sny, ct, omega, x0)
    f = (d_hat - 1j * omega * s_hat) * sw[None, :]
    fn = (t_hat - 1j * omega * dstar_hat) * sw[None, :]
    return np.vstack([f, fn])


def matrix_c_parts(bd: Boundary, ct: Contour, omega, d, p: int = 1):
    """C~ = alpha^P C_L - alpha^{-(P+1)} C_R with C_L from image +P at wall L and C_R from
    image -P at wall R (Sec. 2.4, reading above)."""
    cl = wall_fourier_rows(bd.x + p * d, bd.y, bd.nx, bd.ny, bd.w, ct, omega, -0.5 * d)
    cr = wall_fourier_rows(bd.x - p * d, bd.y, bd.nx, bd.ny, bd.w, ct, omega, 0.5 * d)
    return cl, cr


def matrix_q(ct: Contour, omega, d, alpha) -> np.ndarray:
    """Q (2M x 2M): four diagonal blocks, derived from (urep) and (f), (fn) (reading above)."""
    s = sqrt_branch(omega, ct.k)
    e = np.exp(1j * s * d)
    ap = alpha + 1.0 / alpha
    am = alpha - 1.0 / alpha
    m = ct.m
    q = np.zeros((2 * m, 2 * m), dtype=np.complex128)
    i = np.arange(m)
    q[i, i] = e * 1j * am / (2.0 * s)
    q[i, m + i] = 1.0 - e * ap / 2.0
    q[m + i, i] = -1.0 + e * ap / 2.0
    q[m + i, m + i] = e * 1j * s * am / 2.0
    return q


# --------------------------------------------------------------------------
# Rayleigh-Bloch modes and Wood's anomalies (Secs. 2.1, 2.4)
# --------------------------------------------------------------------------

def kappa_n(omega, d, theta, n):
    return omega * math.cos(theta) + 2.0 * math.pi * np.asarray(n) / d


def k_n(omega, kappa):
    """k_n = +sqrt(omega^2 - kappa_n^2), non-negative real or positive imaginary.  An order
    within rounding of a Rayleigh-Wood anomaly, |omega^2 - kappa_n^2| <= 1e-12 omega^2, is
    taken at the anomaly (k_n = 0): an angle given as the anomaly in FP64 is only that close
    to it, and the amplitudes have a square-root singularity in the angle there (reading of
    Sec. 2.4 for exact anomalies)."""
    kappa = np.asarray(kappa, dtype=np.complex128)
    v = omega * omega - kappa * kappa
    v = np.where(np.abs(v) <= 1e-12 * omega * omega, 0.0, v)
    return np.sqrt(v)


def mode_range(omega, d, theta, extra: int = 0):
    """Indices n of propagating orders |kappa_n| <= omega, widened by `extra` on each side."""
    ki = omega * math.cos(theta)
    nmin = math.ceil((-omega - ki) * d / (2.0 * math.pi))
    nmax = math.floor((omega - ki) * d / (2.0 * math.pi))
    return np.arange(nmin - extra, nmax + extra + 1)


def flipped_modes(omega, d, theta, ct: Contour):
    """Modes n whose pole +k_n lies between the standard contour (crossing 0) and `ct`
    (crossing t0 > 0): real 0 <= k_n < t0, or imaginary k_n with |k_n| < c tanh(t0/w)."""
    if ct.t0 <= 0.0:
        return np.zeros(0, dtype=np.int64)
    ns = mode_range(omega, d, theta, extra=4)
    kn = k_n(omega, kappa_n(omega, d, theta, ns))
    height = ct.c * math.tanh(ct.t0 / ct.w)
    out = []
    for n, kv in zip(ns, kn):
        if abs(kv.imag) < 1e-300 or kv.imag == 0.0:
            if 0.0 <= kv.real < ct.t0:
                out.append(n)
        elif kv.real == 0.0 and kv.imag < height:
            out.append(n)
    return np.array(out, dtype=np.int64)


# --------------------------------------------------------------------------
# Field evaluation and Bragg extraction (Remarks 2.2, 2.3)
# --------------------------------------------------------------------------

def eval_rows(tx, ty, bd: Boundary, ct: Contour, omega, d, alpha, p: int = 1, deriv=None):
    """Rows mapping (eta, xi) to u (or u_x, u_y) at the targets, for the representation
    (urepP): sum_{j=-P}^{P} alpha^j (D - i w S)_{dOmega + j d} eta + wall potentials."""
    tx = np.asarray(tx, dtype=np.float64)
    ty = np.asarray(ty, dtype=np.float64)
    rows_eta = np.zeros((len(tx), bd.n), dtype=np.complex128)
    for j in range(-p, p + 1):
        sx = bd.x[None, :] + j * d
        if deriv is None:
            kk = combined(tx[:, None], ty[:, None], sx, bd.y[None, :], bd.nx[None, :],
                          bd.ny[None, :], omega)
        else:
            kx, ky = combined_grad(tx[:, None], ty[:, None], sx, bd.y[None, :],
                                   bd.nx[None, :], bd.ny[None, :], omega)
            kk = kx if deriv == "x" else ky
        rows_eta += (alpha ** j) * kk * bd.w[None, :]
    sl, sr, dl, dr = wall_field_rows(tx, ty, ct, omega, d, deriv)
    rows_xi = np.hstack([sl + alpha * sr, dl + alpha * dr])
    return rows_eta, rows_xi


def plane_wave(tx, ty, kappa, kn, deriv=None):
    v = np.exp(1j * (kappa * np.asarray(tx) + kn * np.asarray(ty)))
    if deriv == "y":
        return 1j * kn * v
    if deriv == "x":
        return 1j * kappa * v
    return v


@dataclasses.dataclass
class Options:
    m: int = 120
    h: float = 0.5
    c: float = 1.0
    w: float = 1.0
    t0: float = 0.0
    p: int = 1
    n_samples: int = 64
    y0: float | None = None


@dataclasses.dataclass
class Solution:
    eta: np.ndarray
    xi: np.ndarray
    wood_coef: np.ndarray
    wood_modes: np.ndarray
    orders: np.ndarray   # propagating n
    c: np.ndarray        # upward Bragg amplitudes
    d: np.ndarray        # downward Bragg amplitudes
    flux_error: float
    y0: float
    alpha: complex


def default_y0(bd: Boundary, d: float) -> float:
    return float(np.max(np.abs(bd.y))) + 0.25 * d


def sample_points(d, n_samples):
    return -0.5 * d + (np.arange(n_samples) + 0.5) * d / n_samples


def dft_rows(xs, kappa):
    """Rows of the DFT u^_n = (1/S) sum_s u(x_s) exp(-i kappa_n x_s)."""
    return np.exp(-1j * np.outer(kappa, xs)) / len(xs)


def obstacle_blocks(x, y, dx, dy, omega: float, d: float, p: int = 1, quadrature: str = "kr6"):
    """The angle-independent N x N blocks: A and the neighbour images A_j, 0 < |j| <= P.
    Passing them to dense_solve for several angles of one obstacle saves refilling them.
    quadrature "kr6" (Sec. 2.3, the paper's) or "kress" (oracle/kress.py, a second
    discretization of the same operator, used to pin the first) for the log-singular A."""
    bd = boundary(x, y, dx, dy)
    imgs = {j: matrix_a_image(bd, omega, d, j) for j in range(-p, p + 1) if j != 0}
    if quadrature == "kress":
        from . import kress
        return kress.matrix_a(x, y, dx, dy, omega), imgs
    if quadrature != "kr6":
        raise ValueError(quadrature)
    return matrix_a(bd, omega), imgs


def dense_solve(x, y, dx, dy, omega: float, d: float, theta: float, opts: Options,
                blocks=None) -> Solution:
    """Fill and solve Eq. (block2) (plus Wood's rows) densely, then extract Bragg
    amplitudes and the flux error.  This is the oracle's answer for one angle.
    `blocks` = obstacle_blocks(...) of the same obstacle, omega, d and P, or None."""
    bd = boundary(x, y, dx, dy)
    alpha = np.exp(1j * omega * d * math.cos(theta))
    ct = contour(opts.m, opts.h, opts.c, opts.w, opts.t0)
    y0 = opts.y0 if opts.y0 is not None else default_y0(bd, d)
    p = opts.p

    a0, imgs = blocks if blocks is not None else obstacle_blocks(x, y, dx, dy, omega, d, p)
    a = a0.copy()
    for j in range(-p, p + 1):
        if j != 0:
            a += (alpha ** j) * imgs[j]
    bl, br = matrix_b_parts(bd, ct, omega, d)
    b = bl + alpha * br
    cl, cr = matrix_c_parts(bd, ct, omega, d, p)
    c = (alpha ** p) * cl - alpha ** (-(p + 1)) * cr
    q = matrix_q(ct, omega, d, alpha)

    ki = omega * math.cos(theta)
    kiy = omega * math.sin(theta)
    rhs_b = -np.exp(1j * (ki * bd.x + kiy * bd.y))

    wood = flipped_modes(omega, d, theta, ct)
    nw = len(wood)
    nn, m2 = bd.n, 2 * ct.m
    size = nn + m2 + nw
    big = np.zeros((size, size), dtype=np.complex128)
    big[:nn, :nn] = a
    big[:nn, nn:nn + m2] = b
    big[nn:nn + m2, :nn] = c
    big[nn:nn + m2, nn:nn + m2] = q
    xs = sample_points(d, opts.n_samples)
    ys_lo = np.full_like(xs, -y0)
    if nw:
        kap_w = kappa_n(omega, d, theta, wood)
        kn_w = k_n(omega, kap_w)
        u_eta, u_xi = eval_rows(xs, ys_lo, bd, ct, omega, d, alpha, p)
        uy_eta, uy_xi = eval_rows(xs, ys_lo, bd, ct, omega, d, alpha, p, deriv="y")
        for i, (kap, kn) in enumerate(zip(kap_w, kn_w)):
            col = nn + m2 + i
            big[:nn, col] = plane_wave(bd.x, bd.y, kap, kn)
            f = dft_rows(xs, np.array([kap]))[0]
            row = nn + m2 + i
            big[row, :nn] = 1j * kn * (f @ u_eta) + f @ uy_eta
            big[row, nn:nn + m2] = 1j * kn * (f @ u_xi) + f @ uy_xi
            for i2, (kap2, kn2) in enumerate(zip(kap_w, kn_w)):
                pw = plane_wave(xs, ys_lo, kap2, kn2)
                pwy = plane_wave(xs, ys_lo, kap2, kn2, deriv="y")
                big[row, nn + m2 + i2] = 1j * kn * (f @ pw) + f @ pwy
    rhs = np.zeros(size, dtype=np.complex128)
    rhs[:nn] = rhs_b
    sol = scipy.linalg.solve(big, rhs)
    eta = sol[:nn]
    xi = sol[nn:nn + m2]
    wc = sol[nn + m2:]
    return bragg(bd, ct, omega, d, theta, alpha, eta, xi, wood, wc, y0, opts.n_samples, p)


def bragg(bd, ct, omega, d, theta, alpha, eta, xi, wood, wc, y0, n_samples, p=1) -> Solution:
    """Bragg amplitudes c_n, d_n of the propagating orders and the flux error."""
    xs = sample_points(d, n_samples)
    orders = mode_range(omega, d, theta)
    kap = kappa_n(omega, d, theta, orders)
    f = dft_rows(xs, kap)
    out = []
    for ysign in (+1.0, -1.0):
        ys = np.full_like(xs, ysign * y0)
        r_eta, r_xi = eval_rows(xs, ys, bd, ct, omega, d, alpha, p)
        u = r_eta @ eta + r_xi @ xi
        for i, n in enumerate(wood):
            kw = kappa_n(omega, d, theta, n)
            u = u + wc[i] * plane_wave(xs, ys, kw, k_n(omega, kw))
        out.append(f @ u)
    cn, dn = out
    kn = k_n(omega, kap).real
    k0 = omega * abs(math.sin(theta))
    inc = np.where(orders == 0, np.exp(1j * k0 * y0), 0.0)
    flux = float(np.sum((kn / k0) * (np.abs(cn) ** 2 + np.abs(dn + inc) ** 2)))
    return Solution(eta, xi, wc, wood, orders, cn, dn, abs(flux - 1.0), y0, alpha)


def bragg_vector(sol: Solution) -> np.ndarray:
    """All propagating amplitudes (c_n then d_n) as one vector, for relative-error checks."""
    return np.concatenate([sol.c, sol.d])


def a_rows(bd: Boundary, omega: float, rows) -> np.ndarray:
    """Selected rows of A (Sec. 2.3), each evaluated directly: delta/2 + (2 pi/N) R_{|n-m|} K w."""
    rows = np.asarray(rows, dtype=np.int64)
    n = bd.n
    idx = np.arange(n)
    out = np.zeros((len(rows), n), dtype=np.complex128)
    rw_all = kr6.weights(n)
    for t, i in enumerate(rows):
        dist = np.abs(idx - i)
        dist = np.minimum(dist, n - dist)
        with np.errstate(divide="ignore", invalid="ignore"):
            k = combined(bd.x[i], bd.y[i], bd.x, bd.y, bd.nx, bd.ny, omega)
        k[i] = 0.0
        out[t] = rw_all[dist] * k * bd.w
        out[t, i] += 0.5
    return out
