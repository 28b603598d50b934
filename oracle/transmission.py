"""Dense FP64 oracle for the quasi-periodic transmission problem (Sec. 5): a grating of
dielectric obstacles of refractive index n in a background of index 1.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the tests,
`__graft_entry__.smoke()` and the benchmark's CPU legs call it.  It shares no code with the
CUDA path.

Sec. 5 states the boundary value problem (pdein, pdeout, bcm, bcmn), names the
Mueller-Rokhlin pair of densities and the interlacing of the unknowns, and leaves the
operator itself to a cited paper that is not at hand.  The operator here is derived from the
jump relations of the layer potentials.  The readings:

* Representation.  With sigma a single-layer and tau a double-layer density on dOmega,
      u = S_w sigma + D_w tau        outside the obstacle (w = omega),
      u = S_nw sigma + D_nw tau      inside it,
  S_k, D_k being the layers (S), (D) with wavenumber k.  Outside, the quasi-periodic field
  adds the images 0 < |j| <= P of the same pair, weighted alpha^j, and the wall potentials of
  Sec. 2.4, exactly where the Dirichlet problem has its combined layer (D - i w S) eta.
  The inside field uses the obstacle's own pair only.
* Jump relations (normal out of the obstacle, + = outside): (D tau)^(+-) = K tau +- tau/2,
  d(S sigma)/dn^(+-) = K' sigma -+ sigma/2; S sigma and d(D tau)/dn are continuous (K, K',
  T: direct values of D, of dS/dn_x and of dD/dn_x).  The matching conditions (bcm),
  (bcmn) at boundary node p are then
      sigma row:  sigma - (K'_w - K'_nw) sigma - (T_w - T_nw) tau = + du_inc/dn,
      tau row:    tau + (S_w - S_nw) sigma + (K_w - K_nw) tau     = - u_inc.
  Every operator is a difference of two kernels in which the 1/r^2 of T and the log r of S
  cancel to at most a log r singularity: the identity plus a compact operator, as Sec. 5
  says.
* Scaling.  The sigma rows are divided by w and the single-layer density is carried as
  s = sigma / w, so that the field is u = w S s + D tau.  This is a diagonal similarity of
  the system above (the same fields and Bragg amplitudes); it balances the 2 x 2 blocks,
  whose T difference grows like w^2: on a wiggly obstacle at w = 30 (n = 1.3) the operator's
  condition number falls from 3557 to 24, at w = 60 from 9.3e4 to 61, the Dirichlet
  operator's own level.  Interpolative decompositions with a relative tolerance then resolve
  both kinds of rows alike.
* Row functionals.  The tau row of node p takes the value of a field at y_p, the sigma row
  minus its normal derivative divided by w.  Every outside contribution (images, wall
  potentials, Wood's plane waves) enters a row through its functional, and the right-hand
  side is minus the functional of u_inc.  The tau rows are the Dirichlet problem's rows.
* Interlacing (Sec. 5): unknowns [s_1; tau_1; s_2; tau_2; ...], rows in the same order
  (sigma row of node 1, tau row of node 1, ...).
* Quadrature: the Kapur-Rokhlin corrections of Sec. 2.3 on every kernel difference (each is
  of the form phi(s) log|s| + psi(s) with phi, psi smooth); the diagonal 2 x 2 blocks are
  the identity (R_0 = 0).  Images take plain trapezoid weights.
* Periodizer.  B holds the row functionals of the four wall potentials.  C~ holds the wall
  discrepancies of Sec. 2.4 for the pair: a sigma column contributes S^ to the f rows and
  D*^ to the fn rows, a tau column D^ and T^.  Q is unchanged (Sec. 5).
* Wood's anomalies, the Bragg extraction and the flux balance are the Dirichlet oracle's.
  For real n the obstacle absorbs nothing, so the flux still balances.
* Setting s = -i eta, tau = eta turns the pair into the combined layer (D - i w S) eta, so
  every outside row of this module reduces to the Dirichlet oracle's (a pin).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.special

from . import kr6
from . import proxy_periodizer as pp
from . import qp_dense as qd


# --------------------------------------------------------------------------
# Kernels of the pair (Eqs. S, D and their normal derivatives)
# --------------------------------------------------------------------------

def layer_values(tx, ty, sx, sy, snx, sny, k):
    """G = (i/4) H0(k r) and dG/dn_y = (i k/4) H1(k r) ((x - y).n_y)/r at targets x for
    sources y with normals n_y (broadcast)."""
    ddx, ddy = tx - sx, ty - sy
    r = np.hypot(ddx, ddy)
    z = k * r
    g = 0.25j * scipy.special.hankel1(0, z)
    dg = 0.25j * k * scipy.special.hankel1(1, z) * (ddx * snx + ddy * sny) / r
    return g, dg


def layer_gradients(tx, ty, sx, sy, snx, sny, k):
    """Target gradients of G and of dG/dn_y.  With d = x - y, H_j = H_j^(1)(k r):
        grad G       = -(i k/4) H1 d / r,
        grad dG/dn_y = (i k/4) [k H0 d (d.n_y)/r^2 + (H1/r)(n_y - 2 d (d.n_y)/r^2)]
    (H1' = H0 - H1/z).  Returns (Gx, Gy, Dx, Dy)."""
    ddx, ddy = tx - sx, ty - sy
    r = np.hypot(ddx, ddy)
    z = k * r
    h0 = scipy.special.hankel1(0, z)
    h1 = scipy.special.hankel1(1, z)
    cy = (ddx * snx + ddy * sny) / r
    gx = -0.25j * k * h1 * ddx / r
    gy = -0.25j * k * h1 * ddy / r
    a = 0.25j * k * k * h0 * cy / r          # multiplies d
    b = 0.25j * k * h1 / r                    # multiplies (n_y - 2 d (d.n_y)/r^2)
    dx_ = a * ddx + b * (snx - 2.0 * ddx * cy / r)
    dy_ = a * ddy + b * (sny - 2.0 * ddy * cy / r)
    return gx, gy, dx_, dy_


def boundary_kernels(bd: qd.Boundary, sx, k):
    """For targets the boundary nodes (rows) and sources the nodes shifted to sx (columns):
    S = G, D = dG/dn_y, K' = dG/dn_x and T = d^2 G/dn_x dn_y (N x N each)."""
    tx, ty = bd.x[:, None], bd.y[:, None]
    tnx, tny = bd.nx[:, None], bd.ny[:, None]
    sy, snx, sny = bd.y[None, :], bd.nx[None, :], bd.ny[None, :]
    s, d = layer_values(tx, ty, sx, sy, snx, sny, k)
    gx, gy, dx_, dy_ = layer_gradients(tx, ty, sx, sy, snx, sny, k)
    return s, d, tnx * gx + tny * gy, tnx * dx_ + tny * dy_


def interlace_rows(sigma_rows, tau_rows):
    """[sigma row 1; tau row 1; sigma row 2; ...] from two row blocks of equal shape."""
    out = np.empty((2 * sigma_rows.shape[0],) + sigma_rows.shape[1:], dtype=np.complex128)
    out[0::2] = sigma_rows
    out[1::2] = tau_rows
    return out


def interlace_cols(sigma_cols, tau_cols):
    out = np.empty(sigma_cols.shape[:-1] + (2 * sigma_cols.shape[-1],), dtype=np.complex128)
    out[..., 0::2] = sigma_cols
    out[..., 1::2] = tau_cols
    return out


def row_functional(bd: qd.Boundary, omega, value, gx, gy):
    """Rows of a field sampled at the boundary nodes: sigma row = -(du/dn)/w, tau row = u."""
    nx = bd.nx.reshape((-1,) + (1,) * (np.ndim(value) - 1))
    ny = bd.ny.reshape((-1,) + (1,) * (np.ndim(value) - 1))
    return interlace_rows(-(nx * gx + ny * gy) / omega, value)


# --------------------------------------------------------------------------
# The 2N x 2N blocks
# --------------------------------------------------------------------------

def matrix_a(bd: qd.Boundary, omega: float, index: float) -> np.ndarray:
    """The Mueller-type operator of the reading above on one obstacle, interlaced and scaled,
    with the Kapur-Rokhlin weights (2 pi/N) R_{|p-q|} |z'(t_q)| on every kernel difference."""
    n = bd.n
    idx = np.arange(n)
    dist = np.abs(idx[:, None] - idx[None, :])
    dist = np.minimum(dist, n - dist)
    rw = kr6.weights(n)[dist] * bd.w[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        so, do, kpo, to = boundary_kernels(bd, bd.x[None, :], omega)
        si, di, kpi, ti = boundary_kernels(bd, bd.x[None, :], index * omega)
    parts = []
    for v in (kpo - kpi, to - ti, so - si, do - di):
        v = np.array(v)
        v[idx, idx] = 0.0
        parts.append(v * rw)
    kp, t, s, dd = parts
    a = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    a[0::2, 0::2] = -kp            # (1/w) row, w column
    a[0::2, 1::2] = -t / omega
    a[1::2, 0::2] = s * omega
    a[1::2, 1::2] = dd
    a[np.arange(2 * n), np.arange(2 * n)] += 1.0
    return a


def matrix_a_image(bd: qd.Boundary, omega: float, d: float, j: int) -> np.ndarray:
    """A_j: the row functionals of the pair on the image obstacle shifted by j d (outside
    wavenumber only), plain trapezoid weights."""
    s, dd, kp, t = boundary_kernels(bd, bd.x[None, :] + j * d, omega)
    w = bd.w[None, :]
    a = np.zeros((2 * bd.n, 2 * bd.n), dtype=np.complex128)
    a[0::2, 0::2] = -kp * w
    a[0::2, 1::2] = -t * w / omega
    a[1::2, 0::2] = s * w * omega
    a[1::2, 1::2] = dd * w
    return a


def obstacle_blocks(x, y, dx, dy, omega: float, index: float, d: float, p: int = 1):
    """The angle-independent blocks A and A_j (0 < |j| <= P) of one obstacle."""
    bd = qd.boundary(x, y, dx, dy)
    imgs = {j: matrix_a_image(bd, omega, d, j) for j in range(-p, p + 1) if j != 0}
    return matrix_a(bd, omega, index), imgs


def matrix_b_parts(bd: qd.Boundary, ct: qd.Contour, omega, d):
    """B = B_L + alpha B_R: the row functionals of the wall potentials [S^ | D^] of the left
    and right walls (2N x 2M each)."""
    v = qd.wall_field_rows(bd.x, bd.y, ct, omega, d)
    gx = qd.wall_field_rows(bd.x, bd.y, ct, omega, d, "x")
    gy = qd.wall_field_rows(bd.x, bd.y, ct, omega, d, "y")
    # each is (SL, SR, DL, DR)
    bl = row_functional(bd, omega, np.hstack([v[0], v[2]]), np.hstack([gx[0], gx[2]]), np.hstack([gy[0], gy[2]]))
    br = row_functional(bd, omega, np.hstack([v[1], v[3]]), np.hstack([gx[1], gx[3]]), np.hstack([gy[1], gy[3]]))
    return bl, br


def wall_fourier_rows_pair(sx, sy, snx, sny, sw, ct: qd.Contour, omega, x0):
    """Wall discrepancy rows [f; fn] (2M x 2N) of the pair's sources: s columns
    w [S^; D*^], tau columns [D^; T^], times the source weights."""
    s_hat, d_hat, dstar_hat, t_hat = qd.wall_fourier_parts(sx, sy, snx, sny, ct, omega, x0)
    s_hat, dstar_hat = omega * s_hat, omega * dstar_hat
    w = sw[None, :]
    return np.vstack([interlace_cols(s_hat * w, d_hat * w), interlace_cols(dstar_hat * w, t_hat * w)])


def matrix_c_parts(bd: qd.Boundary, ct: qd.Contour, omega, d, p: int = 1):
    """C~ = alpha^P C_L - alpha^{-(P+1)} C_R, images as in the Dirichlet reading."""
    cl = wall_fourier_rows_pair(bd.x + p * d, bd.y, bd.nx, bd.ny, bd.w, ct, omega, -0.5 * d)
    cr = wall_fourier_rows_pair(bd.x - p * d, bd.y, bd.nx, bd.ny, bd.w, ct, omega, 0.5 * d)
    return cl, cr


def eval_rows(tx, ty, bd: qd.Boundary, ct: qd.Contour, omega, d, alpha, p: int = 1, deriv=None):
    """Rows mapping (eta, xi) to the outside field u (or u_x, u_y) at targets in the cell:
    the images |j| <= P of the pair plus the wall potentials."""
    tx = np.asarray(tx, dtype=np.float64)[:, None]
    ty = np.asarray(ty, dtype=np.float64)[:, None]
    sig = np.zeros((tx.shape[0], bd.n), dtype=np.complex128)
    tau = np.zeros_like(sig)
    for j in range(-p, p + 1):
        args = (tx, ty, bd.x[None, :] + j * d, bd.y[None, :], bd.nx[None, :], bd.ny[None, :], omega)
        if deriv is None:
            gs, gt = layer_values(*args)
        else:
            gx, gy, dx_, dy_ = layer_gradients(*args)
            gs, gt = (gx, dx_) if deriv == "x" else (gy, dy_)
        sig += (alpha ** j) * omega * gs * bd.w[None, :]
        tau += (alpha ** j) * gt * bd.w[None, :]
    sl, sr, dl, dr = qd.wall_field_rows(tx[:, 0], ty[:, 0], ct, omega, d, deriv)
    return interlace_cols(sig, tau), np.hstack([sl + alpha * sr, dl + alpha * dr])


def incident_rhs(bd: qd.Boundary, omega, theta):
    """Minus the row functionals of u_inc = exp(i w (x cos theta + y sin theta))."""
    kx, ky = omega * math.cos(theta), omega * math.sin(theta)
    u = np.exp(1j * (kx * bd.x + ky * bd.y))
    return -row_functional(bd, omega, u, 1j * kx * u, 1j * ky * u)


# --------------------------------------------------------------------------
# The quasi-periodic solve (Eq. block2 with the pair, plus Wood's rows)
# --------------------------------------------------------------------------

def dense_solve(x, y, dx, dy, omega: float, index: float, d: float, theta: float, opts: qd.Options,
                blocks=None) -> qd.Solution:
    """Fill the extended system densely, solve it with LAPACK and return the Bragg
    amplitudes and the flux error.  `blocks` = obstacle_blocks(...) of the same obstacle,
    omega, index, d and P, or None."""
    bd = qd.boundary(x, y, dx, dy)
    alpha = np.exp(1j * omega * d * math.cos(theta))
    ct = qd.contour(opts.m, opts.h, opts.c, opts.w, opts.t0)
    y0 = opts.y0 if opts.y0 is not None else qd.default_y0(bd, d)
    p = opts.p
    a0, imgs = blocks if blocks is not None else obstacle_blocks(x, y, dx, dy, omega, index, d, p)
    a = a0.copy()
    for j in range(-p, p + 1):
        if j != 0:
            a += (alpha ** j) * imgs[j]
    bl, br = matrix_b_parts(bd, ct, omega, d)
    cl, cr = matrix_c_parts(bd, ct, omega, d, p)
    q = qd.matrix_q(ct, omega, d, alpha)
    wood = qd.flipped_modes(omega, d, theta, ct)
    nw = len(wood)
    nn, m2 = 2 * bd.n, 2 * ct.m
    size = nn + m2 + nw
    big = np.zeros((size, size), dtype=np.complex128)
    big[:nn, :nn] = a
    big[:nn, nn:nn + m2] = bl + alpha * br
    big[nn:nn + m2, :nn] = (alpha ** p) * cl - alpha ** (-(p + 1)) * cr
    big[nn:nn + m2, nn:nn + m2] = q
    if nw:
        xs = qd.sample_points(d, opts.n_samples)
        ys_lo = np.full_like(xs, -y0)
        kap_w = qd.kappa_n(omega, d, theta, wood)
        kn_w = qd.k_n(omega, kap_w)
        u_eta, u_xi = eval_rows(xs, ys_lo, bd, ct, omega, d, alpha, p)
        uy_eta, uy_xi = eval_rows(xs, ys_lo, bd, ct, omega, d, alpha, p, deriv="y")
        for i, (kap, kn) in enumerate(zip(kap_w, kn_w)):
            pw = qd.plane_wave(bd.x, bd.y, kap, kn)
            big[:nn, nn + m2 + i] = row_functional(bd, omega, pw, 1j * kap * pw, 1j * kn * pw)
            f = qd.dft_rows(xs, np.array([kap]))[0]
            row = nn + m2 + i
            big[row, :nn] = 1j * kn * (f @ u_eta) + f @ uy_eta
            big[row, nn:nn + m2] = 1j * kn * (f @ u_xi) + f @ uy_xi
            for i2, (kap2, kn2) in enumerate(zip(kap_w, kn_w)):
                pw2 = qd.plane_wave(xs, ys_lo, kap2, kn2)
                pwy2 = qd.plane_wave(xs, ys_lo, kap2, kn2, deriv="y")
                big[row, nn + m2 + i2] = 1j * kn * (f @ pw2) + f @ pwy2
    rhs = np.zeros(size, dtype=np.complex128)
    rhs[:nn] = incident_rhs(bd, omega, theta)
    sol = scipy.linalg.solve(big, rhs)
    eta, xi, wc = sol[:nn], sol[nn:nn + m2], sol[nn + m2:]
    return bragg(bd, ct, omega, d, theta, alpha, eta, xi, wood, wc, y0, opts.n_samples, p)


def bragg(bd, ct, omega, d, theta, alpha, eta, xi, wood, wc, y0, n_samples, p=1) -> qd.Solution:
    """Bragg amplitudes of the propagating orders and the flux error (the Dirichlet
    oracle's extraction with the pair's field rows)."""
    xs = qd.sample_points(d, n_samples)
    orders = qd.mode_range(omega, d, theta)
    kap = qd.kappa_n(omega, d, theta, orders)
    f = qd.dft_rows(xs, kap)
    out = []
    for ysign in (+1.0, -1.0):
        ys = np.full_like(xs, ysign * y0)
        r_eta, r_xi = eval_rows(xs, ys, bd, ct, omega, d, alpha, p)
        u = r_eta @ eta + r_xi @ xi
        for i, n in enumerate(wood):
            kw = qd.kappa_n(omega, d, theta, n)
            u = u + wc[i] * qd.plane_wave(xs, ys, kw, qd.k_n(omega, kw))
        out.append(f @ u)
    cn, dn = out
    kn = qd.k_n(omega, kap).real
    k0 = omega * abs(math.sin(theta))
    inc = np.where(orders == 0, np.exp(1j * k0 * y0), 0.0)
    flux = float(np.sum((kn / k0) * (np.abs(cn) ** 2 + np.abs(dn + inc) ** 2)))
    return qd.Solution(eta, xi, wc, wood, orders, cn, dn, abs(flux - 1.0), y0, alpha)


# --------------------------------------------------------------------------
# One obstacle in free space, and the dielectric disc in closed form
# --------------------------------------------------------------------------

def free_solve(x, y, dx, dy, omega: float, index: float, theta: float):
    """The pair's densities (sigma = w s, tau) for an isolated obstacle (no images, no walls)."""
    bd = qd.boundary(x, y, dx, dy)
    eta = scipy.linalg.solve(matrix_a(bd, omega, index), incident_rhs(bd, omega, theta))
    return bd, omega * eta[0::2], eta[1::2]


def free_field(bd: qd.Boundary, sigma, tau, k, tx, ty):
    """S_k sigma + D_k tau at targets off the boundary (k = w outside, n w inside)."""
    tx = np.asarray(tx, dtype=np.float64)[:, None]
    ty = np.asarray(ty, dtype=np.float64)[:, None]
    g, dg = layer_values(tx, ty, bd.x[None, :], bd.y[None, :], bd.nx[None, :], bd.ny[None, :], k)
    return (g * bd.w[None, :]) @ sigma + (dg * bd.w[None, :]) @ tau


def mie_disc(radius, omega, index, theta, tx, ty, mmax: int | None = None):
    """Closed form for the disc |x| < radius of index n lit by exp(i w x.(cos t, sin t)):
    with u_inc = sum_m i^m J_m(w r) e^{i m (phi - t)}, the scattered field outside is
    sum_m b_m H_m(w r) e^{i m phi} and the field inside sum_m a_m J_m(n w r) e^{i m phi}, where
    continuity of u and du/dr at r = radius gives
      b_m = c_m (n J_m(ka) J_m'(nka) - J_m'(ka) J_m(nka)) / (H_m'(ka) J_m(nka) - n H_m(ka) J_m'(nka)),
      a_m = (c_m J_m(ka) + b_m H_m(ka)) / J_m(nka),   c_m = i^m e^{-i m t},  k = w, a = radius.
    Returns the scattered field at outside targets and the total field at inside ones."""
    tx = np.asarray(tx, dtype=np.float64)
    ty = np.asarray(ty, dtype=np.float64)
    ka, nka = omega * radius, index * omega * radius
    if mmax is None:
        mmax = int(max(ka, nka) + 40)
    m = np.arange(-mmax, mmax + 1)
    c = (1j ** m) * np.exp(-1j * m * theta)
    j_ka, jp_ka = scipy.special.jv(m, ka), scipy.special.jvp(m, ka)
    h_ka, hp_ka = scipy.special.hankel1(m, ka), scipy.special.h1vp(m, ka)
    j_n, jp_n = scipy.special.jv(m, nka), scipy.special.jvp(m, nka)
    b = c * (index * j_ka * jp_n - jp_ka * j_n) / (hp_ka * j_n - index * h_ka * jp_n)
    a = (c * j_ka + b * h_ka) / j_n
    r = np.hypot(tx, ty)
    phi = np.arctan2(ty, tx)
    e = np.exp(1j * np.outer(phi, m))
    out = np.where(r > radius,
                   (scipy.special.hankel1(m[None, :], omega * r[:, None]) * e) @ b,
                   (scipy.special.jv(m[None, :], index * omega * r[:, None]) * e) @ a)
    return out


# --------------------------------------------------------------------------
# The second periodizer (proxy points and wall discrepancies) for the pair
# --------------------------------------------------------------------------

def proxy_solve(x, y, dx, dy, omega: float, index: float, d: float, theta: float,
                o: pp.ProxyOptions | None = None, blocks=None) -> pp.ProxySolution:
    """The box scheme of oracle/proxy_periodizer.py with the pair: the obstacle rows are the
    interlaced transmission rows (A~ of the pair, the row functionals of the proxy fields),
    the wall and line rows see the pair's images.  Sizes as in that module."""
    o = o or pp.ProxyOptions()
    bd = qd.boundary(x, y, dx, dy)
    alpha = np.exp(1j * omega * d * math.cos(theta))
    h, rp, mp, kk, mt = pp.resolved(x, y, omega, d, theta, o)
    n2 = 2 * bd.n
    ang = 2.0 * math.pi * np.arange(mp) / mp
    px, py, pnx, pny = rp * np.cos(ang), rp * np.sin(ang), np.cos(ang), np.sin(ang)
    modes = np.arange(-kk, kk + 1)
    kap = qd.kappa_n(omega, d, theta, modes)
    kn = qd.k_n(omega, kap)
    a0, imgs = blocks if blocks is not None else obstacle_blocks(x, y, dx, dy, omega, index, d)
    at = a0 + alpha * imgs[1] + imgs[-1] / alpha

    def img(tx, ty, j, der):
        args = (tx[:, None], ty[:, None], bd.x[None, :] + j * d, bd.y[None, :], bd.nx[None, :],
                bd.ny[None, :], omega)
        if der is None:
            gs, gt = layer_values(*args)
        else:
            gx, gy, dx_, dy_ = layer_gradients(*args)
            gs, gt = (gx, dx_) if der == "x" else (gy, dy_)
        return interlace_cols(omega * gs * bd.w[None, :], gt * bd.w[None, :])

    def prox(tx, ty, der=None):
        return pp._proxy_field(tx, ty, px, py, pnx, pny, omega, der)

    gy_nodes, _ = np.polynomial.legendre.leggauss(o.m_wall)
    yw = h * gy_nodes
    xl, xr = np.full_like(yw, -0.5 * d), np.full_like(yw, 0.5 * d)
    xt = -0.5 * d + (np.arange(mt) + 0.5) * d / mt
    nu = 2 * kk + 1
    ncol = n2 + mp + 2 * nu
    rows = []
    r0 = np.zeros((n2, ncol), dtype=np.complex128)
    r0[:, :n2] = at
    r0[:, n2:n2 + mp] = row_functional(bd, omega, prox(bd.x, bd.y), prox(bd.x, bd.y, "x"), prox(bd.x, bd.y, "y"))
    rows.append(r0)
    for der in (None, "x"):
        r = np.zeros((o.m_wall, ncol), dtype=np.complex128)
        r[:, :n2] = alpha * img(xl, yw, 1, der) - img(xr, yw, -1, der) / alpha ** 2
        r[:, n2:n2 + mp] = prox(xl, yw, der) - prox(xr, yw, der) / alpha
        rows.append(r)
    for sgn, off in ((1.0, n2 + mp), (-1.0, n2 + mp + nu)):
        yy = np.full_like(xt, sgn * h)
        ex = np.exp(1j * np.outer(xt, kap))
        for der in (None, "y"):
            r = np.zeros((mt, ncol), dtype=np.complex128)
            for j in (-1, 0, 1):
                r[:, :n2] += (alpha ** j) * img(xt, yy, j, der)
            r[:, n2:n2 + mp] = prox(xt, yy, der)
            r[:, off:off + nu] = -(ex if der is None else ex * (1j * sgn * kn)[None, :])
            rows.append(r)
    big = np.vstack(rows)
    rhs = np.zeros(big.shape[0], dtype=np.complex128)
    rhs[:n2] = incident_rhs(bd, omega, theta)
    scale = 1.0 / np.maximum(np.linalg.norm(big, axis=0), 1e-300)
    sol, *_ = scipy.linalg.lstsq(big * scale[None, :], rhs, lapack_driver="gelsd")
    sol = sol * scale
    res = float(np.linalg.norm(big @ sol - rhs) / np.linalg.norm(rhs))
    a = sol[n2 + mp:n2 + mp + nu]
    b = sol[n2 + mp + nu:]
    orders = qd.mode_range(omega, d, theta)
    sel = orders + kk
    return pp.ProxySolution(orders, a, b, modes, a[sel], b[sel], h, res)
