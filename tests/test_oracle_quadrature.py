"""Pins for the oracle's quadrature and boundary operator A (Sec. 2.3)."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import kr6, qp_dense as qd
from paper_1301_1247_gb300 import inputs


def test_kr6_table_solves_moment_conditions():
    """The stored gamma_j satisfy the six moment conditions (re-derived in 50 digits)."""
    mp = pytest.importorskip("mpmath")
    derived = [float(v) for v in kr6.derive()]
    assert np.allclose(kr6.gamma(), derived, rtol=1e-15, atol=0)
    g = kr6.gamma()
    j = np.arange(1, 7)
    assert abs(g.sum() - 0.5) < 1e-13
    assert abs((g * np.log(j)).sum() + 0.5 * math.log(2 * math.pi)) < 1e-12
    assert abs((g * j ** 2).sum()) < 1e-11
    assert abs((g * j ** 2 * np.log(j)).sum() - float(mp.zeta(-2, derivative=1))) < 1e-11


def _log_integral(n):
    t = 2 * np.pi * np.arange(n) / n
    with np.errstate(divide="ignore"):
        f = np.log(4 * np.sin(t / 2) ** 2) * np.exp(np.cos(t))
    f[0] = 0.0
    return (2 * np.pi / n) * np.sum(kr6.weights(n) * f)


def test_kr6_sixth_order_on_closed_form():
    """int_0^{2pi} log(4 sin^2(t/2)) e^{cos t} dt = -4 pi sum_m I_m(1)/m (Fourier series of both
    factors); the corrected trapezoid rule must converge at order ~6."""
    exact = -4 * np.pi * sum(sp.iv(m, 1.0) / m for m in range(1, 60))
    errs = [abs(_log_integral(n) - exact) for n in (128, 256, 512)]
    assert errs[-1] < 1e-9
    order = math.log2(errs[1] / errs[2])
    assert order > 5.3, errs
    # a plain punctured trapezoid rule is only first order: the corrections matter
    n = 512
    t = 2 * np.pi * np.arange(n) / n
    with np.errstate(divide="ignore"):
        f = np.log(4 * np.sin(t / 2) ** 2) * np.exp(np.cos(t))
    f[0] = 0
    assert abs((2 * np.pi / n) * f.sum() - exact) > 1e-3


def _circle(a, n):
    t = 2 * np.pi * np.arange(n) / n
    return qd.boundary(a * np.cos(t), a * np.sin(t), -a * np.sin(t), a * np.cos(t)), t


@pytest.mark.parametrize("m", [0, 1, 4, 9])
def test_circle_eigenvalues(m):
    """On a circle of radius a, A = 1/2 + D - i w S is diagonal in e^{imt} with eigenvalue
    (i pi w a / 2) H_m(wa) [J_m'(wa) - i J_m(wa)] (separation of variables: exterior
    limit of the double layer plus -i w times the single layer)."""
    a, omega = 0.4, 10.0
    z = omega * a
    lam = (1j * np.pi * z / 2) * sp.hankel1(m, z) * (sp.jvp(m, z) - 1j * sp.jv(m, z))
    errs = []
    for n in (256, 512):
        bd, t = _circle(a, n)
        v = np.exp(1j * m * t)
        av = qd.matrix_a(bd, omega) @ v
        errs.append(np.max(np.abs(av - lam * v)))
    assert errs[1] < 2e-6
    assert errs[0] / errs[1] > 30  # high order in N


def test_green_representation_exterior_field():
    """A point source p inside the obstacle radiates u = G(., p) outside.  Solving
    A eta = u|_dOmega and evaluating (D - i w S) eta outside must give G(., p) back."""
    obs = inputs.star(0.3, 0.3, 5)
    omega = 10.0
    x, y, dx, dy = obs.sample(600)
    bd = qd.boundary(x, y, dx, dy)
    px, py = 0.05, -0.03
    f = qd.green(bd.x, bd.y, px, py, omega)
    eta = np.linalg.solve(qd.matrix_a(bd, omega), f)
    ang = np.linspace(0, 2 * np.pi, 17)[:-1]
    tx, ty = 0.8 * np.cos(ang), 0.8 * np.sin(ang)
    k = qd.combined(tx[:, None], ty[:, None], bd.x[None, :], bd.y[None, :],
                    bd.nx[None, :], bd.ny[None, :], omega)
    u = (k * bd.w[None, :]) @ eta
    exact = qd.green(tx, ty, px, py, omega)
    assert np.max(np.abs(u - exact)) / np.max(np.abs(exact)) < 1e-6


def test_target_gradient_matches_finite_differences():
    """combined_grad is the target gradient of combined (central differences)."""
    omega = 30.0
    sx, sy, snx, sny = 0.1, -0.2, 0.6, 0.8
    tx, ty = np.array([0.7, -0.4]), np.array([0.3, 0.9])
    gx, gy = qd.combined_grad(tx, ty, sx, sy, snx, sny, omega)
    e = 1e-6
    fx = (qd.combined(tx + e, ty, sx, sy, snx, sny, omega) - qd.combined(tx - e, ty, sx, sy, snx, sny, omega)) / (2 * e)
    fy = (qd.combined(tx, ty + e, sx, sy, snx, sny, omega) - qd.combined(tx, ty - e, sx, sy, snx, sny, omega)) / (2 * e)
    assert np.allclose(gx, fx, rtol=1e-7, atol=1e-7)
    assert np.allclose(gy, fy, rtol=1e-7, atol=1e-7)


def test_a_rows_are_rows_of_a():
    """The row-by-row evaluation used at full size reproduces rows of the dense A."""
    x, y, dx, dy = inputs.star(0.3, 0.3, 5).sample(200)
    bd = qd.boundary(x, y, dx, dy)
    rows = [0, 1, 7, 100, 199]
    assert np.allclose(qd.a_rows(bd, 10.0, rows), qd.matrix_a(bd, 10.0)[rows], rtol=0, atol=1e-15)


@pytest.mark.parametrize("m", [0, 3, 11])
def test_kress_circle_eigenvalues_spectral(m):
    """The oracle's second quadrature (Kress's, oracle/kress.py) has the same circle
    eigenvalues to rounding at modest N: it is spectrally accurate for analytic curves."""
    from oracle import kress
    a, omega, n = 0.4, 10.0, 96
    z = omega * a
    lam = (1j * np.pi * z / 2) * sp.hankel1(m, z) * (sp.jvp(m, z) - 1j * sp.jv(m, z))
    t = 2 * np.pi * np.arange(n) / n
    mat = kress.matrix_a(a * np.cos(t), a * np.sin(t), -a * np.sin(t), a * np.cos(t), omega)
    v = np.exp(1j * m * t)
    assert np.max(np.abs(mat @ v - lam * v)) < 1e-12


def test_kress_and_kr6_give_the_same_bragg_amplitudes():
    """Two discretizations of one continuum problem (Sec. 2.3's KR6 and Kress's spectral rule)
    converge to the same Bragg amplitudes: Kress at N = 256 against KR6 at N = 1024 and 2048
    (same contour, samples and y0); KR6's gap shrinks at its sixth order."""
    import math
    from oracle import readings as rd
    obs = inputs.star(0.3, 0.3, 5)
    omega, th = 10.0, -math.pi / 5

    def amps(quad, n):
        x, y, dx, dy = obs.sample(n)
        o = rd.options(x, y, omega, 1.0, th)
        o.y0 = 0.7  # one sampling line for all N (y0 = max|y| + d/4 moves with the samples)
        b = qd.obstacle_blocks(x, y, dx, dy, omega, 1.0, quadrature=quad)
        return qd.bragg_vector(qd.dense_solve(x, y, dx, dy, omega, 1.0, th, o, b))

    ref = amps("kress", 256)
    e1 = np.linalg.norm(amps("kr6", 1024) - ref) / np.linalg.norm(ref)
    e2 = np.linalg.norm(amps("kr6", 2048) - ref) / np.linalg.norm(ref)
    assert e2 < 1e-10
    assert e1 / e2 > 40
