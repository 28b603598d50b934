"""Helpers for the GPU tests: build the library once, torch device buffers."""
import os

import numpy as np


def require_lib():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    from paper_1301_1247_gb300 import build, hbs
    if not os.path.exists(hbs.LIB_PATH):
        build.build()
    return hbs


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_library_readings(info, x, y, omega, d=1.0):
    """The library's contour, Bragg sampling and y0 (hbs_info) equal the oracle's own
    (oracle/readings.py, Secs. 2.3-2.4, Remark 2.2): nothing is taken from the library."""
    from oracle import readings as rd
    disc = rd.discretization(x, y, omega, d)
    assert info["m"] == disc.m, (info["m"], disc.m)
    assert info["contour_h"] == disc.h and info["contour_c"] == disc.c and info["contour_w"] == disc.w
    assert abs(info["wood_t0"] - disc.shift) <= 1e-12 * max(1.0, disc.shift), (info["wood_t0"], disc.shift)
    assert info["n_bragg_samples"] == disc.n_samples
    assert abs(info["y0"] - disc.y0) <= 1e-14
    return disc


def oracle_options_checked(res, i, x, y, omega, theta, d=1.0, tie=1e-3):
    """Oracle options for angle i of a library result: the oracle chooses the contour itself and
    the test asserts the library chose the same (unless the oracle's two pole distances tie
    within `tie`, where both contours are exact and either choice is valid)."""
    from oracle import readings as rd
    disc = rd.discretization(x, y, omega, d)
    t0, margin = rd.choose_t0(omega, d, theta, disc)
    nw, t0_lib = res.angle_info(i)
    if margin > tie:
        assert abs(t0_lib - t0) <= 1e-12 * max(1.0, t0), (theta, t0_lib, t0, margin)
        return rd.options(x, y, omega, d, theta, t0)
    assert t0_lib == 0.0 or abs(t0_lib - disc.shift) <= 1e-12 * disc.shift, t0_lib
    return rd.options(x, y, omega, d, theta, t0_lib)
