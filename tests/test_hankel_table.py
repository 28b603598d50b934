"""The library's Chebyshev tables for H0, H1 (csrc/hankel_table.h), evaluated on the CPU the
way the device does (Clenshaw on intervals of width 1/kHankelPerUnit; below z = 4, Y0 and Y1
rebuilt from the regular parts of Neumann's expansions with one logarithm, above it
tabulated directly), against SciPy's Bessel functions on 20 000 points in (1e-4, 120) and mpmath's on 300.  The
double-float table and recurrence (float pairs, error-free transformations) are emulated
in float32 arithmetic."""
import math
import os
import re

import numpy as np
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _table():
    txt = open(os.path.join(ROOT, "paper_1301_1247_gb300", "csrc", "hankel_table.h")).read()
    ni = int(re.search(r"kHankelIntervals = (\d+)", txt).group(1))
    nd = int(re.search(r"kHankelDegree = (\d+)", txt).group(1))
    pu = int(re.search(r"kHankelPerUnit = (\d+)", txt).group(1))
    direct = int(re.search(r"kHankelDirect = (\d+)", txt).group(1))
    body = txt.split("kHankelCheb[", 1)[1].split("= {", 1)[1].split("};", 1)[0]
    vals = np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])
    assert vals.size == ni * 4 * nd
    bdf = txt.split("kHankelChebDF[", 1)[1].split("= {", 1)[1].split("};", 1)[0]
    dvals = np.array([float(v.strip().rstrip("f")) for v in bdf.replace("\n", " ").split(",") if v.strip()],
                     dtype=np.float32)
    assert dvals.size == 2 * ni * 4 * nd
    return dict(zmax=ni // pu, nd=nd, pu=pu, direct=direct, tab=vals.reshape(ni, 4, nd),
                hi=dvals[0::2].reshape(ni, 4, nd), lo=dvals[1::2].reshape(ni, 4, nd))


def _combine(T, iv, z, j0, j1, a0, a1):
    if iv >= T["direct"]:
        return j0, j1, a0, a1
    lg = 2.0 / math.pi * (math.log(0.5 * z) + 0.57721566490153286061)
    return j0, j1, lg * j0 + a0, lg * j1 - 2.0 / (math.pi * z) + a1


def _eval(T, z):
    i = int(T["pu"] * z)
    t = 2.0 * (T["pu"] * z - i) - 1.0
    out = []
    for f in range(4):
        c = T["tab"][i, f]
        b1 = b2 = 0.0
        for k in range(T["nd"] - 1, 0, -1):
            b1, b2 = 2.0 * t * b1 - b2 + c[k], b1
        out.append(t * b1 - b2 + c[0])
    return _combine(T, i, z, *out)


def _worst(T, zs, ev):
    worst = 0.0
    for z in zs:
        j0, j1, y0, y1 = ev(T, z)
        h0 = complex(special.j0(z), special.y0(z))
        h1 = complex(special.j1(z), special.y1(z))
        worst = max(worst, abs(complex(j0, y0) - h0) / abs(h0), abs(complex(j1, y1) - h1) / abs(h1))
    return worst


def _points(T, n):
    rng = np.random.default_rng(0)
    return np.concatenate([10.0 ** rng.uniform(-4, math.log10(T["zmax"] - 1e-9), n),
                           [1e-4, 0.5, 1.0, 3.999, 4.0, 17.5, 39.99]])


def test_hankel_table_matches_scipy():
    """SciPy's own J1, Y1 carry errors near 6e-15 beyond z = 40, hence the 1e-14 bar here;
    the 40-digit check below is the sharp one."""
    T = _table()
    assert _worst(T, _points(T, 20000), _eval) < 1e-14


def test_hankel_table_matches_mpmath():
    mp = __import__("pytest").importorskip("mpmath")
    mp.mp.dps = 30
    T = _table()
    rng = np.random.default_rng(1)
    zs = np.concatenate([rng.uniform(1e-3, T["zmax"] - 1e-9, 300), [3.999, 4.0, 39.99, 40.0, 119.99]])
    worst = 0.0
    for z in zs:
        j0, j1, y0, y1 = _eval(T, z)
        h0 = complex(mp.besselj(0, z) + 1j * mp.bessely(0, z))
        h1 = complex(mp.besselj(1, z) + 1j * mp.bessely(1, z))
        worst = max(worst, abs(complex(j0, y0) - h0) / abs(h0), abs(complex(j1, y1) - h1) / abs(h1))
    assert worst < 1e-15, worst


# ---- double-float emulation (float32 numpy scalars; fmaf emulated through float64, exact
# for the error-free products used here) ----
F = np.float32


def _fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def _add_to(bh, bl, ah, al):
    s = F(ah + bh)
    v = F(s - ah)
    t = F(F(ah - F(s - v)) + F(bh - v))
    return s, F(al + F(t + bl))


def _mac(xh, xl, yh, yl, ah, al):
    p = F(xh * yh)
    e = _fma(xh, yh, -p)
    e = _fma(xh, yl, e)
    e = _fma(xl, yh, e)
    return _add_to(p, e, ah, al)


def _norm(ah, al):
    s = F(ah + al)
    return s, F(al - F(s - ah))


def _split(x):
    hi = F(x)
    return hi, F(x - np.float64(hi))


def _eval_df(T, z):
    i = int(T["pu"] * z)
    t = 2.0 * (T["pu"] * z - i) - 1.0
    th, tl = _split(t)
    t2h, t2l = F(2 * th), F(2 * tl)
    out = []
    for f in range(4):
        ch, cl = T["hi"][i, f], T["lo"][i, f]
        b1 = b2 = (F(0), F(0))
        for k in range(T["nd"] - 1, 0, -1):
            bh, bl = _add_to(-b2[0], -b2[1], ch[k], cl[k])
            bh, bl = _mac(t2h, t2l, b1[0], b1[1], bh, bl)
            b2, b1 = b1, _norm(bh, bl)
        bh, bl = _add_to(-b2[0], -b2[1], ch[0], cl[0])
        bh, bl = _mac(th, tl, b1[0], b1[1], bh, bl)
        out.append(float(bh) + float(bl))
    return _combine(T, i, z, *out)


def test_double_float_table_and_recurrence():
    """The float-pair table reproduces the FP64 table to 2^-48, and the double-float
    Clenshaw recurrence of the device stays within 5e-14 of SciPy."""
    T = _table()
    tab = T["tab"]
    rec = T["hi"].astype(np.float64) + T["lo"].astype(np.float64)
    assert np.all(np.abs(rec - tab) <= 2.0 ** -47 * np.abs(tab) + 1e-300)
    worst = _worst(T, _points(T, 1500), _eval_df)
    assert worst < 5e-14, worst
