"""The library's Chebyshev table for H0, H1 (csrc/hankel_table.h), evaluated on the CPU the
way the device does (Clenshaw on intervals of width 1/kHankelPerUnit, Y0 and Y1 rebuilt with one logarithm),
against SciPy's Bessel functions on 20 000 points in (1e-4, 40)."""
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
    body = txt.split("= {", 1)[1].split("};", 1)[0]
    vals = np.array([float(v) for v in body.replace("\n", " ").split(",") if v.strip()])
    assert vals.size == ni * 4 * nd
    return ni // pu, nd, pu, vals.reshape(ni, 4, nd)


def _eval(tab, nd, pu, z):
    i = int(pu * z)
    t = 2.0 * (pu * z - i) - 1.0
    out = []
    for f in range(4):
        c = tab[i, f]
        b1 = b2 = 0.0
        for k in range(nd - 1, 0, -1):
            b1, b2 = 2.0 * t * b1 - b2 + c[k], b1
        out.append(t * b1 - b2 + c[0])
    j0, j1, r0, r1 = out
    lg = 2.0 / math.pi * (math.log(0.5 * z) + 0.57721566490153286061)
    return j0, j1, lg * j0 + r0, lg * j1 - 2.0 / (math.pi * z) + r1


def test_hankel_table_matches_scipy():
    zmax, nd, pu, tab = _table()
    rng = np.random.default_rng(0)
    zs = np.concatenate([10.0 ** rng.uniform(-4, math.log10(zmax - 1e-9), 20000), [1e-4, 0.5, 1.0, 17.5, 39.99]])
    worst = 0.0
    for z in zs:
        j0, j1, y0, y1 = _eval(tab, nd, pu, z)
        h0 = complex(special.j0(z), special.y0(z))
        h1 = complex(special.j1(z), special.y1(z))
        worst = max(worst, abs(complex(j0, y0) - h0) / abs(h0), abs(complex(j1, y1) - h1) / abs(h1))
    assert worst < 5e-15, worst
