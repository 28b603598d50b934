"""Writes dense_n8200.txt: Bragg amplitudes from the dense FP64 oracle (Eq. block2 with exact
neighbour images, LAPACK solve; Sec. 2.4 Wood's rows; Remarks 2.2-2.3) for two obstacles at
N = 8200, where the fast solver's production paths differ from the small cases: every third
node is a neighbour-ID candidate, the periodizer IDs run on a subsample, and the leaf level
has 256 nodes.

Every value comes from oracle/ (qp_dense, readings) and the seeded inputs; nothing from the
CUDA library.  Run from the repository root:  python tests/golden/make_dense_n8200.py
(about ten minutes on 8 cores, 10 GB of memory).
"""
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import qp_dense as qd  # noqa: E402
from oracle import readings as rd  # noqa: E402
from paper_1301_1247_gb300 import inputs  # noqa: E402

N = 8200
D = 1.0

# (name, obstacle, omega, angles: two Bloch groups of three plus one exact Wood's anomaly)
CASES = [
    ("complicated_w60", lambda: inputs.wiggly(0, 0.3, 60, 0.05), 60.0, 31, 3),
    ("wiggly_w30", lambda: inputs.wiggly(0, 0.35, 20, 0.03), 30.0, 32, 2),
]


def case_angles(omega, seed, wood_order):
    th = [float(t) for t in inputs.bloch_grouped_angles(seed, omega, D, 2, 3).ravel()]
    th.append(-math.acos(1.0 - 2.0 * math.pi * wood_order / (omega * D)))
    return th


def main(path):
    lines = [
        "# Dense FP64 oracle at N = 8200: Bragg amplitudes c_n (at +y0) and d_n (at -y0) of the",
        "# propagating orders, Eq. (block2) with exact images A_{+-1} (Sec. 2.4), the Sommerfeld",
        "# contour, Wood's rows and Bragg sampling of oracle/readings.py (Secs. 2.3-2.4, Remark 2.2).",
        "# Written by tests/golden/make_dense_n8200.py from oracle/ only.",
        "# case <name> <omega> <N> <sum x> <sum y>",
        "# angle <name> <i> <theta> <t0> <n_wood> <flux_error> <t0_margin>",
        "# amp <name> <i> <c|d> <n> <re> <im>",
    ]
    for name, make, omega, seed, wood_order in CASES:
        t_start = time.time()
        x, y, dx, dy = make().sample(N)
        lines.append(f"case {name} {float(omega)!r} {N} {float(np.sum(x))!r} {float(np.sum(y))!r}")
        disc = rd.discretization(x, y, omega, D)
        blocks = qd.obstacle_blocks(x, y, dx, dy, omega, D)
        for i, th in enumerate(case_angles(omega, seed, wood_order)):
            t0, margin = rd.choose_t0(omega, D, th, disc)
            sol = qd.dense_solve(x, y, dx, dy, omega, D, th, rd.options(x, y, omega, D, th, t0), blocks)
            lines.append(f"angle {name} {i} {float(th)!r} {float(t0)!r} {len(sol.wood_modes)} "
                         f"{float(sol.flux_error)!r} {float(margin)!r}")
            for kind, vals in (("c", sol.c), ("d", sol.d)):
                for n, v in zip(sol.orders, vals):
                    lines.append(f"amp {name} {i} {kind} {int(n)} {float(v.real)!r} {float(v.imag)!r}")
            print(f"{name} angle {i}: theta={th:.6f} t0={t0:.4f} nw={len(sol.wood_modes)} "
                  f"flux={sol.flux_error:.2e} ({time.time() - t_start:.0f} s)", flush=True)
        del blocks
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def load(path=None):
    """Parse the file: {name: dict(omega, n, sum_x, sum_y, angles=[dict(theta, t0, nw, flux,
    margin, orders, c, d)])}."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "dense_n8200.txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if not f or f[0].startswith("#"):
                continue
            if f[0] == "case":
                out[f[1]] = dict(omega=float(f[2]), n=int(f[3]), sum_x=float(f[4]), sum_y=float(f[5]), angles=[])
            elif f[0] == "angle":
                out[f[1]]["angles"].append(dict(theta=float(f[3]), t0=float(f[4]), nw=int(f[5]), flux=float(f[6]),
                                                margin=float(f[7]), orders=[], c={}, d={}))
            elif f[0] == "amp":
                a = out[f[1]]["angles"][int(f[2])]
                n = int(f[4])
                a[f[3]][n] = complex(float(f[5]), float(f[6]))
                if f[3] == "c":
                    a["orders"].append(n)
    return out


if __name__ == "__main__":
    main(os.path.join(os.path.dirname(os.path.abspath(__file__)), "dense_n8200.txt"))
