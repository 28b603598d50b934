"""Kapur-Rokhlin 6th-order log-singular corrections (oracle side; test infrastructure).

Sec. 2.3 modifies the periodic trapezoid weights next to the diagonal:
R_0 = 0 and R_j = R_{N-j} = 1 + gamma_j for 1 <= j <= 6 (the paper writes the
per-side sum of the table entries; for a symmetric log singularity they are one
number per distance j), R_j = 1 otherwise.  The table itself lives in the cited
Kapur-Rokhlin paper, which is not at hand, so the oracle derives the values.

Derivation (generalised Euler-Maclaurin / zeta regularisation).  For
f(t) = g(t) log|t| + psi(t) with g, psi smooth, the punctured trapezoid sum
h sum_{j != 0} f(jh) misses, at each even order 2p, a term
2 h^{2p+1} g^{(2p)}(0)/(2p)! (zeta'(-2p) - log(h) zeta(-2p)) (and h psi(0) at
p = 0).  Adding h sum_{j=1}^{6} gamma_j (f(jh) + f(-jh)) cancels the orders
p = 0, 1, 2 exactly when
    sum gamma_j = 1/2,             sum gamma_j log j = -log(2 pi)/2,
    sum gamma_j j^{2p} = 0,        sum gamma_j j^{2p} log j = zeta'(-2p),  p = 1, 2,
a 6x6 linear system.  `derive()` solves it in 50-digit arithmetic (mpmath) and
`derive_kr6.py` writes the result to `kr6_gamma.txt`, which `gamma()` reads so
that the oracle needs no mpmath at run time.
"""
from __future__ import annotations

import os

import numpy as np

_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kr6_gamma.txt")


def derive(dps: int = 50):
    """Solve the six moment conditions above; returns a list of 6 mpmath numbers."""
    import mpmath as mp

    mp.mp.dps = dps
    js = range(1, 7)
    rows = [[mp.mpf(1) for _ in js], [mp.log(j) for j in js]]
    rhs = [mp.mpf(1) / 2, -mp.log(2 * mp.pi) / 2]
    for p in (1, 2):
        rows.append([mp.mpf(j) ** (2 * p) for j in js])
        rhs.append(mp.mpf(0))
        rows.append([mp.mpf(j) ** (2 * p) * mp.log(j) for j in js])
        rhs.append(mp.zeta(-2 * p, derivative=1))
    sol = mp.lu_solve(mp.matrix(rows), mp.matrix(rhs))
    return [sol[i] for i in range(6)]


def gamma() -> np.ndarray:
    """gamma_1..gamma_6 as float64, read from the table written by derive_kr6.py."""
    vals = []
    with open(_TABLE) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(float(line.split()[1]))
    if len(vals) != 6:
        raise RuntimeError("kr6_gamma.txt must hold six values")
    return np.array(vals)


def weights(n: int) -> np.ndarray:
    """R_j for j = 0..n-1 (R_0 = 0, R_j = R_{n-j} = 1 + gamma_j for j <= 6, else 1)."""
    if n < 13:
        raise ValueError("KR6 needs at least 13 nodes")
    r = np.ones(n)
    r[0] = 0.0
    g = gamma()
    for j in range(1, 7):
        r[j] = 1.0 + g[j - 1]
        r[n - j] = 1.0 + g[j - 1]
    return r
