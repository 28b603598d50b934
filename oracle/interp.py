"""Interpolative decomposition by column-pivoted QR (oracle side; test infrastructure).

Def. 3.1: an m x n matrix M of rank l is written M = P M(J, :), where J picks
l rows and P (m x l) contains the l x l identity in rows J.  The oracle obtains
J and P from a column-pivoted QR of M^T (LAPACK zgeqp3 via scipy):
M^T Pi = Q [R11 R12], J = Pi(1:l), and the remaining rows of M are
M(Pi(l+1:), :) ~ (R11^{-1} R12)^T M(J, :), so P(J, :) = I and
P(Pi(l+1:), :) = (R11^{-1} R12)^T (a plain transpose, no conjugate).
The rank is the number of diagonal entries with |R_ii| > tol |R_11|.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def row_id(m: np.ndarray, tol: float):
    """Return (J, P, rank) with m ~= P @ m[J, :]."""
    m = np.asarray(m)
    rows = m.shape[0]
    if rows == 0 or m.shape[1] == 0:
        return np.zeros(0, dtype=np.int64), np.zeros((rows, 0), dtype=m.dtype), 0
    _, r, piv = scipy.linalg.qr(m.T, mode="economic", pivoting=True)
    diag = np.abs(np.diag(r))
    if diag.size == 0 or diag[0] == 0.0:
        return np.zeros(0, dtype=np.int64), np.zeros((rows, 0), dtype=m.dtype), 0
    rank = int(np.sum(diag > tol * diag[0]))
    j = piv[:rank]
    t = scipy.linalg.solve_triangular(r[:rank, :rank], r[:rank, rank:rows])
    p = np.zeros((rows, rank), dtype=np.result_type(m.dtype, np.float64))
    p[j, :] = np.eye(rank)
    p[piv[rank:], :] = t.T
    return j, p, rank
