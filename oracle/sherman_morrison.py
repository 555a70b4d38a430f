"""Sherman-Morrison update of an inverse Slater matrix after one accepted move.

TEST INFRASTRUCTURE ONLY (see the package docstring).

When the move of electron j is accepted, row j of D (D[j][l] = psi_l(r_j))
is replaced by the new orbital row psi'.  The paper names this O(N^2) update
of the inverse as the second bottleneck of the Monte Carlo step (Sec. VI.D).
With D^{-1} stored as Dinv[l][k] and

    w_k = sum_l psi'_l Dinv[l][k]        (w_j = xi, the acceptance ratio),

the updated inverse is

    Dinv'[l][k] = Dinv[l][k] - Dinv[l][j] (w_k - delta_jk) / w_j,

so column j becomes Dinv[.][j] / xi.  This module writes that formula out in
FP64, step by step; the tests pin it against a direct inverse of the updated
matrix and against D' Dinv' = I.
"""
from __future__ import annotations

import numpy as np


def sm_update(dinv, row, j):
    """FP64 Sherman-Morrison row update.  dinv [n][n] (Dinv[l][k]), row [n]."""
    Di = np.asarray(dinv, dtype=np.float64)
    r = np.asarray(row, dtype=np.float64)
    w = r @ Di                              # w_k = sum_l psi'_l Dinv[l][k]
    colj = Di[:, j].copy()
    f = w.copy()
    f[j] -= 1.0                             # w_k - delta_jk
    return Di - np.outer(colj, f) / w[j], w


def sm_update_terms(dinv, row, j):
    """Magnitudes for an FP32 rounding bound: |Dinv|, |col j| x |w - e_j| /
    |w_j|, and the absolute sums S_k = sum_l |psi'_l Dinv[l][k]| behind each
    w_k."""
    Di = np.asarray(dinv, dtype=np.float64)
    r = np.asarray(row, dtype=np.float64)
    w = r @ Di
    S = np.abs(r) @ np.abs(Di)
    f = w.copy()
    f[j] -= 1.0
    colj = np.abs(Di[:, j])
    return np.abs(Di), np.outer(colj, np.abs(f)) / abs(w[j]), S, w
