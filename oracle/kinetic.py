"""Slater-only local kinetic energy from orbital values and Laplacians.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a Slater determinant Psi_D = prod_sigma det D_sigma with
D_sigma[j][l] = psi_l(r_j) (electrons j of spin sigma, Eq. eq5 of Sec. II.A),
the kinetic part of the local energy is

    T_L = -1/2 sum_sigma sum_{j in sigma} lap_j Psi_D / Psi_D
        = -1/2 sum_sigma sum_j sum_l lap psi_l(r_j) (D_sigma^{-1})_{lj}
        = -1/2 sum_sigma trace(D_sigma^{-1} Lap_sigma),

with Lap_sigma[j][l] = lap psi_l(r_j).  This is the quantity through which the
paper judges single-precision orbital errors against ~1e-3 hartree per
primitive cell (Sec. V.B).  Computed in FP64 with an LU factorisation with
partial pivoting (scipy), which serves as the library step.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def local_kinetic(values, laps, blocks):
    """T_L for spin blocks ``blocks = [(j0, j1), ...]`` of electrons.

    Each block uses orbitals 0..(j1 - j0 - 1), so D_sigma is square.
    Returns ``(T_L, [cond(D_sigma)])``.
    """
    v = np.asarray(values, dtype=np.float64)
    lp = np.asarray(laps, dtype=np.float64)
    total = 0.0
    conds = []
    for j0, j1 in blocks:
        m = j1 - j0
        D = v[j0:j1, :m]
        Lap = lp[j0:j1, :m]
        lu = sla.lu_factor(D)
        Z = sla.lu_solve(lu, Lap)        # D^{-1} Lap
        total += -0.5 * float(np.trace(Z))
        conds.append(float(np.linalg.cond(D)))
    return total, conds
