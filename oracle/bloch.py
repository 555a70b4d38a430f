"""Bloch-phase orbitals from a periodic blip expansion (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a k-point orbital psi_l(r) = exp(i k_l . r) u_l(r), with u_l periodic and
expanded in blips (Eqs. 11.12.24.1 and 11.12.24.2 give u_l and its
derivatives), the product rule gives

    grad psi = exp(i k.r) (grad u + i k u)
    lap psi  = exp(i k.r) (lap u + 2 i k . grad u - |k|^2 u).

k_l = 2 pi B kappa_l with B = A^{-T} (reciprocal lattice), so
k.r = 2 pi kappa . (A^{-1} r): the phase is evaluated from the fractional
coordinates.  Orbitals [koffs[q], koffs[q + 1]) share kappa_q.  Oracle A
(the C stencil evaluator) supplies u and its derivatives as a library step;
this module only applies the phase, in plain numpy FP64.
"""
from __future__ import annotations

import numpy as np


def eval_bloch(grid, lattice, coeffs, pos, kfrac, koffs, norm: int = 0, eval_u=None):
    """values [E][L], grads [E][3][L], laps [E][L] (complex128) of
    psi_l = exp(i k_l . r) u_l for a complex table ``coeffs`` of u_l."""
    from . import eval_stencil
    ev = eval_u or eval_stencil
    u, gu, lu = ev(grid, lattice, coeffs, pos, norm=norm)
    A = np.asarray(lattice, dtype=np.float64).T          # columns = lattice vectors
    Ainv = np.linalg.inv(A)
    kfrac = np.asarray(kfrac, dtype=np.float64).reshape(-1, 3)
    kcart = 2.0 * np.pi * kfrac @ Ainv                   # rows: k_q = 2 pi A^{-T} kappa_q
    L = u.shape[1]
    kq = np.zeros((L, 3))
    for q in range(len(kfrac)):
        kq[koffs[q]:koffs[q + 1]] = kcart[q]
    frac = np.asarray(pos, dtype=np.float64) @ Ainv.T     # [E][3] fractional coordinates
    ph = np.exp(2j * np.pi * (frac @ kfrac.T))            # [E][nk]
    phase = np.zeros((len(frac), L), dtype=np.complex128)
    for q in range(len(kfrac)):
        phase[:, koffs[q]:koffs[q + 1]] = ph[:, q:q + 1]
    v = phase * u
    g = phase[:, None, :] * (gu + 1j * kq.T[None, :, :] * u[:, None, :])
    kg = np.einsum("lc,ecl->el", kq, gu)
    lp = phase * (lu + 2j * kg - (kq * kq).sum(1)[None, :] * u)
    return v, g, lp
