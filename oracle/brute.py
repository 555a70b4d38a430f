"""Oracle B: brute-force blip evaluation over every grid site and image.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sums a_{l,s} * Theta(r - R_s - T) over every site s of the grid and every
periodic image T of the cell near r, in Cartesian coordinates, with r taken as
given (no wrapping, no modulo, no stencil selection).  Eq. 11.12.24.1 restricts
the same sum to the 64 sites where Theta is non-zero (Eq. 7); because the
cubic B-spline has support [-2, 2] the two sums are equal, so this checks the
stencil oracle's wrap, modulo, site selection and Jacobian independently.

The B-spline here is a separate numpy transcription of the piecewise cubic
(Eq. 11.12.24.2 with phi read as the cubic B-spline), and the cell inverse
comes from ``numpy.linalg.inv``, not from the C oracle.  Tiny grids only:
the cost is E x 5^3 images x n1 n2 n3 sites.

``absmag_brute`` recomputes, in the same way, the rounding scale that the
stencil oracle returns beside every output: sum over the (site, image) pairs
whose basis function touches r of |W_k| |a_ls|, with W_k the Cartesian
weight of output kind k (value, the three gradient components, Laplacian).
"""
from __future__ import annotations

import itertools

import numpy as np


def bspline(x):
    ax = np.abs(x)
    return np.where(ax <= 1.0, 2.0 / 3.0 - ax ** 2 + 0.5 * ax ** 3,
                    np.where(ax <= 2.0, (2.0 - ax) ** 3 / 6.0, 0.0))


def bspline_d1(x):
    ax = np.abs(x)
    return np.where(ax <= 1.0, -2.0 * x + 1.5 * x * ax,
                    np.where(ax <= 2.0, -np.sign(x) * 0.5 * (2.0 - ax) ** 2, 0.0))


def bspline_d2(x):
    ax = np.abs(x)
    return np.where(ax <= 1.0, -2.0 + 3.0 * ax, np.where(ax <= 2.0, 2.0 - ax, 0.0))


def eval_brute(grid, lattice, coeffs, pos, norm: int = 0, image_radius: int = 2):
    """values [E][L], grads [E][3][L], laps [E][L] by direct summation."""
    n = np.array(grid, dtype=np.float64)
    A = np.asarray(lattice, dtype=np.float64).T          # columns = lattice vectors
    Ainv = np.linalg.inv(A)
    J = np.diag(n) @ Ainv
    c = np.asarray(coeffs)
    L = c.shape[-1]
    cf = c.reshape(-1, L)                                 # [P][L], site-major
    sites = np.array(list(itertools.product(range(grid[0]), range(grid[1]), range(grid[2]))),
                     dtype=np.float64)                    # same order as the table's rows
    scale = 1.5 ** 3 if norm == 1 else 1.0
    p = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    E = p.shape[0]
    dt = np.complex128 if np.iscomplexobj(c) else np.float64
    vals = np.zeros((E, L), dtype=dt)
    grads = np.zeros((E, 3, L), dtype=dt)
    laps = np.zeros((E, L), dtype=dt)
    rr = range(-image_radius, image_radius + 1)
    for e in range(E):
        r = p[e]
        T0 = np.floor(Ainv @ r)
        th = np.zeros(len(sites)); gr = np.zeros((len(sites), 3)); lp = np.zeros(len(sites))
        for dT in itertools.product(rr, rr, rr):
            T = T0 + np.array(dT, dtype=np.float64)
            R = (A @ ((sites + n * T) / n).T).T           # Cartesian site positions
            delta = (J @ (r[None, :] - R).T).T            # offsets in grid units
            b0 = bspline(delta); b1 = bspline_d1(delta); b2 = bspline_d2(delta)
            t = b0[:, 0] * b0[:, 1] * b0[:, 2]
            if not np.any(t != 0.0) and not np.any(b1 != 0.0):
                continue
            dg = np.stack([b1[:, 0] * b0[:, 1] * b0[:, 2],
                           b0[:, 0] * b1[:, 1] * b0[:, 2],
                           b0[:, 0] * b0[:, 1] * b1[:, 2]], axis=1)
            H = np.empty((len(sites), 3, 3))
            for a in range(3):
                for b in range(3):
                    f = [b0[:, 0], b0[:, 1], b0[:, 2]]
                    if a == b:
                        f[a] = b2[:, a]
                    else:
                        f[a] = b1[:, a]
                        f[b] = b1[:, b]
                    H[:, a, b] = f[0] * f[1] * f[2]
            th += t
            gr += dg @ J                                  # grad_r = J^T grad_g
            lp += np.einsum("sab,ac,bc->s", H, J, J)      # sum_ab (J J^T)_ab H_ab
        vals[e] = scale * (th @ cf)
        grads[e] = scale * (gr.T @ cf)
        laps[e] = scale * (lp @ cf)
    return vals, grads, laps


def _site_weights(grid, lattice, pos_e, sites, T0, dT):
    """Cartesian weights of every site for one periodic image: value
    [S], gradient [S][3] and Laplacian [S], from the grid-unit offsets."""
    n = np.array(grid, dtype=np.float64)
    A = np.asarray(lattice, dtype=np.float64).T
    J = np.diag(n) @ np.linalg.inv(A)
    T = T0 + np.array(dT, dtype=np.float64)
    R = (A @ ((sites + n * T) / n).T).T
    delta = (J @ (pos_e[None, :] - R).T).T
    b0 = bspline(delta); b1 = bspline_d1(delta); b2 = bspline_d2(delta)
    th = b0[:, 0] * b0[:, 1] * b0[:, 2]
    dg = np.stack([b1[:, 0] * b0[:, 1] * b0[:, 2],
                   b0[:, 0] * b1[:, 1] * b0[:, 2],
                   b0[:, 0] * b0[:, 1] * b1[:, 2]], axis=1)
    H = np.empty((len(sites), 3, 3))
    for a in range(3):
        for b in range(3):
            f = [b0[:, 0], b0[:, 1], b0[:, 2]]
            if a == b:
                f[a] = b2[:, a]
            else:
                f[a] = b1[:, a]
                f[b] = b1[:, b]
            H[:, a, b] = f[0] * f[1] * f[2]
    return th, dg @ J, np.einsum("sab,ac,bc->s", H, J, J)


def absmag_brute(grid, lattice, coeffs, pos, norm: int = 0, image_radius: int = 2):
    """C [E][5][L]: sum over every (site, periodic image) pair of
    |W_k| |a_ls| for k = value, d/dx, d/dy, d/dz, Laplacian (Eq. 11.12.24.1
    with the weights of Eq. 11.12.24.2 differentiated by the chain rule).

    Each (site, image) pair is one term of the expansion, so its absolute
    weight is taken on its own, after the Jacobian contraction and before
    any sum over images.  Real tables only; tiny grids only."""
    A = np.asarray(lattice, dtype=np.float64).T
    Ainv = np.linalg.inv(A)
    c = np.abs(np.asarray(coeffs, dtype=np.float64))
    L = c.shape[-1]
    cf = c.reshape(-1, L)
    sites = np.array(list(itertools.product(range(grid[0]), range(grid[1]), range(grid[2]))),
                     dtype=np.float64)
    scale = 1.5 ** 3 if norm == 1 else 1.0
    p = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((p.shape[0], 5, L))
    rr = range(-image_radius, image_radius + 1)
    for e in range(p.shape[0]):
        T0 = np.floor(Ainv @ p[e])
        w = np.zeros((len(sites), 5))
        for dT in itertools.product(rr, rr, rr):
            th, gr, lp = _site_weights(grid, lattice, p[e], sites, T0, dT)
            w[:, 0] += np.abs(th)
            w[:, 1:4] += np.abs(gr)
            w[:, 4] += np.abs(lp)
        out[e] = scale * (w.T @ cf)
    return out
