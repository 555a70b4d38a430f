"""Pins for the FP64 oracle: checks against what the mathematics fixes.

Each ``check_*`` function takes an evaluator with the signature of
``oracle.eval_stencil`` and returns the largest normalised error it sees; the
tests assert it is below the stated tolerance, and the mutation test asserts
that an oracle with a planted mistake fails at least one of them.

Nothing here calls the CUDA library.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle
from oracle import brute

RNG = np.random.default_rng(20120404)


def triclinic_lattice():
    """A skewed cell: every off-diagonal entry of A is non-zero."""
    return np.array([[7.0, 0.4, -0.3],
                     [1.1, 6.2, 0.5],
                     [-0.6, 0.9, 5.3]])


def frac_to_cart(lattice, u):
    """r = A u with A's columns the lattice vectors (rows of ``lattice``)."""
    return np.asarray(u) @ np.asarray(lattice)


def _ainv(lattice):
    return np.linalg.inv(np.asarray(lattice, dtype=np.float64).T)


# ---------------------------------------------------------------------------
# 1. the B-spline: closed-form values and continuity at the knots
# ---------------------------------------------------------------------------

def check_bspline_closed_forms(lib=None):
    L = lib or oracle.lib()
    B, dB, d2B = L.oracle_B, L.oracle_dB, L.oracle_d2B
    exact = [
        (B, 0.0, 2.0 / 3.0), (B, 1.0, 1.0 / 6.0), (B, -1.0, 1.0 / 6.0), (B, 2.0, 0.0),
        (B, -2.0, 0.0), (B, 0.5, 23.0 / 48.0), (B, 1.5, 1.0 / 48.0), (B, -1.5, 1.0 / 48.0),
        (B, 3.0, 0.0),
        (dB, 0.0, 0.0), (dB, 1.0, -0.5), (dB, -1.0, 0.5), (dB, 0.5, -5.0 / 8.0),
        (dB, -0.5, 5.0 / 8.0), (dB, 1.5, -1.0 / 8.0), (dB, -1.5, 1.0 / 8.0), (dB, 2.0, 0.0),
        (d2B, 0.0, -2.0), (d2B, 1.0, 1.0), (d2B, -1.0, 1.0), (d2B, 0.5, -0.5),
        (d2B, 1.5, 0.5), (d2B, -1.5, 0.5), (d2B, 2.0, 0.0), (d2B, 2.5, 0.0),
    ]
    return max(abs(f(x) - v) for f, x, v in exact)


def check_bspline_continuity(lib=None):
    """Largest jump of B, B', B'' across the knots 0, +-1, +-2 (step 1e-9)."""
    L = lib or oracle.lib()
    eps = 1e-9
    return max(abs(f(x0 + eps) - f(x0 - eps))
               for x0 in (-2.0, -1.0, 0.0, 1.0, 2.0)
               for f in (L.oracle_B, L.oracle_dB, L.oracle_d2B))


def check_bspline_derivatives_fd(lib=None):
    """B' and B'' against 4th-order central differences inside each piece."""
    L = lib or oracle.lib()
    B, dB, d2B = L.oracle_B, L.oracle_dB, L.oracle_d2B
    h = 1e-3
    err = 0.0
    for x in np.linspace(-2.4, 2.4, 97):
        if min(abs(x - k) for k in (-2, -1, 0, 1, 2)) < 3 * h:
            continue
        fd1 = (8 * (B(x + h) - B(x - h)) - (B(x + 2 * h) - B(x - 2 * h))) / (12 * h)
        fd2 = (8 * (dB(x + h) - dB(x - h)) - (dB(x + 2 * h) - dB(x - 2 * h))) / (12 * h)
        err = max(err, abs(fd1 - dB(x)), abs(fd2 - d2B(x)))
    return err


# ---------------------------------------------------------------------------
# 2. partition of unity: a constant table gives psi = c, grad = lap = 0
# ---------------------------------------------------------------------------

def check_partition_of_unity(ev=oracle.eval_stencil):
    grid = (6, 7, 5)
    lat = triclinic_lattice()
    c0 = np.array([1.0, -2.5, 3.25])
    tab = np.broadcast_to(c0, grid + (3,)).copy()
    u = RNG.uniform(-3.0, 4.0, size=(200, 3))
    pos = frac_to_cart(lat, u)
    err = 0.0
    for norm, scale in ((0, 1.0), (1, 1.5 ** 3)):
        v, g, lp = ev(grid, lat, tab, pos, norm=norm)
        err = max(err, np.abs(v - scale * c0).max() / scale,
                  np.abs(g).max() / scale, np.abs(lp).max() / scale)
    return err


# ---------------------------------------------------------------------------
# 3. exact reproduction of polynomials of degree <= 3 per grid coordinate
# ---------------------------------------------------------------------------

def _qmono(i, x):
    """(1 - d^2/6) x^i: the blip coefficients that reproduce the monomial x^i."""
    return x ** i - (i * (i - 1) / 6.0) * (x ** (i - 2) if i >= 2 else 0.0)


def _dmono(i, k, x):
    """k-th derivative of x^i."""
    if k > i:
        return np.zeros_like(x)
    f = 1.0
    for j in range(k):
        f *= (i - j)
    return f * x ** (i - k)


def check_polynomial_reproduction(ev=oracle.eval_stencil):
    grid = (11, 10, 9)
    lat = triclinic_lattice()
    n = np.array(grid, dtype=np.float64)
    P = RNG.normal(size=(4, 4, 4)) * np.array([1, 0.3, 0.05, 0.005])[:, None, None] \
        * np.array([1, 0.3, 0.05, 0.005])[None, :, None] \
        * np.array([1, 0.3, 0.05, 0.005])[None, None, :]
    m = np.stack(np.meshgrid(*[np.arange(k, dtype=np.float64) for k in grid], indexing="ij"), -1)
    tab = np.zeros(grid + (1,))
    for i, j, k in itertools.product(range(4), repeat=3):
        tab[..., 0] += P[i, j, k] * _qmono(i, m[..., 0]) * _qmono(j, m[..., 1]) * _qmono(k, m[..., 2])
    # positions whose stencils stay inside the grid: g in [1, n - 2)
    g = 1.05 + RNG.uniform(0, 1, size=(300, 3)) * (n - 3.1)
    pos = frac_to_cart(lat, g / n)
    Ainv = _ainv(lat)
    J = np.diag(n) @ Ainv
    M = J @ J.T

    def poly(dx, dy, dz):
        out = np.zeros(len(g))
        for i, j, k in itertools.product(range(4), repeat=3):
            out += P[i, j, k] * _dmono(i, dx, g[:, 0]) * _dmono(j, dy, g[:, 1]) * _dmono(k, dz, g[:, 2])
        return out

    val = poly(0, 0, 0)
    gg = np.stack([poly(1, 0, 0), poly(0, 1, 0), poly(0, 0, 1)], 1)
    grad = gg @ J                                     # J^T grad_g
    H = np.empty((len(g), 3, 3))
    for a in range(3):
        for b in range(3):
            d = [0, 0, 0]
            d[a] += 1
            d[b] += 1
            H[:, a, b] = poly(*d)
    lap = np.einsum("eab,ab->e", H, M)
    v, gr, lp = ev(grid, lat, tab, pos)
    scale = 1.0 + np.abs(val).max()
    return max(np.abs(v[:, 0] - val).max() / scale,
               np.abs(gr[:, :, 0] - grad).max() / (scale * np.abs(J).max()),
               np.abs(lp[:, 0] - lap).max() / (scale * np.abs(M).max()))


# ---------------------------------------------------------------------------
# 4. plane waves: closed-form coefficients interpolate exp(i theta.g) at nodes
# ---------------------------------------------------------------------------

def plane_wave_table(grid, kvec, is_complex):
    """c[m] = prod_a exp(i theta_a m_a) / D(theta_a), theta_a = 2 pi k_a / n_a,
    D(theta) = sum_m B(m) exp(-i theta m) = (2 + cos theta) / 3."""
    th = 2 * np.pi * np.asarray(kvec, dtype=np.float64) / np.asarray(grid, dtype=np.float64)
    D = (2.0 + np.cos(th)) / 3.0
    m = np.stack(np.meshgrid(*[np.arange(k, dtype=np.float64) for k in grid], indexing="ij"), -1)
    c = np.exp(1j * (m @ th)) / np.prod(D)
    return (c if is_complex else c.real)[..., None], th, D


def check_plane_wave_nodes(ev=oracle.eval_stencil):
    lat = triclinic_lattice()
    err = 0.0
    for grid, kvec, cplx in (((8, 7, 9), (1, 2, -3), True), ((8, 7, 9), (3, -1, 2), False),
                             ((5, 6, 4), (2, 1, 1), True), ((12, 12, 12), (5, 0, -4), False)):
        n = np.array(grid, dtype=np.float64)
        tab, th, D = plane_wave_table(grid, kvec, cplx)
        Ainv = _ainv(lat)
        J = np.diag(n) @ Ainv
        M = J @ J.T
        # nodes, including far periodic images and negative images
        mm = np.stack([RNG.integers(0, k, 60) for k in grid], 1).astype(np.float64)
        T = RNG.integers(-4, 5, size=(60, 3)).astype(np.float64)
        pos = frac_to_cart(lat, (mm + n * T) / n)
        ph = np.exp(1j * (mm @ th))
        d1 = 1j * np.sin(th) / D                         # d/dg_a at a node
        d2 = (2 * np.cos(th) - 2) / D                    # d^2/dg_a^2 at a node
        val = ph
        gg = ph[:, None] * d1[None, :]
        H = ph[:, None, None] * (d1[:, None] * d1[None, :])[None]
        for a in range(3):
            H[:, a, a] = ph * d2[a]
        grad = gg @ J
        lap = np.einsum("eab,ab->e", H, M)
        if not cplx:
            val, grad, lap = val.real, grad.real, lap.real
        v, gr, lp = ev(grid, lat, tab, pos)
        err = max(err, np.abs(v[:, 0] - val).max(),
                  np.abs(gr[:, :, 0] - grad).max() / np.abs(J).max(),
                  np.abs(lp[:, 0] - lap).max() / np.abs(M).max())
    return err


# ---------------------------------------------------------------------------
# 5. finite differences of psi and grad psi
# ---------------------------------------------------------------------------

def check_finite_differences(ev=oracle.eval_stencil):
    grid = (9, 8, 10)
    lat = triclinic_lattice()
    n = np.array(grid, dtype=np.float64)
    tab = RNG.normal(size=grid + (4,))
    # keep every grid coordinate away from knots so the 5-point stencil
    # stays inside one cubic piece
    g = RNG.integers(0, 7, size=(40, 3)) + RNG.uniform(0.2, 0.8, size=(40, 3))
    pos = frac_to_cart(lat, g / n)
    h = 1e-4
    v0, g0, l0 = ev(grid, lat, tab, pos)
    fd_g = np.zeros_like(g0)
    fd_l = np.zeros_like(l0)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        vals = {}
        for s in (-2, -1, 1, 2):
            vals[s] = ev(grid, lat, tab, pos + s * e)
        fd_g[:, c, :] = (8 * (vals[1][0] - vals[-1][0]) - (vals[2][0] - vals[-2][0])) / (12 * h)
        fd_l += (8 * (vals[1][1][:, c] - vals[-1][1][:, c])
                 - (vals[2][1][:, c] - vals[-2][1][:, c])) / (12 * h)
    s1 = np.abs(g0).max()
    s2 = np.abs(l0).max()
    return max(np.abs(fd_g - g0).max() / s1, np.abs(fd_l - l0).max() / s2)


# ---------------------------------------------------------------------------
# 6. stencil sum == brute-force sum over all sites and images
# ---------------------------------------------------------------------------

def check_vs_bruteforce(ev=oracle.eval_stencil):
    lat = triclinic_lattice()
    err = 0.0
    for grid in ((4, 4, 4), (5, 4, 7), (7, 8, 5), (8, 8, 8)):
        n = np.array(grid, dtype=np.float64)
        tab = RNG.normal(size=grid + (3,))
        u = [RNG.uniform(-2.0, 3.0, size=(12, 3)),                     # negatives and images
             RNG.uniform(0, 1, size=(4, 3)) + RNG.integers(-9, 10, size=(4, 3)),  # far images
             (RNG.integers(0, 8, size=(4, 3)) % n) / n,                # exact nodes
             np.full((1, 3), 1.0 - 2.0 ** -53),                         # u just below 1
             np.full((1, 3), -2.0 ** -60),                              # u just below 0
             np.array([[0.0, 0.5, 1.0]])]
        pos = frac_to_cart(lat, np.concatenate(u))
        v, g, lp = ev(grid, lat, tab, pos)
        vb, gb, lb = brute.eval_brute(grid, lat, tab, pos)
        err = max(err, np.abs(v - vb).max() / (1 + np.abs(vb).max()),
                  np.abs(g - gb).max() / (1 + np.abs(gb).max()),
                  np.abs(lp - lb).max() / (1 + np.abs(lb).max()))
    return err


# ---------------------------------------------------------------------------
# 7. periodicity and grid-shift equivariance
# ---------------------------------------------------------------------------

def check_translation(ev=oracle.eval_stencil):
    grid = (6, 9, 7)
    lat = triclinic_lattice()
    tab = RNG.normal(size=grid + (3,))
    pos = frac_to_cart(lat, RNG.uniform(-1, 2, size=(50, 3)))
    base = ev(grid, lat, tab, pos)
    err = 0.0
    for a in range(3):
        moved = ev(grid, lat, tab, pos + 2 * lat[a] - 3 * lat[(a + 1) % 3])
        for x, y in zip(base, moved):
            err = max(err, np.abs(x - y).max() / (1 + np.abs(x).max()))
        # rolling the table by one node along a == translating r by one grid step
        rolled = np.roll(tab, 1, axis=a)
        shifted = ev(grid, lat, rolled, pos + lat[a] / grid[a])
        for x, y in zip(base, shifted):
            err = max(err, np.abs(x - y).max() / (1 + np.abs(x).max()))
    return err


# ---------------------------------------------------------------------------
# 8. the rounding scale C_o = sum_s |W_o(s)| |a_ls| that the oracle returns
#    beside every output (the GPU parity bounds are multiples of it)
# ---------------------------------------------------------------------------

def check_absmag_vs_bruteforce(ev=oracle.eval_stencil):
    """C_o of the stencil oracle against Oracle B's independent sum over
    every (site, image) pair of |W_k| |a_ls| (Eqs. 11.12.24.1, 11.12.24.2:
    each pair is one term, its weight taken after the Jacobian contraction),
    on triclinic tiny grids with coefficients of both signs, for all five
    output kinds and both normalisations."""
    lat = triclinic_lattice()
    err = 0.0
    for grid, norm in (((4, 4, 4), 0), ((5, 4, 7), 1), ((7, 6, 5), 0)):
        n = np.array(grid, dtype=np.float64)
        tab = RNG.normal(size=grid + (3,))
        u = np.concatenate([RNG.uniform(-2.0, 3.0, size=(8, 3)),
                            (RNG.integers(0, 8, size=(2, 3)) % n) / n])
        pos = frac_to_cart(lat, u)
        _, _, _, mag = ev(grid, lat, tab, pos, norm=norm, absmag=True)
        ref = brute.absmag_brute(grid, lat, tab, pos, norm=norm)
        err = max(err, float(np.max(np.abs(mag - ref) / (np.abs(ref) + 1e-300))))
    return err


def _exact_1d(t):
    """Exact (b, b', b'') of the 4 stencil sites at offset t in {0, 1/2}:
    site k sits at grid distance t + 1 - k, and B, B', B'' at the distances
    1, 0, -1, -2 and 3/2, 1/2, -1/2, -3/2 are the rationals of the golden
    B-spline table."""
    from fractions import Fraction as F
    if t == 0:
        return ([F(1, 6), F(2, 3), F(1, 6), F(0)], [F(-1, 2), F(0), F(1, 2), F(0)],
                [F(1), F(-2), F(1), F(0)])
    return ([F(1, 48), F(23, 48), F(23, 48), F(1, 48)], [F(-1, 8), F(-5, 8), F(5, 8), F(1, 8)],
            [F(1, 2), F(-1, 2), F(-1, 2), F(1, 2)])


def check_absmag_closed_forms(ev=oracle.eval_stencil):
    """C_o for a table of ones on an orthorhombic cell with J = diag(1, 2, 2),
    at offsets t_a in {0, 1/2}, against exact rational sums:
    C_value = 1 (non-negative weights, partition of unity);
    C_d/dx_a = J_aa sum_k |b'_k(t_a)| (the other two factors sum to 1);
    C_lap = sum over the 64 sites of |sum_a J_aa^2 b''_a prod_{b != a} b_b|
    (the absolute value of the combined weight, not of its three terms)."""
    from fractions import Fraction as F
    lat = np.diag([8.0, 6.0, 5.0])
    grid = (8, 12, 10)
    jd = [F(1), F(2), F(2)]                        # n_a / |a_a|
    err = 0.0
    for tt in ((0, 0, 0), (1, 1, 1), (0, 1, 0), (1, 0, 1)):
        t = [F(k, 2) for k in tt]
        g = [F(3) + t[0], F(5) + t[1], F(7) + t[2]]
        pos = np.array([[float(g[a] / grid[a]) * lat[a, a] for a in range(3)]])
        f = [_exact_1d(x) for x in t]
        cv = F(0)
        cl = F(0)
        for kx, ky, kz in itertools.product(range(4), repeat=3):
            k = (kx, ky, kz)
            b = [f[a][0][k[a]] for a in range(3)]
            cv += abs(b[0] * b[1] * b[2])
            lap = F(0)
            for a in range(3):
                term = jd[a] ** 2 * f[a][2][k[a]]
                for c in range(3):
                    if c != a:
                        term *= b[c]
                lap += term
            cl += abs(lap)
        cg = [jd[a] * sum(abs(x) for x in f[a][1]) for a in range(3)]
        for norm, s in ((0, 1.0), (1, 1.5 ** 3)):
            _, _, _, mag = ev(grid, lat, np.ones(grid + (1,)), pos, norm=norm, absmag=True)
            want = np.array([float(cv)] + [float(x) for x in cg] + [float(cl)]) * s
            err = max(err, float(np.max(np.abs(mag[0, :, 0] - want) / want)))
    return err
