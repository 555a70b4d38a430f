"""The FP64 oracle against what the paper and the mathematics fix.

Eq. 11.12.24.1 (the 64-term blip expansion), Eq. 11.12.24.2 (the
tensor-product basis, phi read as the centred cubic B-spline) and Eq. 7 (the
stencil of 4 sites per direction) define the oracle; these pins check it
without comparing it to itself.
"""
import numpy as np
import pytest

import oracle
import pins


def test_bspline_closed_forms():
    assert pins.check_bspline_closed_forms() < 1e-15


def test_bspline_continuity():
    assert pins.check_bspline_continuity() < 1e-8


def test_bspline_derivatives_match_fd():
    assert pins.check_bspline_derivatives_fd() < 1e-9


def test_partition_of_unity_and_zero_sum_derivatives():
    assert pins.check_partition_of_unity() < 1e-13


def test_cubic_polynomial_reproduction_triclinic():
    assert pins.check_polynomial_reproduction() < 1e-12


def test_plane_waves_interpolated_at_nodes_with_images():
    assert pins.check_plane_wave_nodes() < 1e-12


def test_finite_differences():
    assert pins.check_finite_differences() < 1e-7


def test_stencil_equals_bruteforce_on_tiny_grids():
    assert pins.check_vs_bruteforce() < 1e-13


def test_periodicity_and_grid_shift():
    assert pins.check_translation() < 1e-12


def test_absmag_equals_bruteforce_sum_of_absolute_terms():
    """The rounding scale C_o = sum_s |W_o(s)| |a_ls| of all five output
    kinds (Eqs. 11.12.24.1, 11.12.24.2) against Oracle B's independent sum
    over every (site, image) pair: pinned from above and below."""
    assert pins.check_absmag_vs_bruteforce() < 1e-12


def test_absmag_closed_forms_orthorhombic():
    assert pins.check_absmag_closed_forms() < 1e-13


def test_golden_bspline_table():
    """Exact rational values of B, B', B'' (tests/golden/bspline_values.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bspline_values.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 9
    for x, b, db, d2b in rows:
        from fractions import Fraction as F
        assert oracle.B(float(F(x))) == pytest.approx(float(F(b)), abs=1e-16)
        assert oracle.dB(float(F(x))) == pytest.approx(float(F(db)), abs=1e-16)
        assert oracle.d2B(float(F(x))) == pytest.approx(float(F(d2b)), abs=1e-16)


def test_nonfinite_position_gives_nan():
    grid = (4, 4, 4)
    tab = np.ones(grid + (2,))
    pos = np.array([[np.nan, 0, 0], [0.1, 0.2, 0.3], [np.inf, 1, 1]])
    v, g, l = oracle.eval_stencil(grid, np.eye(3) * 4, tab, pos)
    assert np.isnan(v[0]).all() and np.isnan(v[2]).all() and np.isnan(l[0]).all()
    assert np.allclose(v[1], 1.0)


def test_thread_count_does_not_change_results():
    grid = (6, 6, 6)
    rng = np.random.default_rng(3)
    tab = rng.normal(size=grid + (5,))
    pos = rng.uniform(-5, 10, size=(37, 3))
    a = oracle.eval_stencil(grid, pins.triclinic_lattice(), tab, pos, threads=1)
    b = oracle.eval_stencil(grid, pins.triclinic_lattice(), tab, pos, threads=7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_complex_table_splits_into_parts():
    grid = (5, 6, 7)
    rng = np.random.default_rng(4)
    re = rng.normal(size=grid + (3,))
    im = rng.normal(size=grid + (3,))
    pos = rng.uniform(-3, 9, size=(11, 3))
    lat = pins.triclinic_lattice()
    vc, gc, lc = oracle.eval_stencil(grid, lat, re + 1j * im, pos)
    vr, gr, lr = oracle.eval_stencil(grid, lat, re, pos)
    vi, gi, li = oracle.eval_stencil(grid, lat, im, pos)
    assert np.allclose(vc, vr + 1j * vi, atol=1e-14)
    assert np.allclose(gc, gr + 1j * gi, atol=1e-13)
    assert np.allclose(lc, lr + 1j * li, atol=1e-12)


def test_absmag_bounds_outputs():
    grid = (6, 5, 7)
    rng = np.random.default_rng(5)
    tab = rng.normal(size=grid + (4,))
    pos = rng.uniform(-3, 9, size=(20, 3))
    v, g, l, mag = oracle.eval_stencil(grid, pins.triclinic_lattice(), tab, pos, absmag=True)
    assert (np.abs(v) <= mag[:, 0] + 1e-14).all()
    for c in range(3):
        assert (np.abs(g[:, c]) <= mag[:, 1 + c] + 1e-13).all()
    assert (np.abs(l) <= mag[:, 4] + 1e-12).all()
    # the value weights are non-negative B-spline products summing to 1
    assert np.allclose(mag[:, 0], oracle.eval_stencil(grid, pins.triclinic_lattice(),
                                                      np.abs(tab), pos)[0])


def test_local_kinetic_closed_form():
    """Orbitals with lap psi_l = -k_l^2 psi_l give T_L = 1/2 sum_sigma sum_l k_l^2."""
    rng = np.random.default_rng(6)
    n = 12
    k2 = rng.uniform(0.5, 3.0, size=n)
    vals = rng.normal(size=(2 * n, n))
    laps = -vals * k2[None, :]
    T, conds = oracle.kinetic.local_kinetic(vals, laps, [(0, n), (n, 2 * n)])
    assert T == pytest.approx(0.5 * 2 * k2.sum(), rel=1e-12)
    assert len(conds) == 2 and all(c >= 1 for c in conds)


def test_local_kinetic_detects_swapped_index():
    """A transposed Laplacian matrix changes T_L (so the index order is pinned)."""
    rng = np.random.default_rng(7)
    n = 8
    vals = rng.normal(size=(n, n))
    laps = rng.normal(size=(n, n))
    T, _ = oracle.kinetic.local_kinetic(vals, laps, [(0, n)])
    ref = -0.5 * sum(laps[j, l] * np.linalg.inv(vals)[l, j] for j in range(n) for l in range(n))
    assert T == pytest.approx(ref, rel=1e-10)
    Tt, _ = oracle.kinetic.local_kinetic(vals, laps.T, [(0, n)])
    assert abs(Tt - T) > 1e-6


def _bloch_case():
    rng = np.random.default_rng(31)
    grid = (7, 6, 8)
    lat = pins.triclinic_lattice()
    tab = rng.normal(size=grid + (5,)) + 1j * rng.normal(size=grid + (5,))
    kfrac = np.array([[0.0, 0.0, 0.0], [0.25, -0.5, 0.125], [0.5, 0.5, 0.5]])
    koffs = [0, 1, 3, 5]
    return grid, lat, tab, kfrac, koffs, rng


def test_bloch_constant_u_is_a_plane_wave():
    """u = c gives psi = c e^{ik.r}, grad = i k psi, lap = -|k|^2 psi."""
    grid, lat, _, kfrac, koffs, rng = _bloch_case()
    c = np.array([1.0 + 0.5j, -0.3 + 2j, 0.7 - 1j, 2.0 + 0j, -1j])
    tab = np.broadcast_to(c, grid + (5,)).copy()
    pos = rng.uniform(-5, 12, size=(30, 3))
    v, g, lp = oracle.bloch.eval_bloch(grid, lat, tab, pos, kfrac, koffs)
    kcart = 2 * np.pi * kfrac @ np.linalg.inv(lat.T)
    for q in range(3):
        for l in range(koffs[q], koffs[q + 1]):
            k = kcart[q]
            ref = c[l] * np.exp(1j * pos @ k)
            assert np.abs(v[:, l] - ref).max() < 1e-12
            assert np.abs(g[:, :, l] - 1j * k[None, :] * ref[:, None]).max() < 1e-11
            assert np.abs(lp[:, l] + (k @ k) * ref).max() < 1e-10


def test_bloch_theorem_translation():
    """psi(r + R) = e^{ik.R} psi(r) for a lattice vector R."""
    grid, lat, tab, kfrac, koffs, rng = _bloch_case()
    pos = rng.uniform(0, 6, size=(20, 3))
    R = 2 * lat[0] - lat[1] + 3 * lat[2]
    a = oracle.bloch.eval_bloch(grid, lat, tab, pos, kfrac, koffs)
    b = oracle.bloch.eval_bloch(grid, lat, tab, pos + R, kfrac, koffs)
    kcart = 2 * np.pi * kfrac @ np.linalg.inv(lat.T)
    for q in range(3):
        f = np.exp(1j * kcart[q] @ R)
        sl = slice(koffs[q], koffs[q + 1])
        assert np.abs(b[0][:, sl] - f * a[0][:, sl]).max() < 1e-11
        assert np.abs(b[1][:, :, sl] - f * a[1][:, :, sl]).max() < 1e-10
        assert np.abs(b[2][:, sl] - f * a[2][:, sl]).max() < 1e-9


def test_bloch_finite_differences():
    grid, lat, tab, kfrac, koffs, rng = _bloch_case()
    n = np.array(grid, dtype=np.float64)
    g = rng.integers(0, 5, size=(12, 3)) + rng.uniform(0.2, 0.8, size=(12, 3))
    pos = (g / n) @ lat
    h = 1e-4
    v0, g0, l0 = oracle.bloch.eval_bloch(grid, lat, tab, pos, kfrac, koffs)
    fdg = np.zeros_like(g0)
    fdl = np.zeros_like(l0)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        vals = {s: oracle.bloch.eval_bloch(grid, lat, tab, pos + s * e, kfrac, koffs)
                for s in (-2, -1, 1, 2)}
        fdg[:, c] = (8 * (vals[1][0] - vals[-1][0]) - (vals[2][0] - vals[-2][0])) / (12 * h)
        fdl += (8 * (vals[1][1][:, c] - vals[-1][1][:, c])
                - (vals[2][1][:, c] - vals[-2][1][:, c])) / (12 * h)
    assert np.abs(fdg - g0).max() / np.abs(g0).max() < 1e-7
    assert np.abs(fdl - l0).max() / np.abs(l0).max() < 1e-6


def test_bloch_gamma_point_is_the_plain_expansion():
    grid, lat, tab, _, _, rng = _bloch_case()
    pos = rng.uniform(-3, 9, size=(15, 3))
    a = oracle.bloch.eval_bloch(grid, lat, tab, pos, [[0, 0, 0]], [0, 5])
    b = oracle.eval_stencil(grid, lat, tab, pos)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_sherman_morrison_matches_direct_inverse():
    rng = np.random.default_rng(51)
    n = 40
    D = rng.normal(size=(n, n)) + 4 * np.eye(n)
    Dinv = np.linalg.inv(D)
    for j in (0, 17, n - 1):
        row = rng.normal(size=n)
        new, w = oracle.sherman_morrison.sm_update(Dinv, row, j)
        D2 = D.copy()
        D2[j] = row
        assert np.abs(new - np.linalg.inv(D2)).max() < 1e-10 * np.linalg.cond(D2)
        assert np.abs(D2 @ new - np.eye(n)).max() < 1e-10 * np.linalg.cond(D2)
        # w_j is the determinant ratio det(D') / det(D)
        assert w[j] == pytest.approx(np.linalg.det(D2) / np.linalg.det(D), rel=1e-9)


def test_sherman_morrison_unchanged_row_is_identity():
    rng = np.random.default_rng(52)
    n = 16
    D = rng.normal(size=(n, n)) + 3 * np.eye(n)
    Dinv = np.linalg.inv(D)
    new, w = oracle.sherman_morrison.sm_update(Dinv, D[5], 5)
    assert w[5] == pytest.approx(1.0, abs=1e-12)
    assert np.abs(new - Dinv).max() < 1e-12 * np.abs(Dinv).max()
