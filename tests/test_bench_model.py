"""The benchmark's traffic model: U, the number of distinct grid sites a
launch's 4 x 4 x 4 stencils touch (the compulsory-bytes term U L b_c of the
roofline), counted by bench.touched_sites.  Checked on the CPU against a
brute-force set of the sites, against the cases with a known answer, and
against the expected value P (1 - exp(-64 E / P)) for uniform positions."""
import os
import sys

import numpy as np

import blip_inputs as bi
import pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _brute_sites(grid, lattice, pos):
    n = np.array(grid)
    sites = set()
    for r in pos:
        u = np.linalg.solve(np.asarray(lattice).T, r)     # r = u @ lattice
        u = u - np.floor(u)
        u[u >= 1.0] = 0.0
        base = np.floor(u * n).astype(int) % n
        for kx in range(4):
            for ky in range(4):
                for kz in range(4):
                    m = (base + np.array([kx, ky, kz]) - 1) % n
                    sites.add(tuple(int(x) for x in m))
    return len(sites)


def test_touched_sites_matches_a_brute_force_count():
    # positions off the node planes: on a plane the anchor cell is decided by
    # the last bit of the FP64 reduction (either choice gives the same
    # values, the far slab's weight being B(2) = 0), so counts made with
    # different arithmetic may differ by a slab there
    lat = pins.triclinic_lattice()
    rng = np.random.default_rng(3)
    for grid in [(7, 9, 11), (5, 6, 4), (12, 10, 8)]:
        n = np.array(grid)
        u = rng.uniform(-2, 3, size=(60, 3))
        frac = (u * n) % 1.0
        u = u[((frac > 1e-6) & (frac < 1 - 1e-6)).all(1)]
        pos = u @ lat
        assert bench.touched_sites(grid, lat, pos) == _brute_sites(grid, lat, pos), grid


def test_touched_sites_known_cases():
    lat = np.diag([9.0, 8.0, 11.0])
    one = np.array([[1.3, 2.2, 5.5]])
    assert bench.touched_sites((20, 20, 20), lat, one) == 64
    # a repeated position, and its periodic image, add nothing
    rep = np.concatenate([one, one, one + lat[0] - 2 * lat[2]])
    assert bench.touched_sites((20, 20, 20), lat, rep) == 64
    # on a 4-point grid every stencil covers the whole grid
    pos = bi.uniform_positions(lat, 10, seed=1)
    assert bench.touched_sites((4, 4, 4), lat, pos) == 64
    assert bench.touched_sites((4, 5, 4), lat, pos) <= 80
    # two electrons in neighbouring cells along a_1 share 3 of 4 slabs
    g = np.array([20, 20, 20])
    a = (np.array([5.5, 7.5, 9.5]) / g) @ lat
    b = (np.array([6.5, 7.5, 9.5]) / g) @ lat
    assert bench.touched_sites(tuple(g), lat, np.stack([a, b])) == 64 + 16


def test_touched_sites_expected_value_for_uniform_positions():
    # P sites, E uniform electrons: each site is missed by one stencil with
    # probability 1 - 64/P, so E[U] = P (1 - (1 - 64/P)^E) ~ P (1 - exp(-64 E / P))
    w = bi.workload("tio2")
    pos, _ = w.positions()
    P = int(np.prod(w.grid))
    E = len(pos)
    expect = P * (1.0 - (1.0 - 64.0 / P) ** E)
    got = bench.touched_sites(w.grid, w.lattice, pos)
    assert abs(got - expect) / expect < 0.01
    assert got == 81324                       # the headline launch's figure
