"""Staged-tile kernel (variant 8) on dense batches.

The kernel copies the union of the stencil rows of 2 x 2 x TZ cells into
shared memory and contracts every electron of those cells from there.  Its
per-site FMA order is the register kernels', so outputs must be bitwise equal
to them; they are also checked against the FP64 oracle under the parity
bound (FP32: 8e-6 x sum_s |W||a|; quantised tables add the storage unit
roundoff).  Cases: clusters of more than 32 electrons in one tile (several
parts per tile), tiles cut by odd grid sizes along every axis, grids of 4
points (the 5-column union wraps onto itself), periodic images, far and
non-finite positions, values-only, every storage kind, and the full-size
TiO2-shaped batches in the benchmark's launch configuration.
"""
import numpy as np
import pytest

import blip_inputs as bi
import pins
from gpu_util import cached_table, compare, gpu_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _dense_positions(lat, grid, rng, background=2000):
    n = np.array(grid, dtype=np.float64)
    u = [rng.uniform(0, 1, size=(background, 3))]
    for k in (40, 70, 33, 5, 97):                  # one cell holding k electrons
        c = rng.integers(0, grid)
        u.append((c + rng.uniform(0.01, 0.99, size=(k, 3))) / n)
    last = n - 1                                   # the cell of the last tile on every axis
    u.append((last + rng.uniform(0, 1, size=(25, 3))) / n)
    u.append((rng.integers(0, 64, size=(16, 3)) % n) / n)          # exact grid nodes
    u.append(np.array([[1.0 - 2.0 ** -53] * 3, [-2.0 ** -60] * 3]))
    u = np.concatenate(u)
    u = np.concatenate([u, u[:60] + rng.integers(-3, 4, size=(60, 3))])   # periodic images
    pos = u @ lat
    pos = np.concatenate([pos, [[np.nan, 0.0, 0.0], [0.0, np.inf, 1.0], [1e13, 0.0, 0.0]]])
    rng.shuffle(pos)
    return pos


def _scales(tab):
    if np.iscomplexobj(tab):
        r = np.abs(tab.view(np.float64).reshape(-1, 2 * tab.shape[-1])).max(0)
        r = np.maximum(r[0::2], r[1::2]).repeat(2)
    else:
        r = np.abs(tab.reshape(-1, tab.shape[-1])).max(0)
    return np.where(r > 0, r, 1.0)


@pytest.mark.parametrize("grid,n_orb,storage", [
    ((5, 7, 9), 300, "f32"),        # odd sizes: partial tiles on every axis, 3 chunks (last partial)
    ((8, 8, 8), 128, "f32"),
    ((4, 6, 4), 129, "f32"),        # 4-point axes: union columns wrap onto themselves
    ((5, 7, 9), 300, "bf16"),
    ((6, 5, 7), 520, "f16"),
    ((5, 7, 9), 70, "c64"),
])
def test_staged_matches_register_kernel_and_oracle(pb, grid, n_orb, storage):
    rng = np.random.default_rng(grid[0] * 10007 + grid[2] * 101 + n_orb + len(storage))
    lat = pins.triclinic_lattice()
    cplx = storage == "c64"
    tab = bi.smooth_random_table(grid, n_orb, seed=41, is_complex=cplx)
    pos = _dense_positions(lat, grid, rng)
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16, "c64": pb.C64}[storage]
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    t.set_kernel(1, 1, 8, 0)
    ref = gpu_eval(t, pos)
    ref_vo = gpu_eval(t, pos, values_only=True)
    t.status()
    for tz, cw in ((2, 16), (4, 16), (2, 12), (4, 12)):
        t.set_kernel(8, tz, cw, 1)
        out = gpu_eval(t, pos)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b, equal_nan=True), (tz, cw)
        st = t.status()
        assert st & pb.STATUS_NONFINITE_POS and st & pb.STATUS_FAR_POS
        vo = gpu_eval(t, pos, values_only=True)
        assert np.array_equal(ref_vo[0], vo[0], equal_nan=True), (tz, cw)
        t.status()
    bad = ~np.isfinite(pos).all(1)
    assert np.isnan(ref[0][bad]).all() and np.isnan(ref[1][bad]).all()
    # the far position (|u| > 2^40, flagged) keeps only a few fractional bits,
    # so its value depends on the last bits of A^-1: checked for the flag only
    good = ~bad & (np.abs(pos).max(1) < 1e9)
    compare(grid, lat, tab, pos[good], [r[good] for r in ref], storage=kind,
            scales=None if kind == pb.F32 or cplx else _scales(tab),
            sample=np.random.default_rng(5).choice(good.sum(), 300, replace=False))


def test_staged_with_walker_offsets_and_ragged_batches(pb):
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 200, seed=42)
    sizes = [300, 1, 0, 517, 64, 999, 2]
    pos, offs = bi.walker_positions(lat, len(sizes), 1000, sizes, seed=42)
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(3, 1, 8, 0)
    ref = gpu_eval(t, pos, offsets=offs)
    for tz, cw in ((2, 16), (4, 12)):
        t.set_kernel(8, tz, cw, 1)
        out = gpu_eval(t, pos, offsets=offs)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b), (tz, cw)
    assert t.status() == 0
    bad = offs.copy()
    bad[3] = bad[2] - 1
    gpu_eval(t, pos, offsets=bad)
    assert t.status() & pb.STATUS_BAD_OFFSETS


def test_staged_sparse_batch_and_single_electron(pb):
    """Few electrons per tile (most tiles empty), one electron, and a batch
    whose positions are all non-finite."""
    grid = (12, 10, 14)
    lat = np.diag([9.0, 8.0, 11.0])
    tab = bi.smooth_random_table(grid, 256, seed=43)
    t = pb.BlipTable(grid, lat, tab)
    for pos in (bi.uniform_positions(lat, 37, seed=43), bi.uniform_positions(lat, 1, seed=44)):
        t.set_kernel(1, 1, 8, 0)
        ref = gpu_eval(t, pos)
        t.set_kernel(8, 4, 16, 1)
        out = gpu_eval(t, pos)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b)
        compare(grid, lat, tab, pos, out)
    assert t.status() == 0
    nanpos = np.full((5, 3), np.nan)
    v, g, lp = gpu_eval(t, nanpos)
    assert np.isnan(v).all() and np.isnan(g).all() and np.isnan(lp).all()
    assert t.status() & pb.STATUS_NONFINITE_POS


def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, size=k)]))


@pytest.mark.parametrize("name,storage,tz,cw", [("tio2_batch", "f32", 4, 12),
                                                ("tio2_batch", "f32", 2, 16),
                                                ("tio2_precision", "bf16", 4, 16)])
def test_staged_full_size_tio2(pb, name, storage, tz, cw):
    """Full-size TiO2-shaped table (72 x 72 x 48, 768 orbitals): 256 walkers x
    1,536 moved electrons, or 64 walkers of the precision workload in BF16;
    sampled electrons against the oracle, a slice against the register
    kernel bitwise."""
    w, tab = cached_table("tio2")
    wl = bi.workload(name, batch=1536) if name == "tio2_batch" else bi.workload(name, n_walkers=64)
    pos, offs = wl.positions()
    kind = pb.F32 if storage == "f32" else pb.BF16
    t = pb.BlipTable(wl.grid, wl.lattice, tab, storage=kind)
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    t.set_kernel(8, tz, cw, 1)
    v, g, lp = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    assert t.status() == 0
    idx = _sample(len(pos), 48, tz)
    sub = [v[idx].cpu().numpy(), g[idx].cpu().numpy(), lp[idx].cpu().numpy()]
    compare(wl.grid, wl.lattice, tab, pos[idx], sub, storage=kind,
            scales=None if kind == pb.F32 else _scales(tab))
    # bitwise against the register kernel on a contiguous slice
    t.set_kernel(3, 1, 8, 0)
    sl = slice(0, 4096)
    rv, rg, rl = t.eval(dpos[sl].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(rv, v[sl]) and torch.equal(rg, g[sl]) and torch.equal(rl, lp[sl])


def test_staged_in_a_cuda_graph(pb):
    """The sorted staged-tile evaluation captured into a CUDA graph (after one
    eager call has grown the sort scratch) replays bitwise equal to the eager
    call, including after the positions change in place."""
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=44)
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(8, 4, 12, 1)
    pos_a = bi.uniform_positions(lat, 6000, seed=45)
    pos_b = bi.uniform_positions(lat, 6000, seed=46)
    dpos = torch.from_numpy(pos_a).cuda()
    t.eval(dpos)                       # grows the sort scratch outside capture
    torch.cuda.synchronize()
    out = t.alloc_outputs(len(pos_a))
    gr = t.graph(dpos, out, per_launch=len(pos_a))
    for p_np in (pos_a, pos_b):
        dpos.copy_(torch.from_numpy(p_np))
        ref = t.eval(dpos.clone())
        gr.launch()
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            assert torch.equal(r, o)
    gr.close()
    assert t.status() == 0
