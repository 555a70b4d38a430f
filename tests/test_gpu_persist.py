"""Persistent two-batch register kernel (variant 11).

A grid of resident warps walks the (electron, chunk) items; each warp
prefetches the next item's position (or its sort record) and runs its FP64
wrap while the current item's rows are in flight.  The arithmetic is the
two-batch kernel's (variant 9), so the outputs must be bitwise equal to it;
they are also checked against the FP64 oracle under the parity bound.
Cases: many items per warp (the item walk and the stride arithmetic,
input order and both sorted orders), non-finite and far positions between
ordinary ones (the path that skips the rows and takes the next geometry
synchronously), ragged walker batches, values only, a CUDA graph, the
full-size TiO2-shaped headline batch, and the configurations it refuses.
The measurement probe built from the same kernel (blip_probe_gather) is
checked to load exactly the rows an evaluation loads.
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


def _positions_with_bad_entries(lat, n, seed):
    pos = bi.uniform_positions(lat, n, seed=seed)
    rng = np.random.default_rng(seed)
    # non-finite and far positions scattered through the batch, and a run of
    # consecutive ones, so warps meet them before, after and between others
    at = rng.choice(n, size=40, replace=False)
    pos[at[:10]] = np.nan
    pos[at[10:20], 1] = np.inf
    pos[at[20:30]] = [1e13, -2e13, 5e12]
    pos[at[30:40]] = pos[at[30:40]] + rng.integers(-40, 40, size=(10, 3)) @ lat
    pos[n // 2:n // 2 + 7] = np.nan
    return pos


@pytest.mark.parametrize("sort", [0, 1, 2])
def test_persist_bitwise_equal_to_two_batch_kernel(pb, sort):
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 700, seed=61)          # 6 chunks, the last partial
    pos = _positions_with_bad_entries(lat, 30000, seed=61 + sort)   # ~70 items per warp
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(9, 1, 4, sort)
    ref = gpu_eval(t, pos)
    ref_vo = gpu_eval(t, pos, values_only=True)
    st_ref = t.status()
    assert st_ref & pb.STATUS_NONFINITE_POS and st_ref & pb.STATUS_FAR_POS
    for w in (1, 4, 16):
        t.set_kernel(11, 1, w, sort)
        out = gpu_eval(t, pos)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b, equal_nan=True), (w, sort)
        vo = gpu_eval(t, pos, values_only=True)
        assert np.array_equal(ref_vo[0], vo[0], equal_nan=True), (w, sort)
        assert t.status() == st_ref
    bad = ~np.isfinite(pos).all(1)
    assert np.isnan(ref[0][bad]).all() and np.isnan(ref[1][bad]).all()
    good = ~bad & (np.abs(pos).max(1) < 1e9)
    sample = np.flatnonzero(good)[np.random.default_rng(sort).choice(good.sum(), 200, replace=False)]
    compare(grid, lat, tab, pos[sample], [r[sample] for r in ref])


def test_persist_with_walker_offsets(pb):
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 256, seed=62)
    sizes = [300, 1, 0, 5170, 64, 999, 2, 4000]
    pos, offs = bi.walker_positions(lat, len(sizes), 6000, sizes, seed=62)
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(3, 1, 8, 0)
    ref = gpu_eval(t, pos, offsets=offs)
    for cfg in ((11, 1, 4, 0), (11, 1, 8, 1), (11, 1, 2, 2)):
        t.set_kernel(*cfg)
        out = gpu_eval(t, pos, offsets=offs)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b), cfg
    assert t.status() == 0
    bad = offs.copy()
    bad[3] = bad[2] - 1
    t.set_kernel(11, 1, 4, 0)
    gpu_eval(t, pos, offsets=bad)
    assert t.status() & pb.STATUS_BAD_OFFSETS


def test_persist_few_items_and_one_electron(pb):
    """Fewer items than resident warps (every warp at most one item), one
    electron, and a batch of non-finite positions only."""
    grid = (12, 10, 14)
    lat = np.diag([9.0, 8.0, 11.0])
    tab = bi.smooth_random_table(grid, 128, seed=63)
    t = pb.BlipTable(grid, lat, tab)
    for pos in (bi.uniform_positions(lat, 37, seed=63), bi.uniform_positions(lat, 1, seed=64)):
        t.set_kernel(1, 1, 8, 0)
        ref = gpu_eval(t, pos)
        t.set_kernel(11, 1, 4, 0)
        out = gpu_eval(t, pos)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b)
        compare(grid, lat, tab, pos, out)
    assert t.status() == 0
    v, g, lp = gpu_eval(t, np.full((5, 3), np.nan))
    assert np.isnan(v).all() and np.isnan(g).all() and np.isnan(lp).all()
    assert t.status() & pb.STATUS_NONFINITE_POS


def test_persist_in_a_cuda_graph(pb):
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=65)
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(11, 1, 4, 1)
    pos_a = bi.uniform_positions(lat, 6000, seed=65)
    pos_b = bi.uniform_positions(lat, 6000, seed=66)
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


def test_persist_full_size_headline(pb):
    """The TiO2-shaped headline batch (72 x 72 x 48 grid, 768 orbitals,
    1,536 electrons): bitwise equal to variant 9, sampled electrons against
    the oracle."""
    w, tab = cached_table("tio2")
    pos, _ = w.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab)
    dpos = torch.from_numpy(pos).cuda()
    t.set_kernel(9, 1, 4, 0)
    ref = t.eval(dpos)
    t.set_kernel(11, 1, 4, 0)
    out = t.eval(dpos)
    torch.cuda.synchronize()
    for r, o in zip(ref, out):
        assert torch.equal(r, o)
    assert t.status() == 0
    idx = np.unique(np.concatenate([[0, len(pos) - 1], np.random.default_rng(7).integers(0, len(pos), 40)]))
    compare(w.grid, w.lattice, tab, pos[idx], [o[idx].cpu().numpy() for o in out])


def test_persist_rejections(pb):
    grid = (6, 6, 6)
    lat = np.diag([5.0, 5.0, 5.0])
    tab = bi.smooth_random_table(grid, 64, seed=67)
    t16 = pb.BlipTable(grid, lat, tab, storage=pb.BF16)
    with pytest.raises(Exception):
        t16.set_kernel(11, 1, 4, 0)                    # FP32 tables only
    t = pb.BlipTable(grid, lat, tab)
    for cfg in ((11, 2, 4, 0), (11, 1, 0, 0), (11, 1, 17, 0), (11, 1, 4, 3)):
        with pytest.raises(Exception):
            t.set_kernel(*cfg)
    ctab = bi.smooth_random_table(grid, 8, seed=68, is_complex=True)
    tc = pb.BlipTable(grid, lat, ctab, storage=pb.C64)
    tc.set_kernel(11, 1, 4, 0)
    tc.set_kpoints(np.zeros((1, 3)), [0, 8])           # no Bloch epilogue: choice reset
    with pytest.raises(Exception):
        tc.set_kernel(11, 1, 4, 0)


def test_probe_gather_reads_the_evaluation_rows(pb):
    """blip_probe_gather folds (XOR) the 16 bytes each lane loads from the 64
    stencil rows of its (electron, chunk) item.  With output stores on, the
    folded word lands in the item's value slice, so it can be checked exactly
    against the same fold over the FP32-rounded coefficients of the 64 sites
    around each position: the probe reads the rows an evaluation reads.
    Without stores the outputs are left untouched."""
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    L = 700
    tab = bi.smooth_random_table(grid, L, seed=69)
    pos = bi.uniform_positions(lat, 3000, seed=69)
    t = pb.BlipTable(grid, lat, tab)
    dpos = torch.from_numpy(pos).cuda()
    sentinel = 0x7F7F7F7F
    out = t.alloc_outputs(len(pos))
    for o in out:
        o.view(torch.int32).fill_(sentinel)
    t.probe_gather(dpos, out=out, store=False)
    torch.cuda.synchronize()
    assert all(bool((o.view(torch.int32) == sentinel).all()) for o in out)
    t.probe_gather(dpos, out=out, store=True)
    torch.cuda.synchronize()
    got = out[0].view(torch.int32).cpu().numpy().view(np.uint32)

    n = np.array(grid)
    u = np.linalg.solve(lat.T, pos.T).T               # r = u @ lat
    g = (u - np.floor(u)) * n
    base = np.floor(g).astype(np.int64) % n
    words = tab.astype(np.float32).view(np.uint32)   # [n1][n2][n3][L]
    ref = np.zeros((len(pos), L), dtype=np.uint32)
    for kx in range(4):
        for ky in range(4):
            for kz in range(4):
                m = (base + np.array([kx, ky, kz]) - 1) % n
                ref ^= words[m[:, 0], m[:, 1], m[:, 2]]
    lanes = ref.reshape(len(pos), -1, 4)             # 4 components per lane
    fold = np.bitwise_xor.reduce(lanes, axis=2)
    assert np.array_equal(got.reshape(len(pos), -1, 4), np.repeat(fold[:, :, None], 4, axis=2))
    assert t.status() == 0
    t16 = pb.BlipTable(grid, lat, tab, storage=pb.BF16)
    with pytest.raises(Exception):
        t16.probe_gather(dpos, out=t16.alloc_outputs(len(pos)))
