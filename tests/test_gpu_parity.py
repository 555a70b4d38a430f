"""CUDA path (through the C ABI) against the FP64 oracle.

Every comparison is element by element under the bound documented in
``gpu_util`` (FP32: 8e-6 x sum_s |W||a|; quantised tables add the storage
unit roundoff).  Small cases compare every output; the full-size TiO2-shaped
workloads compare a seeded sample of electrons in the launch configuration the
benchmark uses.
"""
import numpy as np
import pytest

import blip_inputs as bi
import oracle
import pins
from gpu_util import TAU32, cached_table, compare, gpu_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _edge_positions(lat, grid, rng, n=96):
    n_ = np.array(grid, dtype=np.float64)
    u = [rng.uniform(-2.0, 3.0, size=(n, 3)),
         rng.uniform(0, 1, size=(8, 3)) + rng.integers(-50, 50, size=(8, 3)),
         (rng.integers(0, 64, size=(8, 3)) % n_) / n_,           # exact nodes
         np.full((1, 3), 1.0 - 2.0 ** -53), np.full((1, 3), -2.0 ** -60),
         np.array([[0.0, 0.5, 1.0], [1e6, -1e6, 3e5]])]
    return np.concatenate(u) @ lat


def _scales(tab, pairs):
    a = np.abs(tab.reshape(-1, tab.shape[-1] if not np.iscomplexobj(tab) else tab.shape[-1]))
    if np.iscomplexobj(tab):
        r = np.abs(tab.view(np.float64).reshape(-1, 2 * tab.shape[-1])).max(0)
        r = np.maximum(r[0::2], r[1::2]).repeat(2)
        return np.where(r > 0, r, 1.0)
    s = a.max(0)
    return np.where(s > 0, s, 1.0)


# ---------------------------------------------------------------------------
# small cases: every output
# ---------------------------------------------------------------------------

def test_cubic16_fp32_all_outputs(pb):
    w, tab = cached_table("cubic16")
    pos, _ = w.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=pb.F32)
    out = gpu_eval(t, pos)
    st = compare(w.grid, w.lattice, tab, pos, out)
    assert st["value"]["max_bound_ratio"] <= 1.0
    assert t.status() == 0


@pytest.mark.parametrize("L", [1, 5, 37, 128, 300, 769])
def test_triclinic_ragged_orbitals_and_edge_positions(pb, L):
    rng = np.random.default_rng(L)
    grid = (9, 7, 11)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, L, seed=L, sigma=2.0)
    pos = _edge_positions(lat, grid, rng)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    compare(grid, lat, tab, pos, gpu_eval(t, pos))


@pytest.mark.parametrize("grid", [(4, 4, 4), (5, 4, 7), (4, 9, 4)])
def test_tiny_grids_against_bruteforce(pb, grid):
    rng = np.random.default_rng(sum(grid))
    lat = pins.triclinic_lattice()
    tab = rng.normal(size=grid + (6,))
    pos = _edge_positions(lat, grid, rng, n=24)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    v, g, lp = gpu_eval(t, pos)
    vb, gb, lb = oracle.brute.eval_brute(grid, lat, tab, pos)
    _, _, _, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    assert (np.abs(v - vb) <= TAU32 * mag[:, 0] + 1e-12).all()
    assert (np.abs(g - gb) <= TAU32 * mag[:, 1:4] + 1e-11).all()
    assert (np.abs(lp - lb) <= TAU32 * mag[:, 4] + 1e-10).all()


def test_kernel_configs_bitwise_identical(pb):
    w, tab = cached_table("cubic16")
    rng = np.random.default_rng(11)
    grid = (8, 9, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 700, seed=5)
    pos = _edge_positions(lat, grid, rng)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    ref = gpu_eval(t, pos)
    cfgs = [(v, c, w, s) for v in (1, 3, 4, 6, 7) for c in (1, 2, 3) for w in (1, 4, 16) for s in (0, 1)]
    cfgs += [(5, g, w, 1) for g in (2, 4) for w in (1, 4, 8)]
    cfgs += [(2, tw, st, s) for tw in (1, 2, 4, 6, 8) for st in (2, 3, 8) for s in (0, 1)]
    cfgs += [(8, tz, cw, 1) for tz in (2, 4) for cw in (12, 16)]
    cfgs += [(v, c, w, 2) for v in (1, 3, 4) for c in (1, 2, 3) for w in (1, 8)]
    cfgs += [(9, 1, w, s) for w in (1, 4, 16) for s in (0, 1, 2)]
    cfgs += [(11, 1, w, s) for w in (1, 4, 16) for s in (0, 1, 2)]
    for cfg in cfgs:
        t.set_kernel(*cfg)
        out = gpu_eval(t, pos)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b), cfg
    assert t.status() == 0


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_grouped_kernel_on_dense_cells(pb, storage):
    """Many electrons per cell (groups of 1..4 plus remainders), duplicates and
    cell-less positions: the cell-grouped kernel equals the register kernel
    bitwise and the oracle within the bound."""
    rng = np.random.default_rng(23)
    grid = (6, 5, 7)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=23)
    n = np.array(grid, dtype=np.float64)
    cells = rng.integers(0, 5, size=(12, 3))
    counts = [1, 2, 3, 4, 5, 6, 7, 8, 9, 13, 17, 30]
    u = np.concatenate([(c + rng.uniform(0.05, 0.95, size=(k, 3))) / n
                        for c, k in zip(cells, counts)])
    u = np.concatenate([u, u[:5], u[7:9] + 3.0])            # duplicates, far images
    pos = u @ lat
    pos = np.concatenate([pos[:40], [[np.nan, 0, 0], [0, np.inf, 1]], pos[40:]])
    rng.shuffle(pos[42:])
    kind = pb.F32 if storage == "f32" else pb.BF16
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    t.set_kernel(1, 1, 8, 0)
    ref = gpu_eval(t, pos)
    t.status()
    for cfg in [(5, 2, 4, 1), (5, 4, 8, 1), (5, 4, 1, 1), (5, 2, 8, 1), (7, 1, 4, 1), (7, 1, 8, 0),
                (6, 1, 4, 1)]:
        t.set_kernel(*cfg)
        for vo in (False, True):
            out = gpu_eval(t, pos, values_only=vo)
            for a, b in zip(ref, out):
                assert np.array_equal(a, b, equal_nan=True), (cfg, vo)
        assert t.status() & pb.STATUS_NONFINITE_POS
    good = np.isfinite(pos).all(1)
    compare(grid, lat, tab, pos[good], [r[good] for r in ref], storage=kind,
            scales=_scales(tab, False))


@pytest.mark.parametrize("kind", ["bf16", "c64"])
def test_bulk_kernel_matches_register_kernel(pb, kind):
    grid = (7, 9, 8)
    lat = pins.triclinic_lattice()
    cplx = kind == "c64"
    tab = bi.smooth_random_table(grid, 333 if cplx else 1000, seed=12, is_complex=cplx)
    pos = _edge_positions(lat, grid, np.random.default_rng(12))
    t = pb.BlipTable(grid, lat, tab, storage=pb.C64 if cplx else pb.BF16)
    ref = gpu_eval(t, pos)
    for cfg in [(2, 1, 4, 0), (2, 3, 2, 1), (2, 8, 6, 0), (2, 5, 3, 0), (3, 1, 8, 0), (3, 1, 2, 1),
                (4, 1, 4, 1), (5, 2, 4, 1), (5, 4, 8, 1)]:
        t.set_kernel(*cfg)
        for vo in (False, True):
            out = gpu_eval(t, pos, values_only=vo)
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), (cfg, vo)
    assert t.status() == 0


def test_values_only_matches_full(pb):
    grid = (8, 8, 8)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 260, seed=2)
    pos = _edge_positions(lat, grid, np.random.default_rng(2))
    t = pb.BlipTable(grid, lat, tab)
    full = gpu_eval(t, pos)
    vo = gpu_eval(t, pos, values_only=True)
    assert np.array_equal(full[0], vo[0])


def test_alfe_gillan_normalisation(pb):
    grid = (6, 6, 6)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 16, seed=4)
    pos = _edge_positions(lat, grid, np.random.default_rng(4))
    t = pb.BlipTable(grid, lat, tab, norm=pb.NORM_ALFE_GILLAN)
    compare(grid, lat, tab, pos, gpu_eval(t, pos), norm=1)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_quantised_storage_bound(pb, storage):
    grid = (10, 9, 8)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 100, seed=7)
    pos = _edge_positions(lat, grid, np.random.default_rng(7))
    kind = pb.BF16 if storage == "bf16" else pb.F16
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    st = compare(grid, lat, tab, pos, gpu_eval(t, pos), storage=kind, scales=_scales(tab, False))
    # the rounding is really there: the error is well above the FP32 path's
    assert st["value"]["max_rel_to_C"] > 10 * 2.0 ** -24


@pytest.mark.parametrize("storage", ["c64", "bf16pair"])
def test_complex_storage(pb, storage):
    grid = (8, 10, 6)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 70, seed=8, is_complex=True)
    pos = _edge_positions(lat, grid, np.random.default_rng(8))
    kind = pb.C64 if storage == "c64" else pb.BF16PAIR
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    out = gpu_eval(t, pos)
    compare(grid, lat, tab, pos, out, storage=kind, scales=_scales(tab, True))
    v = pb.BlipTable.as_complex(out[0])
    assert v.shape == (len(pos), 70) and v.dtype == np.complex64


def test_plane_wave_table_on_gpu(pb):
    """A closed-form table: the GPU reproduces exp(i theta.g) at nodes."""
    grid = (12, 10, 8)
    lat = pins.triclinic_lattice()
    tab, th, D = pins.plane_wave_table(grid, (2, -3, 1), True)
    n = np.array(grid, dtype=np.float64)
    rng = np.random.default_rng(9)
    mm = np.stack([rng.integers(0, k, 40) for k in grid], 1).astype(np.float64)
    pos = ((mm + n * rng.integers(-3, 4, size=(40, 3))) / n) @ lat
    t = pb.BlipTable(grid, lat, tab, storage=pb.C64)
    v = pb.BlipTable.as_complex(gpu_eval(t, pos)[0])[:, 0]
    assert np.abs(v - np.exp(1j * (mm @ th))).max() < 2e-5


@pytest.mark.parametrize("cfg", [(1, 1, 8, 0), (2, 1, 4, 0), (2, 2, 3, 1)])
def test_nonfinite_and_far_positions_flagged(pb, cfg):
    grid = (6, 6, 6)
    lat = np.diag([6.0, 6.0, 6.0])
    tab = bi.smooth_random_table(grid, 10, seed=1)
    pos = np.array([[0.5, 0.5, 0.5], [np.nan, 0, 0], [1.0, np.inf, 2.0], [1e13, 0, 0]])
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(*cfg)
    v, g, lp = gpu_eval(t, pos)
    assert np.isnan(v[1]).all() and np.isnan(g[2]).all() and np.isnan(lp[1]).all()
    assert np.isfinite(v[0]).all() and np.isfinite(v[3]).all()
    st = t.status()
    assert st & pb.STATUS_NONFINITE_POS and st & pb.STATUS_FAR_POS
    assert t.status() == 0          # cleared by the read


def test_walker_offsets_checked(pb):
    grid = (5, 5, 5)
    lat = np.diag([5.0, 5.0, 5.0])
    tab = bi.smooth_random_table(grid, 4, seed=1)
    pos = np.random.default_rng(1).uniform(0, 5, size=(10, 3))
    t = pb.BlipTable(grid, lat, tab)
    gpu_eval(t, pos, offsets=[0, 3, 3, 10])
    assert t.status() == 0
    gpu_eval(t, pos, offsets=[0, 4, 2, 10])
    assert t.status() & pb.STATUS_BAD_OFFSETS
    gpu_eval(t, pos, offsets=[0, 4, 9])
    assert t.status() & pb.STATUS_BAD_OFFSETS


def test_empty_batch_and_bad_arguments(pb):
    grid = (4, 4, 4)
    t = pb.BlipTable(grid, np.eye(3) * 4, np.ones(grid + (3,)))
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    v, g, lp = t.eval(e)
    assert v.shape == (0, 3)
    L = pb.lib()
    assert L.blip_eval(t.handle, None, 5, None, 0, None, None, None, None) == -1
    assert L.blip_set_kernel(t.handle, 1, 4, 8, 0) == -1
    assert L.blip_set_kernel(t.handle, 1, 1, 0, 0) == -1
    with pytest.raises(pb.BlipError):
        pb.BlipTable((3, 4, 4), np.eye(3), np.ones((3, 4, 4, 1)))


def test_host_entry_point_and_graph_match_device(pb):
    grid = (8, 8, 8)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 64, seed=3)
    pos = _edge_positions(lat, grid, np.random.default_rng(3))
    t = pb.BlipTable(grid, lat, tab)
    ref = gpu_eval(t, pos)
    hv, hg, hl = t.eval_host(pos)
    for a, b in zip(ref, (hv, hg, hl)):
        assert np.array_equal(a, b)
    # page-locked buffers take the zero-copy path
    hp = torch.from_numpy(pos).pin_memory()
    pv = torch.empty(ref[0].shape, dtype=torch.float32).pin_memory()
    pg = torch.empty(ref[1].shape, dtype=torch.float32).pin_memory()
    pl = torch.empty(ref[2].shape, dtype=torch.float32).pin_memory()
    t.eval_host(hp, out=(pv, pg, pl))
    for a, b in zip(ref, (pv, pg, pl)):
        assert np.array_equal(a, b.numpy())
    po = torch.tensor([0, 40, len(pos)], dtype=torch.int32).pin_memory()
    t.eval_host(hp, po, out=(pv, pg, pl))
    assert np.array_equal(ref[0], pv.numpy()) and t.status() == 0
    dpos = torch.from_numpy(pos).cuda()
    for per in (1, 7, len(pos)):
        out = t.alloc_outputs(len(pos))
        gr = t.graph(dpos, out, per)
        gr.launch()
        torch.cuda.synchronize()
        for a, b in zip(ref, out):
            assert np.array_equal(a, b.cpu().numpy()), per
        gr.close()


def test_autotune_keeps_results(pb):
    grid = (8, 8, 8)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 256, seed=6)
    pos = _edge_positions(lat, grid, np.random.default_rng(6))
    t = pb.BlipTable(grid, lat, tab)
    ref = gpu_eval(t, pos)
    dpos = torch.from_numpy(pos).cuda()
    ch = t.autotune(dpos)
    assert 1 <= ch[0] <= 10 and 1 <= ch[1] <= 8 and ch[3] in (0, 1, 2)
    t.set_kernel(*ch)                  # the chosen configuration is a valid one
    out = gpu_eval(t, pos)
    if ch[0] == 10:                    # split stencil: another summation order
        compare(grid, lat, tab, pos, out)
    else:
        for a, b in zip(ref, out):
            assert np.array_equal(a, b)


def test_repeat_runs_bitwise_identical(pb):
    w, tab = cached_table("cubic16")
    pos, _ = w.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab)
    a = gpu_eval(t, pos)
    b = gpu_eval(t, pos)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# full-size TiO2-shaped workloads (sampled electrons)
# ---------------------------------------------------------------------------

def _sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, size=k)]))


def test_tio2_all_at_once_and_one_at_a_time(pb):
    w, tab = cached_table("tio2")
    pos, offs = w.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=pb.F32)
    out = gpu_eval(t, pos, offsets=offs)
    compare(w.grid, w.lattice, tab, pos, out, sample=_sample(len(pos), 96, 1))
    assert t.status() == 0
    # one electron per launch (particle-by-particle order), captured in a graph
    dpos = torch.from_numpy(pos).cuda()
    o1 = t.alloc_outputs(len(pos))
    gr = t.graph(dpos, o1, 1)
    gr.launch()
    torch.cuda.synchronize()
    for a, b in zip(out, o1):
        assert np.array_equal(a, b.cpu().numpy())


@pytest.mark.parametrize("batch", [1, 32, 128, 1536])
def test_tio2_batched_walkers(pb, batch):
    w, tab = cached_table("tio2")
    wb = bi.workload("tio2_batch", batch=batch)
    pos, offs = wb.positions()
    t = pb.BlipTable(wb.grid, wb.lattice, tab, storage=pb.F32)
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    t.autotune(dpos, doffs)
    v, g, lp = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    idx = _sample(len(pos), 64, batch)
    sub = [v[idx].cpu().numpy(), g[idx].cpu().numpy(), lp[idx].cpu().numpy()]
    compare(wb.grid, wb.lattice, tab, pos[idx], sub)
    assert t.status() == 0


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_tio2_precision_storage_and_kinetic_energy(pb, storage):
    """Precision workload shape (1,536 electrons per walker, 768 orbitals):
    bound check on sampled electrons, and the Slater-only local kinetic
    energy of two walkers against the oracle, within the first-order bound
    propagated from the elementwise output bounds (its second-order terms are
    products of the elementwise bounds, below 1e-6 of it here).  FP32 tables
    must also meet the paper's ~1e-3 hartree per primitive cell (64 cells,
    abstract and Sec. V.B); quantised tables are held to their propagated
    bound only (they are for the Metropolis ratio, see the ratio tests)."""
    import json
    from gpu_util import TAU32, U_Q, kinetic_error_bound, sum_abs_weights
    w, tab = cached_table("tio2")
    wp = bi.workload("tio2_precision", n_walkers=4)
    pos, offs = wp.positions()
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16}[storage]
    t = pb.BlipTable(wp.grid, wp.lattice, tab, storage=kind)
    out = gpu_eval(t, pos, offsets=offs)
    scales = _scales(tab, False)
    stats = compare(wp.grid, wp.lattice, tab, pos, out, storage=kind, scales=scales,
                    sample=_sample(len(pos), 48, 3))
    blocks = [(0, 768), (768, 1536)]
    report = {"storage": storage, "outputs": stats, "walkers": []}
    for wk in range(2):
        p0 = pos[1536 * wk:1536 * (wk + 1)]
        rv, _, rl, mag = oracle.eval_stencil(wp.grid, wp.lattice, tab, p0, absmag=True)
        T_ref, conds = oracle.kinetic.local_kinetic(rv, rl, blocks)
        gv = out[0][1536 * wk:1536 * (wk + 1)].astype(np.float64)
        gl = out[2][1536 * wk:1536 * (wk + 1)].astype(np.float64)
        T_gpu, _ = oracle.kinetic.local_kinetic(gv, gl, blocks)
        tau = TAU32 + U_Q.get(kind, 0.0)
        bv, bl = tau * mag[:, 0], tau * mag[:, 4]
        if kind == pb.F16:
            sw = sum_abs_weights(wp.grid, wp.lattice, p0)
            bv = bv + 2.0 ** -25 * sw[:, 0:1] * scales[None, :]
            bl = bl + 2.0 ** -25 * sw[:, 4:5] * scales[None, :]
        bound = kinetic_error_bound(rv, rl, bv, bl, blocks)
        err = abs(T_gpu - T_ref)
        report["walkers"].append({"T_ref": T_ref, "T_gpu": T_gpu, "abs_err": err,
                                  "err_per_cell": err / 64.0, "bound": bound,
                                  "bound_per_cell": bound / 64.0, "cond": max(conds)})
        assert err <= bound, (err, bound)
        if kind == pb.F32:
            assert err / 64.0 <= 1e-3, err / 64.0
    print("\n" + json.dumps(report))


@pytest.mark.parametrize("storage", ["c64", "bf16pair"])
def test_supercell_complex_ragged_full_size(pb, storage):
    """The ragged complex workload at full size: 2 x 2 x 2 supercell grid
    144 x 144 x 96, 1,536 complex orbitals, 512 walkers with 1..512 electrons
    each, in the tuned launch configuration.  Sampled electrons are checked
    against the oracle on the first and last 16 orbitals (the generator makes
    any orbital range on its own, so the oracle reads a host copy of just
    those orbitals)."""
    import gc
    w = bi.workload("tio2_super_complex")
    pos, offs = w.positions()
    kind = pb.C64 if storage == "c64" else pb.BF16PAIR
    dev_tab = w.table(device="cuda")
    t = pb.BlipTable(w.grid, w.lattice, dev_tab, storage=kind)
    del dev_tab
    gc.collect()
    torch.cuda.empty_cache()
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    t.autotune(dpos, doffs)
    v, g, lp = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    assert t.status() == 0
    idx = _sample(len(pos), 24, 44)
    for o0 in (0, w.n_orb - 16):
        sub = bi.spectral_table(w.grid, range(o0, o0 + 16), w.table_seed).numpy()
        cols = slice(2 * o0, 2 * (o0 + 16))
        got = [v[idx][:, cols].cpu().numpy(), g[idx][:, :, cols].cpu().numpy(),
               lp[idx][:, cols].cpu().numpy()]
        scales = None
        if kind == pb.BF16PAIR:
            # the table's per-orbital scale covers the whole orbital: recompute
            # it for these 16 orbitals from the host copy
            r = np.abs(sub.view(np.float64).reshape(-1, 32)).max(0)
            scales = np.maximum(r[0::2], r[1::2]).repeat(2)
        compare(w.grid, w.lattice, sub, pos[idx], got, storage=kind, scales=scales)
    t.close()


@pytest.mark.parametrize("storage", ["c64", "bf16pair"])
@pytest.mark.parametrize("cfg", [(1, 1, 8, 0), (3, 2, 4, 1), (4, 3, 4, 0), (5, 2, 4, 1)])
def test_bloch_kpoints_against_oracle(pb, storage, cfg):
    """psi = exp(i k.r) u with three k-points on a triclinic cell, every
    output against the FP64 Bloch oracle, under the bound propagated through
    the product rule."""
    from gpu_util import U_Q
    rng = np.random.default_rng(41)
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 40, seed=41, is_complex=True, sigma=2.0)
    kfrac = np.array([[0.0, 0.0, 0.0], [0.5, -0.25, 0.125], [0.25, 0.5, -0.5]])
    koffs = [0, 10, 25, 40]
    pos = _edge_positions(lat, grid, rng)
    pos = np.concatenate([pos, pos[:6] + 5 * lat[1] - 2 * lat[2]])      # Bloch theorem images
    kind = pb.C64 if storage == "c64" else pb.BF16PAIR
    if kind == pb.BF16PAIR and cfg[0] in (1, 3, 4):
        cfg = (cfg[0], 1, cfg[2], cfg[3])                # 16-bit storage: one chunk per warp
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    t.set_kpoints(kfrac, koffs)
    t.set_kernel(*cfg)
    v, g, lp = gpu_eval(t, pos)
    vc = v.view(np.complex64).astype(np.complex128)
    gc = g.view(np.complex64).astype(np.complex128)
    lc = lp.view(np.complex64).astype(np.complex128)
    rv, rg, rl = oracle.bloch.eval_bloch(grid, lat, tab, pos, kfrac, koffs)
    _, _, _, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    C = mag[:, :, 0::2] + mag[:, :, 1::2]                # |re| + |im| bound scale per complex output
    kcart = 2 * np.pi * kfrac @ np.linalg.inv(lat.T)
    kq = np.zeros((40, 3))
    for q in range(3):
        kq[koffs[q]:koffs[q + 1]] = kcart[q]
    tau = TAU32 + U_Q.get(kind, 0.0)
    au = np.abs(rv * 0 + oracle.eval_stencil(grid, lat, tab, pos)[0])
    ag = np.abs(oracle.eval_stencil(grid, lat, tab, pos)[1])
    al = np.abs(oracle.eval_stencil(grid, lat, tab, pos)[2])
    ak = np.abs(kq).T[None]                              # [1][3][L]
    ph = 2e-6
    bv = tau * C[:, 0] + ph * au
    bg = tau * (C[:, 1:4] + ak * C[:, None, 0]) + ph * (ag + ak * au[:, None])
    bl = tau * (C[:, 4] + 2 * (ak * C[:, 1:4]).sum(1) + (kq ** 2).sum(1)[None] * C[:, 0]) \
        + ph * (al + 2 * (ak * ag).sum(1) + (kq ** 2).sum(1)[None] * au)
    assert (np.abs(vc - rv) <= bv + 1e-30).all()
    assert (np.abs(gc - rg) <= bg + 1e-30).all()
    assert (np.abs(lc - rl) <= bl + 1e-30).all()
    assert t.status() == 0


def test_bloch_gamma_only_is_bitwise_the_plain_expansion(pb):
    grid = (8, 8, 8)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 24, seed=3, is_complex=True)
    pos = _edge_positions(lat, grid, np.random.default_rng(3))
    t = pb.BlipTable(grid, lat, tab, storage=pb.C64)
    ref = gpu_eval(t, pos)
    t.set_kpoints([[0, 0, 0]], [0, 24])
    out = gpu_eval(t, pos)
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)
    t.set_kpoints(None, None)
    with pytest.raises(pb.BlipError):
        t.set_kpoints([[0, 0, 0]], [0, 23])          # offsets must end at n_orb
    with pytest.raises(pb.BlipError):
        t.set_kpoints([[0, 0, 0]] * 65, [0] * 41 + list(range(24)) + [24])   # at most 64 k-points
    t.set_kpoints([[0.5, 0, 0]], [0, 24])
    with pytest.raises(pb.BlipError):
        t.set_kernel(2, 2, 4, 0)                      # the bulk kernel has no Bloch epilogue
    real = pb.BlipTable(grid, lat, tab.real.copy(), storage=pb.F32)
    with pytest.raises(pb.BlipError):
        real.set_kpoints([[0, 0, 0]], [0, 24])
