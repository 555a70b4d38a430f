"""Split-stencil kernel (variant 10): four warps per (electron, chunk), one
a_1 slab each, partial sums added in a fixed order.  Its summation order
differs from the single-warp kernels, so it is checked against the FP64
oracle under the parity bound (FP32: 8e-6 x sum_s |W||a|; quantised tables
add the storage unit roundoff) rather than bitwise against them; it must be
deterministic run to run."""
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


def _positions(lat, grid, rng, n=300):
    n_ = np.array(grid, dtype=np.float64)
    u = [rng.uniform(-2.0, 3.0, size=(n, 3)),
         (rng.integers(0, 64, size=(8, 3)) % n_) / n_,
         np.full((1, 3), 1.0 - 2.0 ** -53), np.full((1, 3), -2.0 ** -60)]
    pos = np.concatenate(u) @ lat
    return np.concatenate([pos, [[np.nan, 0.0, 0.0], [1e13, 0.0, 0.0]]])


def _scales(tab):
    if np.iscomplexobj(tab):
        r = np.abs(tab.view(np.float64).reshape(-1, 2 * tab.shape[-1])).max(0)
        r = np.maximum(r[0::2], r[1::2]).repeat(2)
    else:
        r = np.abs(tab.reshape(-1, tab.shape[-1])).max(0)
    return np.where(r > 0, r, 1.0)


@pytest.mark.parametrize("grid,n_orb,storage", [((7, 9, 8), 300, "f32"), ((4, 5, 4), 129, "f32"),
                                                ((7, 9, 8), 520, "bf16"), ((6, 5, 7), 300, "f16"),
                                                ((7, 9, 8), 70, "c64")])
def test_split_against_oracle(pb, grid, n_orb, storage):
    rng = np.random.default_rng(grid[0] * 131 + n_orb)
    lat = pins.triclinic_lattice()
    cplx = storage == "c64"
    tab = bi.smooth_random_table(grid, n_orb, seed=71, is_complex=cplx)
    pos = _positions(lat, grid, rng)
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16, "c64": pb.C64}[storage]
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    good = np.isfinite(pos).all(1)
    # the far position (|u| > 2^40, flagged) keeps only a few fractional bits,
    # so its value depends on the last bits of A^-1: checked for the flag only
    cmp = good & (np.abs(pos).max(1) < 1e9)
    for sort in (0, 1):
        t.set_kernel(10, 1, 4, sort)
        out = gpu_eval(t, pos)
        again = gpu_eval(t, pos)
        for a, b in zip(out, again):
            assert np.array_equal(a, b, equal_nan=True)           # deterministic
        assert np.isnan(out[0][~good]).all() and np.isnan(out[2][~good]).all()
        st = t.status()
        assert st & pb.STATUS_NONFINITE_POS and st & pb.STATUS_FAR_POS
        compare(grid, lat, tab, pos[cmp], [o[cmp] for o in out], storage=kind,
                scales=None if kind in (pb.F32, pb.C64) else _scales(tab))
        vo = gpu_eval(t, pos, values_only=True)
        assert np.array_equal(vo[0], out[0], equal_nan=True)
        t.status()


def test_split_walker_offsets_graph_and_host_path(pb):
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 200, seed=72)
    sizes = [5, 0, 17, 1, 40]
    pos, offs = bi.walker_positions(lat, len(sizes), 64, sizes, seed=72)
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(10, 1, 4, 0)
    ref = gpu_eval(t, pos, offsets=offs)
    compare(grid, lat, tab, pos, ref)
    assert t.status() == 0
    # one electron per launch, captured in a CUDA graph
    dpos = torch.from_numpy(pos).cuda()
    out = t.alloc_outputs(len(pos))
    g = t.graph(dpos, out, per_launch=1)
    g.launch()
    torch.cuda.synchronize()
    for r, o in zip(ref, out):
        assert np.array_equal(r, o.cpu().numpy())
    g.close()
    # host buffers
    hv, hg, hl = t.eval_host(pos)
    for r, o in zip(ref, (hv, hg, hl)):
        assert np.array_equal(r, o)
    bad = offs.copy()
    bad[-1] += 1
    gpu_eval(t, pos, offsets=bad)
    assert t.status() & pb.STATUS_BAD_OFFSETS


def test_split_full_size_tio2_sampled(pb):
    """TiO2 shape (72 x 72 x 48, 768 orbitals), 256 walkers x 1 moved
    electron, the small-batch case the kernel is for: sampled electrons
    against the oracle."""
    w, tab = cached_table("tio2")
    wb = bi.workload("tio2_batch", batch=1)
    pos, offs = wb.positions()
    t = pb.BlipTable(wb.grid, wb.lattice, tab)
    t.set_kernel(10, 1, 4, 0)
    out = gpu_eval(t, pos, offsets=offs)
    idx = np.unique(np.concatenate([[0, len(pos) - 1],
                                    np.random.default_rng(9).integers(0, len(pos), 40)]))
    compare(wb.grid, wb.lattice, tab, pos[idx], [o[idx] for o in out])
    assert t.status() == 0


def test_split_rejects_kpoints_and_bad_shapes(pb):
    grid = (6, 6, 6)
    lat = np.diag([6.0, 6.0, 6.0])
    tab = bi.smooth_random_table(grid, 8, seed=73, is_complex=True)
    t = pb.BlipTable(grid, lat, tab, storage=pb.C64)
    for cfg in [(10, 2, 4, 0), (10, 1, 8, 0), (10, 1, 4, 2)]:
        with pytest.raises(Exception):
            t.set_kernel(*cfg)
    t.set_kpoints(np.zeros((1, 3)), [0, 8])
    with pytest.raises(Exception):
        t.set_kernel(10, 1, 4, 0)
