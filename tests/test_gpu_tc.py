"""Tensor-core kernel (variant 12) against the FP64 oracle.

The kernel evaluates Eq. 11.12.24.1 for dense sorted batches as matrix
products over the union rows of parts of up to 25 electrons (tcgen05, FP32
accumulation in tensor memory).  Its rounding differs from the CUDA-core
kernels, so its bound is derived for its own arithmetic:

* FP32 tables enter as two FP16 planes of v = a / s_l (s_l the power of two
  at or above max |a_l|): |v - hi - lo| <= 2^-23 |v|; the FP32 weights
  (about 13 * 2^-24 |W| from their formula) as two FP16 parts,
  |W - hi - lo| <= 2^-22 |W|; the product left out (lo.lo) is below
  2^-22 |W v|.  Accumulation: 24 products of 16 terms per output (16 into
  the hi-part accumulator: 8 K steps x 2 coefficient planes; 8 into the
  lo-part one; the two added once); with at most 2 units in the last place
  of the running sum per product, 24 * 2^-22.  Together about 30 * 2^-22 =
  7.1e-6; the
  bound takes TAU_TC = 1.6e-5.  Parts below the FP16 normal range (a tiny
  coefficient or weight) are rounded to 2^-25 absolute: a floor of
  2^-25 s_l (sum_s |W_s| + 64) per output.
* 16-bit tables enter as stored; the weights as two parts of the table's
  type, |W - hi - lo| <= 2^-17 |W| (BF16) or 2^-22 |W| (FP16); 16 products
  per output (8 per part).  The same TAU_TC covers this beside the
  coefficient rounding u
  of the storage; FP16 has the same subnormal floor with s_l its scale.
"""
import numpy as np
import pytest

import blip_inputs as bi
import oracle
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU_TC = 1.6e-5
U_Q = {0: 0.0, 1: 2.0 ** -8, 2: 2.0 ** -11}


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _scales(tab):
    return np.abs(tab.reshape(-1, tab.shape[-1])).max(0)


def _check(grid, lat, tab, pos, out, storage, idx=None):
    """Every output of electrons idx (all if None) within the bound."""
    idx = np.arange(len(pos)) if idx is None else np.asarray(idx)
    p = pos[idx]
    v, g, lp, mag = oracle.eval_stencil(grid, lat, tab, p, absmag=True)
    tau = TAU_TC + U_Q[storage]
    floor = 0.0
    if storage in (0, 2):
        # FP16 scale: max |a_l|; the FP32 planes' power of two is below twice it
        s = (2.0 if storage == 0 else 1.0) * _scales(tab)[None, :]
        ones = np.ones(tuple(grid) + (1,))
        _, _, _, sw = oracle.eval_stencil(grid, lat, ones, p, absmag=True)
        floor = [2.0 ** -25 * (64.0 + sw[:, 0:1, 0]) * s,
                 2.0 ** -25 * (64.0 + sw[:, 1:4, 0][:, :, None]) * s[:, None, :],
                 2.0 ** -25 * (64.0 + sw[:, 4:5, 0]) * s]
    refs = [v, g, lp]
    mags = [mag[:, 0], mag[:, 1:4], mag[:, 4]]
    worst = 0.0
    for k in range(3):
        got = np.asarray(out[k])[idx].astype(np.float64)
        bound = tau * mags[k] + (floor[k] if storage in (0, 2) else 0.0) + 1e-30
        r = np.abs(got - refs[k]) / bound
        worst = max(worst, float(np.nanmax(r)))
        assert (r <= 1.0).all(), (k, float(np.nanmax(r)))
    return worst


def _dense_positions(lat, grid, n_per_cell, seed):
    """n_per_cell uniform electrons in every cell on average, three cells
    crowded with 60, 26 and 25 electrons (parts split inside one cell), far
    and negative images, and one NaN position."""
    rng = np.random.default_rng(seed)
    n = np.array(grid, dtype=np.float64)
    ncell = int(np.prod(grid))
    u = rng.uniform(0, 1, size=(n_per_cell * ncell, 3))
    crowd = []
    for cell, cnt in (((1, 2, 3), 60), ((5, 0, 11), 26), ((0, 9, 13), 25)):
        crowd.append((np.array(cell) + rng.uniform(0.05, 0.95, size=(cnt, 3))) / n)
    u = np.concatenate([u] + crowd)
    u[:40] += rng.integers(-5, 6, size=(40, 3))           # periodic images
    pos = u @ lat
    pos = np.concatenate([pos, [[np.nan, 1.0, 2.0]]])
    return pos[rng.permutation(len(pos))]


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_tc_dense_ragged_against_oracle(pb, storage):
    grid = (12, 10, 14)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=51, sigma=2.0)   # 3 M tiles, the last ragged
    pos = _dense_positions(lat, grid, 3, 52)
    t = pb.BlipTable(grid, lat, tab, storage=storage)
    t.set_kernel(12, 1, 1, 1)
    dpos = torch.from_numpy(pos).cuda()
    out = t.eval(dpos)
    torch.cuda.synchronize()
    res = [o.cpu().numpy() for o in out]
    bad = np.isnan(pos).any(1)
    assert np.isnan(res[0][bad]).all() and np.isnan(res[2][bad]).all()
    worst = _check(grid, lat, tab, pos, res, storage, np.flatnonzero(~bad))
    print(f"\nstorage {storage}: worst error / bound {worst:.3g}")
    assert t.status() == pb.STATUS_NONFINITE_POS
    # repeated runs are bitwise identical
    again = t.eval(dpos)
    torch.cuda.synchronize()
    for a, b in zip(out, again):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    t.status()


@pytest.mark.parametrize("storage", [0, 1])
def test_tc_values_only_and_walker_offsets(pb, storage):
    """Values-only mode (N = electrons of the part) and a ragged walker
    batch, against the oracle."""
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 130, seed=53)
    pos, offs = bi.walker_positions(lat, 9, 500, [500, 1, 333, 0, 250, 499, 17, 400, 500], seed=54)
    t = pb.BlipTable(grid, lat, tab, storage=storage)
    t.set_kernel(12, 1, 1, 1)
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    v, _, _ = t.eval(dpos, doffs, values_only=True)
    full = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    _check(grid, lat, tab, pos, [o.cpu().numpy() for o in full], storage)
    rv, _, _, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    err = np.abs(v.cpu().numpy().astype(np.float64) - rv)
    assert (err <= (TAU_TC + U_Q[storage]) * mag[:, 0] + 1e-30).all()
    assert t.status() == 0


def test_tc_agrees_with_staged_kernel_on_tio2_batch(pb):
    """256 walkers x 1,536 electrons on the TiO2-shaped table (1.6 electrons
    per cell): the tensor-core kernel against the staged CUDA-core kernel and
    sampled electrons against the oracle."""
    w = bi.workload("tio2")
    tab = w.table()
    wb = bi.workload("tio2_batch", batch=1536)
    pos, offs = wb.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=pb.F32)
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    t.set_kernel(8, 4, 12, 1)
    ref = t.eval(dpos, doffs)
    t.set_kernel(12, 1, 1, 1)
    out = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(55)
    idx = np.unique(np.concatenate([[0, len(pos) - 1], rng.integers(0, len(pos), 48)]))
    res = [o[idx].cpu().numpy() for o in out]
    _check(w.grid, w.lattice, tab, pos[idx], res, 0)
    # the two kernels differ by at most the sum of their bounds
    d = (out[0] - ref[0]).abs().max().item()
    assert d < 1e-3, d
    assert t.status() == 0


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_tc_precision_workload_full_size(pb, storage):
    """The full precision workload (1,024 walkers x 1,536 electrons, 6.3
    electrons per cell) on the tensor cores: sampled electrons against the
    oracle, and the Slater-only local kinetic energy of two walkers; FP32
    tables meet the paper's ~1e-3 hartree per primitive cell."""
    import json
    w = bi.workload("tio2")
    tab = w.table()
    wp = bi.workload("tio2_precision")
    pos, offs = wp.positions()
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=storage)
    t.set_kernel(12, 1, 1, 1)
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    v, g, lp = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(56)
    idx = np.unique(np.concatenate([[0, len(pos) - 1], rng.integers(0, len(pos), 40)]))
    worst = _check(w.grid, w.lattice, tab, pos[idx],
                   [v[idx].cpu().numpy(), g[idx].cpu().numpy(), lp[idx].cpu().numpy()], storage)
    blocks = [(0, 768), (768, 1536)]
    errs = []
    for wk in range(2):
        p0 = pos[1536 * wk:1536 * (wk + 1)]
        rv, _, rl = oracle.eval_stencil(w.grid, w.lattice, tab, p0)
        T_ref, _ = oracle.kinetic.local_kinetic(rv, rl, blocks)
        T_gpu, _ = oracle.kinetic.local_kinetic(v[1536 * wk:1536 * (wk + 1)].cpu().numpy(),
                                                lp[1536 * wk:1536 * (wk + 1)].cpu().numpy(), blocks)
        errs.append(abs(T_gpu - T_ref) / 64.0)
    print("\n" + json.dumps({"storage": storage, "worst_err_over_bound": worst,
                             "kinetic_err_per_cell": errs}))
    if storage == 0:
        assert max(errs) <= 1e-3
    assert t.status() == 0
