"""blip_eval_sorted_noalloc: evaluation that allocates nothing.

Callers that record their Monte Carlo step into a CUDA graph, or that give
all device memory to their own pool and run on a fixed budget, cannot let
the library call cudaMalloc in the middle of a step.  This entry point takes
the spatial sort's scratch from a fixed device buffer inside the library.
These tests call it through the C ABI and check it against blip_eval (the
allocating entry point) within the parity tolerance used everywhere else
(8e-6 x sum_s |W||a| per output), on two calls in a row with different
batches - the buffer keeps the previous call's contents, so the second call
shows the call clears what it must.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import blip_inputs as bi
import oracle
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU32 = 8e-6


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _noalloc(pb, table, pos, offs, out, values_only=False):
    v, g, lp = out
    nw = 0 if offs is None else offs.shape[0] - 1
    return pb.lib().blip_eval_sorted_noalloc(
        table.handle, ctypes.c_void_p(pos.data_ptr()), pos.shape[0],
        ctypes.c_void_p(offs.data_ptr()) if offs is not None else None, nw,
        ctypes.c_void_p(v.data_ptr()),
        None if values_only else ctypes.c_void_p(g.data_ptr()),
        None if values_only else ctypes.c_void_p(lp.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_blip_eval_on_two_calls_in_a_row(pb):
    grid = (20, 18, 16)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=21)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    batches = []
    pos_a, offs_a = bi.walker_positions(lat, 7, 600, [400, 600, 350, 500, 1, 600, 549], seed=31)
    batches.append((pos_a, offs_a))
    pos_b = bi.uniform_positions(lat, 1234, seed=32) - 3.0 * lat[0]
    batches.append((pos_b, None))
    for pos, offs in batches:
        dpos = torch.from_numpy(pos).cuda()
        doffs = None if offs is None else torch.from_numpy(offs).cuda()
        ref = t.eval(dpos, doffs)                      # allocating entry point
        out = t.alloc_outputs(len(pos))
        for o in out:
            o.fill_(float("nan"))
        rc = _noalloc(pb, t, dpos, doffs, out)
        assert rc == 0, pb.lib().blip_strerror(rc)
        torch.cuda.synchronize()
        rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
        bounds = [TAU32 * mag[:, 0], TAU32 * mag[:, 1:4], TAU32 * mag[:, 4]]
        for r, o, b, x in zip(ref, out, bounds, (rv, rg, rl)):
            got = o.cpu().numpy().astype(np.float64)
            # against the allocating entry point, and against the FP64 oracle
            assert (np.abs(got - r.cpu().numpy()) <= b + 1e-30).all()
            assert (np.abs(got - x) <= b + 1e-30).all()
    assert t.status() == 0


def test_noalloc_rejects_a_batch_beyond_the_fixed_scratch(pb):
    grid = (20, 18, 16)
    lat = np.diag([8.0, 7.0, 6.0])
    tab = bi.smooth_random_table(grid, 4, seed=22)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    # 4 (n1 n2 n3 + 1) + 8 n_elec bytes > 8 MiB; the buffers are real and of
    # full size, so nothing could be touched out of bounds even if the check
    # were missing
    n = 1_100_000
    dpos = torch.rand((n, 3), dtype=torch.float64, device="cuda") * 6.0
    v = torch.full((n, 4), 7.0, dtype=torch.float32, device="cuda")
    rc = _noalloc(pb, t, dpos, None, (v, None, None), values_only=True)
    torch.cuda.synchronize()
    assert rc == -7
    assert b"no-allocation" in pb.lib().blip_strerror(rc)
    assert bool((v == 7.0).all())


def test_noalloc_with_the_staged_tile_kernel(pb):
    """The staged-tile kernel through the no-allocation entry point (which
    has no per-electron geometry records, so the kernel wraps the positions
    itself): bitwise equal to blip_eval with the same kernel, on a dense
    batch with a non-finite position."""
    grid = (9, 8, 10)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 200, seed=23)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    pos = bi.uniform_positions(lat, 5000, seed=24)
    pos[17] = [np.nan, 0.0, 0.0]
    dpos = torch.from_numpy(pos).cuda()
    for cfg in [(8, 4, 12, 1), (8, 2, 16, 1)]:
        t.set_kernel(*cfg)
        ref = t.eval(dpos)
        out = t.alloc_outputs(len(pos))
        rc = _noalloc(pb, t, dpos, None, out)
        assert rc == 0, pb.lib().blip_strerror(rc)
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            assert torch.equal(torch.nan_to_num(r, nan=7.0), torch.nan_to_num(o, nan=7.0)), cfg
        assert bool(torch.isnan(out[0][17]).all())
        assert t.status() & pb.STATUS_NONFINITE_POS


@pytest.mark.parametrize("cfg", [(11, 1, 8, 1), (11, 1, 8, 2), (10, 1, 4, 1), (5, 2, 4, 1),
                                 (5, 4, 8, 1), (2, 2, 8, 1), (9, 1, 8, 2), (3, 2, 4, 2),
                                 (6, 1, 8, 1), (7, 1, 8, 1), (12, 1, 1, 1)])
def test_noalloc_with_each_sorted_kernel(pb, cfg):
    """Every kernel the entry point can run on the sorted order - without the
    per-electron geometry records blip_eval's sort makes, so each kernel
    wraps the positions itself - against blip_eval with the same kernel
    choice, on two calls in a row, within the parity tolerance."""
    grid = (20, 18, 16)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, 300, seed=25)
    t = pb.BlipTable(grid, lat, tab, storage=pb.F32)
    t.set_kernel(*cfg)
    for seed, n in ((26, 3000), (27, 1777)):
        pos = bi.uniform_positions(lat, n, seed=seed) + 2.0 * lat[2]
        dpos = torch.from_numpy(pos).cuda()
        ref = t.eval(dpos)
        out = t.alloc_outputs(n)
        for o in out:
            o.fill_(float("nan"))
        rc = _noalloc(pb, t, dpos, None, out)
        assert rc == 0, pb.lib().blip_strerror(rc)
        torch.cuda.synchronize()
        idx = np.arange(0, n, 7)
        rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos[idx], absmag=True)
        bounds = [TAU32 * mag[:, 0], TAU32 * mag[:, 1:4], TAU32 * mag[:, 4]]
        # the oracle bound of the kernel: the tensor-core kernel (variant 12)
        # has its own, 1.6e-5 x sum|W||a| plus the FP16-plane floor
        if cfg[0] == 12:
            s_l = 2.0 * np.abs(tab.reshape(-1, tab.shape[-1])).max(0)
            ones = np.ones(tuple(grid) + (1,))
            _, _, _, sw = oracle.eval_stencil(grid, lat, ones, pos[idx], absmag=True)
            fl = 2.0 ** -25 * (64.0 + sw[:, :, 0])
            obounds = [1.6e-5 * mag[:, 0] + fl[:, 0:1] * s_l,
                       1.6e-5 * mag[:, 1:4] + fl[:, 1:4, None] * s_l[None, None, :],
                       1.6e-5 * mag[:, 4] + fl[:, 4:5] * s_l]
        else:
            obounds = bounds
        for r, o, b, ob, x in zip(ref, out, bounds, obounds, (rv, rg, rl)):
            got = o[idx].cpu().numpy().astype(np.float64)
            assert (np.abs(got - r[idx].cpu().numpy()) <= b + 1e-30).all(), cfg
            assert (np.abs(got - x) <= ob + 1e-30).all(), cfg
            assert not torch.isnan(o).any(), cfg
    assert t.status() == 0
