"""blip_create's out-of-memory path, through the test-only allocation hook.

The hook (blip_test_fail_alloc) makes one of the library's device
allocations fail with cudaErrorMemoryAllocation without calling cudaMalloc,
so the failure is made on the host and the GPU is never short of memory.
For every allocation blip_create makes, the call must return BLIP_ERR_OOM,
leave the handle NULL and give back every byte it had taken; a create
afterwards must succeed and evaluate correctly.
"""
import ctypes

import numpy as np
import pytest

import blip_inputs as bi
import oracle
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _create(pb, grid, lat, tab, storage):
    g = (ctypes.c_int * 3)(*grid)
    la = (ctypes.c_double * 9)(*np.asarray(lat, dtype=np.float64).reshape(-1))
    h = ctypes.c_void_p(0x1234)                       # overwritten on every path
    rc = pb.lib().blip_create(g, la, tab.shape[-1], storage, 0, ctypes.c_void_p(tab.ctypes.data),
                              1, 0, ctypes.byref(h))
    return rc, h


# allocations blip_create makes from a host source: status word, FP32 table,
# host staging slab; quantised kinds add the scales, the max|a| bits and the
# 16-bit table
@pytest.mark.parametrize("storage,points", [(0, 3), (1, 6), (2, 6)])
def test_create_returns_oom_and_frees_everything(pb, storage, points):
    grid = (40, 36, 32)
    lat = pins.triclinic_lattice()
    tab = np.ascontiguousarray(bi.smooth_random_table(grid, 96, seed=9))   # 35 MB FP64
    L = pb.lib()
    rc, h = _create(pb, grid, lat, tab, storage)      # loads the library's kernels
    assert rc == 0
    L.blip_destroy(h)
    torch.cuda.synchronize()
    for k in range(points):
        free0 = torch.cuda.mem_get_info()[0]
        L.blip_test_fail_alloc(k)
        rc, h = _create(pb, grid, lat, tab, storage)
        L.blip_test_fail_alloc(-1)
        assert rc == -3, (k, rc)
        assert not h.value, k
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert abs(free1 - free0) < (2 << 20), (k, free0 - free1)
    # past the last allocation the hook is never reached: the create succeeds
    L.blip_test_fail_alloc(points)
    rc, h = _create(pb, grid, lat, tab, storage)
    L.blip_test_fail_alloc(-1)
    assert rc == 0
    L.blip_destroy(h)
    # and a plain create afterwards evaluates correctly
    t = pb.BlipTable(grid, lat, tab, storage=storage)
    pos = bi.uniform_positions(lat, 200, seed=10)
    v, g, lp = t.eval(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    tau = 8e-6 + {0: 0.0, 1: 2.0 ** -8, 2: 2.0 ** -11}[storage]
    sub = 0.0 if storage != 2 else 2.0 ** -25 * np.abs(tab).max() * 2.0
    assert (np.abs(v.cpu().numpy() - rv) <= tau * mag[:, 0] + sub).all()
    assert t.status() == 0
