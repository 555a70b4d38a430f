"""The bounded waits of the bulk-copy, staged-tile and tensor-core kernels: a
stalled pipeline (test hook: the consumers, or the tensor-core kernel's MMA
thread, never release the first stage) makes the waits run out after about
two seconds; the kernel returns, reports BLIP_STATUS_TIMEOUT, and the same
context evaluates correctly afterwards.  The tensor-core kernel's MMA thread
waits for its issued products before the tensor memory is freed.  No fault,
trap or unbounded spin is involved."""
import time

import numpy as np
import pytest

import blip_inputs as bi
import pins
from gpu_util import compare, gpu_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


@pytest.mark.parametrize("cfg", [(2, 1, 2, 0), (8, 4, 16, 1), (12, 1, 1, 1)])
def test_stalled_pipeline_times_out_and_context_survives(pb, cfg):
    grid = (8, 8, 8)
    lat = pins.triclinic_lattice()
    # 4 chunks per row: every CTA of either kernel fills its first stage again
    tab = bi.smooth_random_table(grid, 512, seed=61)
    pos = np.random.default_rng(61).uniform(0, 1, size=(64, 3)) @ lat
    t = pb.BlipTable(grid, lat, tab)
    t.set_kernel(*cfg)                       # bulk copy with 2 stages, staged tiles, tensor cores
    t.status()
    pb.lib().blip_test_stall_pipeline(t.handle, 1)
    t0 = time.time()
    gpu_eval(t, pos)
    dt = time.time() - t0
    st = t.status()
    assert st & pb.STATUS_TIMEOUT
    assert 1.0 < dt < 30.0
    pb.lib().blip_test_stall_pipeline(t.handle, 0)
    out = gpu_eval(t, pos)
    assert t.status() == 0
    compare(grid, lat, tab, pos, out)
