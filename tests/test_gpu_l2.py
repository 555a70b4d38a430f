"""L2 residency of a small table (blip_set_l2_residency) with k-points.

A primitive-cell table with 64 k-points (15 MB, complex64) stands in for the
4 x 4 x 4 supercell table it replaces (blip_set_kpoints: psi = exp(i k.r) u).
With the table's L2 window on, evaluations on a caller's stream must give
bitwise the same outputs as without it, those outputs must match the FP64
Bloch oracle on sampled electrons, and the window must turn off cleanly.
"""
import numpy as np
import pytest

import blip_inputs as bi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TAU32 = 8e-6


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _bloch_bound(grid, lat, tab, pos, kfrac, koffs):
    """Per-output bound of a complex64 Bloch evaluation: the FP32 bound of u
    and its derivatives through the product rule, plus 2e-6 relative for the
    FP32 phase (as in the k-point parity tests)."""
    u, gu, lu, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    C = mag[:, :, 0::2] + mag[:, :, 1::2]
    kcart = 2 * np.pi * np.asarray(kfrac) @ np.linalg.inv(np.asarray(lat).T)
    L = tab.shape[-1]
    kq = np.zeros((L, 3))
    for q in range(len(koffs) - 1):
        kq[koffs[q]:koffs[q + 1]] = kcart[q]
    ak = np.abs(kq).T[None]
    au, ag, al = np.abs(u), np.abs(gu), np.abs(lu)
    ph = 2e-6
    k2 = (kq ** 2).sum(1)[None]
    bv = TAU32 * C[:, 0] + ph * au
    bg = TAU32 * (C[:, 1:4] + ak * C[:, None, 0]) + ph * (ag + ak * au[:, None])
    bl = TAU32 * (C[:, 4] + 2 * (ak * C[:, 1:4]).sum(1) + k2 * C[:, 0]) \
        + ph * (al + 2 * (ak * ag).sum(1) + k2 * au)
    return bv, bg, bl


def test_l2_window_keeps_outputs_and_turns_off(pb):
    w = bi.workload("tio2_kpoints", batch=64)
    tab = w.table()
    pos, offs = w.positions()
    kf, ko = w.extra["kfrac"], w.extra["koffs"]
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=pb.C64)
    t.set_kpoints(kf, ko)
    s = torch.cuda.Stream()
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    with torch.cuda.stream(s):
        ref = t.eval(dpos, doffs, stream=s)
        t.set_l2_residency(1.0)
        on = [t.eval(dpos, doffs, stream=s) for _ in range(2)]
        t.set_l2_residency(0.0)
        off = t.eval(dpos, doffs, stream=s)
    s.synchronize()
    for run in on + [off]:
        for a, b in zip(ref, run):
            assert torch.equal(a, b)
    assert t.status() == 0
    # sampled electrons against the FP64 Bloch oracle
    idx = np.unique(np.concatenate([[0, len(pos) - 1],
                                    np.random.default_rng(71).integers(0, len(pos), 24)]))
    v = pb.BlipTable.as_complex(on[0][0])[idx].cpu().numpy().astype(np.complex128)
    g = pb.BlipTable.as_complex(on[0][1])[idx].cpu().numpy().astype(np.complex128)
    lp = pb.BlipTable.as_complex(on[0][2])[idx].cpu().numpy().astype(np.complex128)
    rv, rg, rl = oracle.bloch.eval_bloch(w.grid, w.lattice, tab, pos[idx], kf, ko)
    bv, bg, bl = _bloch_bound(w.grid, w.lattice, tab, pos[idx], kf, ko)
    assert (np.abs(v - rv) <= bv + 1e-30).all()
    assert (np.abs(g - rg) <= bg + 1e-30).all()
    assert (np.abs(lp - rl) <= bl + 1e-30).all()
    # bad arguments, and the window turns on and off again
    L = pb.lib()
    assert L.blip_set_l2_residency(t.handle, -0.5) == -1
    assert L.blip_set_l2_residency(t.handle, 1.5) == -1
    assert L.blip_set_l2_residency(None, 0.5) == -1
    t.set_l2_residency(0.5)
    t.set_l2_residency(0.0)
    t.close()


def test_l2_read_probe(pb):
    """The measurement aid runs on a caller's stream and rejects bad sizes."""
    buf = torch.ones(1 << 20, device="cuda")
    s = torch.cuda.Stream()
    pb.probe_l2_read(buf, 3, stream=s)
    s.synchronize()
    L = pb.lib()
    assert L.blip_probe_l2_read(None, 64, 1, None) == -1
    assert L.blip_probe_l2_read(buf.data_ptr(), 24, 1, None) == -1
    assert L.blip_probe_l2_read(buf.data_ptr(), 64, 0, None) == -1
    assert L.blip_probe_l2_read(buf.data_ptr() + 4, 64, 1, None) == -1
