"""The C ABI library loads, exports every symbol include/blip.h declares, and
rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np

import paper_1204_1121_gb300 as pb

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "blip.h")


def declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blip_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared() == sorted(pb.EXPORTED)


def test_library_exports_every_declared_symbol():
    L = pb.lib()
    for name in declared():
        assert hasattr(L, name), name


def test_strerror():
    L = pb.lib()
    assert L.blip_strerror(0) == b"ok"
    assert L.blip_strerror(-2) == b"singular lattice"
    assert L.blip_strerror(-99) == b"unknown error"


def _create(grid, lattice, n_orb=2, storage=0, norm=0, coeffs=True):
    L = pb.lib()
    g = (ctypes.c_int * 3)(*grid)
    lat = (ctypes.c_double * 9)(*np.asarray(lattice, dtype=np.float64).reshape(-1))
    buf = np.zeros(max(1, int(np.prod(grid))) * max(n_orb, 1))
    h = ctypes.c_void_p()
    rc = L.blip_create(g, lat, n_orb, storage, norm,
                       ctypes.c_void_p(buf.ctypes.data) if coeffs else None, 1, 0,
                       ctypes.byref(h))
    return rc, h


def test_create_rejects_bad_arguments_on_host():
    eye = np.eye(3) * 5
    assert _create((3, 4, 4), eye)[0] == -1          # grid < 4
    assert _create((4, 4, 4), eye, n_orb=0)[0] == -1
    assert _create((4, 4, 4), eye, coeffs=False)[0] == -1
    assert _create((4, 4, 4), eye, storage=9)[0] == -5
    assert _create((4, 4, 4), eye, norm=3)[0] == -1
    sing = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 1.0]])
    assert _create((4, 4, 4), sing)[0] == -2
    bad = eye.copy()
    bad[1, 1] = np.nan
    assert _create((4, 4, 4), bad)[0] == -1
    rc, h = _create((4, 4, 4), eye)
    assert rc in (0, -6)                            # -6: no sm_103 device here
    if rc == 0:
        pb.lib().blip_destroy(h)


def test_null_handles_rejected():
    L = pb.lib()
    s = ctypes.c_int()
    assert L.blip_status(None, ctypes.byref(s)) == -1
    assert L.blip_eval(None, None, 0, None, 0, None, None, None, None) == -1
    assert L.blip_destroy(None) == 0
    assert L.blip_graph_launch(None, None) == -1
    assert L.blip_set_kernel(None, 1, 1, 8, 0) == -1
