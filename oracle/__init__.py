"""FP64 CPU oracle for the periodic cubic-blip orbital evaluation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the
CUDA library (``paper_1204_1121_gb300``) and never imports it.

Contents:

* ``eval_stencil`` - Oracle A, the 64-term stencil sum of Eq. 11.12.24.1 with
  the tensor-product basis of Eq. 11.12.24.2 and the stencil selection of
  Eq. 7, in plain C (``blip_oracle.c``), FP64, threaded over electrons.
* ``B, dB, d2B`` - the piecewise cubic B-spline from the same C file.
* ``brute`` - Oracle B, a numpy sum over every grid site and periodic image in
  Cartesian coordinates (tiny grids only).
* ``kinetic`` - the Slater-only local kinetic energy built from orbital
  values and Laplacians (the energy-error probe of Sec. V.B).
* ``bloch`` - k-point orbitals exp(i k.r) u(r) from a periodic table of u.
* ``sherman_morrison`` - the O(N^2) inverse update after an accepted move.

Pins: every function here is checked in ``tests/test_oracle_pins.py`` against
closed forms, invariants, exact polynomial and plane-wave reproduction, finite
differences and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blip_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``blip_oracle.c`` into ``liboracle.so`` (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c99",
                               "-D_POSIX_C_SOURCE=200809L", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    """Load a compiled oracle library from ``path`` and declare its symbols."""
    L = ctypes.CDLL(path)
    for f in ("oracle_B", "oracle_dB", "oracle_d2B"):
        getattr(L, f).restype = ctypes.c_double
        getattr(L, f).argtypes = [ctypes.c_double]
    P = ctypes.c_void_p
    L.oracle_eval.restype = ctypes.c_int
    L.oracle_eval.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_long,
                              P, P, P, P, ctypes.c_int]
    L.oracle_geometry.restype = ctypes.c_int
    L.oracle_geometry.argtypes = [P, P, P, P, P]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(_LIB)
    return _lib


def B(x: float) -> float:
    return lib().oracle_B(float(x))


def dB(x: float) -> float:
    return lib().oracle_dB(float(x))


def d2B(x: float) -> float:
    return lib().oracle_d2B(float(x))


def geometry(grid, lattice):
    """(A^-1, J = diag(n) A^-1, M = J J^T) as 3x3 arrays, from the C oracle."""
    g = np.ascontiguousarray(grid, dtype=np.int32)
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    out = [np.zeros(9) for _ in range(3)]
    rc = lib().oracle_geometry(g.ctypes.data, lat.ctypes.data, *(o.ctypes.data for o in out))
    if rc != 0:
        raise ValueError("singular cell")
    return tuple(o.reshape(3, 3) for o in out)


def _real_view(coeffs):
    c = np.asarray(coeffs)
    if np.iscomplexobj(c):
        c = np.ascontiguousarray(c, dtype=np.complex128)
        return c.view(np.float64), True
    return np.ascontiguousarray(c, dtype=np.float64), False


def eval_stencil(grid, lattice, coeffs, pos, norm: int = 0, absmag: bool = False,
                 threads: int | None = None, _lib=None):
    """Oracle A.  ``coeffs`` is ``[n1][n2][n3][L]`` (real or complex).

    Returns ``values [E][L]``, ``grads [E][3][L]``, ``laps [E][L]`` (complex
    when the table is complex) and, with ``absmag``, ``mag [E][5][L]`` =
    sum_s |W_k(s)| |a_ls| per output k (for a complex table, per real and
    imaginary part: shape ``[E][5][2L]`` interleaved).
    """
    grid = tuple(int(g) for g in grid)
    c, cplx = _real_view(coeffs)
    Lr = c.shape[-1]
    if c.shape[:3] != grid:
        raise ValueError("table shape does not match grid")
    p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    E = p.shape[0]
    vals = np.zeros((E, Lr))
    grads = np.zeros((E, 3, Lr))
    laps = np.zeros((E, Lr))
    mag = np.zeros((E, 5, Lr)) if absmag else None
    g = np.array(grid, dtype=np.int32)
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    nt = threads if threads else (os.cpu_count() or 1)
    rc = (_lib or lib()).oracle_eval(g.ctypes.data, lat.ctypes.data, Lr, int(norm), c.ctypes.data,
                           p.ctypes.data, E, vals.ctypes.data, grads.ctypes.data,
                           laps.ctypes.data, mag.ctypes.data if absmag else None, int(nt))
    if rc != 0:
        raise RuntimeError(f"oracle_eval failed: {rc}")
    if cplx:
        vals = vals.view(np.complex128)
        grads = grads.view(np.complex128)
        laps = laps.view(np.complex128)
    return (vals, grads, laps, mag) if absmag else (vals, grads, laps)


from . import bloch, brute, kinetic, sherman_morrison  # noqa: E402,F401
