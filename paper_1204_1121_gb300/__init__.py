"""Python binding of libblip: periodic cubic-blip orbital evaluation on GB300.

Thin ctypes marshalling over the C ABI in ``include/blip.h``: every step of
the evaluation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams only.  There is no CPU fallback: if ``libblip.so`` cannot
be built or loaded, or no sm_103 GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["lib", "BlipTable", "BlipError", "sm_update", "probe_l2_read", "F32", "BF16", "F16", "C64", "BF16PAIR",
           "NORM_BSPLINE", "NORM_ALFE_GILLAN", "STATUS_NONFINITE_POS", "STATUS_FAR_POS",
           "STATUS_BAD_OFFSETS", "STATUS_TIMEOUT", "STATUS_LAYOUT", "EXPORTED"]

F32, BF16, F16, C64, BF16PAIR = 0, 1, 2, 3, 4
NORM_BSPLINE, NORM_ALFE_GILLAN = 0, 1
STATUS_NONFINITE_POS, STATUS_FAR_POS, STATUS_BAD_OFFSETS, STATUS_TIMEOUT = 1, 2, 4, 8
STATUS_LAYOUT = 16
ERRORS = {0: "ok", -1: "invalid argument", -2: "singular lattice", -3: "out of memory",
          -4: "CUDA error", -5: "unsupported storage kind", -6: "no sm_103 CUDA device",
          -7: "batch too large for the fixed no-allocation scratch"}

P = ctypes.c_void_p
I = ctypes.c_int
# name -> (restype, argtypes); the same names as include/blip.h
EXPORTED = {
    "blip_create": (I, [P, P, I, I, I, P, I, I, ctypes.POINTER(P)]),
    "blip_eval": (I, [P, P, I, P, I, P, P, P, P]),
    "blip_eval_host": (I, [P, P, I, P, I, P, P, P]),
    "blip_status": (I, [P, ctypes.POINTER(I)]),
    "blip_destroy": (I, [P]),
    "blip_strerror": (ctypes.c_char_p, [I]),
    "blip_last_cuda_error": (I, []),
    "blip_info": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
    "blip_set_kernel": (I, [P, I, I, I, I]),
    "blip_autotune": (I, [P, P, I, P, I, P, P, P, P, ctypes.POINTER(I)]),
    "blip_graph_create": (I, [P, P, I, P, I, P, P, P, I, ctypes.POINTER(P)]),
    "blip_graph_launch": (I, [P, P]),
    "blip_graph_destroy": (I, [P]),
    "blip_eval_sorted_noalloc": (I, [P, P, I, P, I, P, P, P, P]),
    "blip_eval_ratio": (I, [P, P, I, P, I, P, P, P, I, P]),
    "blip_set_kpoints": (I, [P, I, P, P]),
    "blip_sm_update": (I, [I, I, P, P, P, P, P]),
    "blip_test_stall_pipeline": (I, [P, I]),
    "blip_test_fail_alloc": (I, [I]),
    "blip_set_l2_residency": (I, [P, ctypes.c_double]),
    "blip_probe_l2_read": (I, [P, ctypes.c_size_t, I, P]),
    "blip_probe_gather": (I, [P, P, I, P, P, P, I, P]),
}

_lock = threading.Lock()
_lib = None


class BlipError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = ERRORS.get(code, "unknown error")
        if code == -4 and _lib is not None:
            msg += f" (cudaError {_lib.blip_last_cuda_error()})"
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def lib():
    """Load libblip.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in EXPORTED.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise BlipError(rc, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class BlipTable:
    """A device-resident blip coefficient table (``blip_create``).

    ``coeffs``: ``[n1][n2][n3][n_orb]`` real or complex, numpy (host) or torch
    (host or CUDA), float64 or float32 (complex128 / complex64).
    """

    def __init__(self, grid, lattice, coeffs, storage=F32, norm=NORM_BSPLINE):
        import torch
        L = lib()
        self.grid = tuple(int(g) for g in grid)
        self.lattice = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
        keep = None
        if isinstance(coeffs, torch.Tensor):
            c = coeffs.contiguous()
            is_cplx = c.is_complex()
            if is_cplx:
                c = torch.view_as_real(c)
            if c.dtype not in (torch.float64, torch.float32):
                raise TypeError("coefficients must be float64/float32 (or complex)")
            on_dev = 1 if c.is_cuda else 0
            ptr, is_double, keep = c.data_ptr(), int(c.dtype == torch.float64), c
            n_orb = coeffs.shape[-1]
        else:
            a = np.asarray(coeffs)
            is_cplx = np.iscomplexobj(a)
            if is_cplx:
                a = np.ascontiguousarray(a, dtype=np.complex128 if a.dtype != np.complex64 else np.complex64)
                is_double = int(a.dtype == np.complex128)
                a = a.view(np.float64 if is_double else np.float32)
            else:
                if a.dtype not in (np.float64, np.float32):
                    a = a.astype(np.float64)
                a = np.ascontiguousarray(a)
                is_double = int(a.dtype == np.float64)
            ptr, on_dev, keep = a.ctypes.data, 0, a
            n_orb = np.asarray(coeffs).shape[-1]
        if tuple(np.shape(coeffs)[:3]) != self.grid:
            raise ValueError("table shape does not match grid")
        if is_cplx != (storage in (C64, BF16PAIR)):
            raise ValueError("complex tables need C64/BF16PAIR storage and vice versa")
        self.n_orb = int(n_orb)
        self.storage = storage
        self.is_complex = storage in (C64, BF16PAIR)
        self.Lreal = self.n_orb * (2 if self.is_complex else 1)
        g = (ctypes.c_int * 3)(*self.grid)
        lat = (ctypes.c_double * 9)(*self.lattice.reshape(-1))
        h = P()
        _check(L.blip_create(g, lat, self.n_orb, storage, norm, P(ptr), is_double, on_dev,
                             ctypes.byref(h)), "blip_create")
        del keep
        self._h = h
        self._lib = L

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.blip_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- evaluation ---------------------------------------------------------
    def alloc_outputs(self, n_elec, values_only=False, device="cuda"):
        import torch
        v = torch.empty((n_elec, self.Lreal), dtype=torch.float32, device=device)
        if values_only:
            return v, None, None
        return (v, torch.empty((n_elec, 3, self.Lreal), dtype=torch.float32, device=device),
                torch.empty((n_elec, self.Lreal), dtype=torch.float32, device=device))

    def eval(self, pos, offsets=None, values_only=False, out=None, stream=None):
        """Device evaluation (``blip_eval``).  ``pos``: CUDA float64 [E][3];
        ``offsets``: CUDA int32 [W+1] or None.  Returns (values, grads, laps)
        as float32 tensors ([E][L], [E][3][L], [E][L]; complex tables give
        [E][2L] interleaved - see ``as_complex``)."""
        import torch
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()):
            raise TypeError("pos must be a contiguous CUDA float64 tensor")
        n = pos.shape[0]
        v, g, lp = out if out is not None else self.alloc_outputs(n, values_only, pos.device)
        nw = 0
        optr = None
        if offsets is not None:
            if not (offsets.is_cuda and offsets.dtype == torch.int32 and offsets.is_contiguous()):
                raise TypeError("offsets must be a contiguous CUDA int32 tensor")
            nw = offsets.shape[0] - 1
            optr = P(offsets.data_ptr())
        _check(self._lib.blip_eval(self._h, P(pos.data_ptr()), n, optr, nw, P(v.data_ptr()),
                                   P(g.data_ptr()) if g is not None else None,
                                   P(lp.data_ptr()) if lp is not None else None,
                                   _stream_ptr(stream)), "blip_eval")
        return v, g, lp

    def eval_host(self, pos, offsets=None, values_only=False, out=None):
        """Host-buffer evaluation (``blip_eval_host``): numpy or CPU torch
        arrays in and out (pinned memory makes the copies faster)."""
        import torch

        def ptr(x):
            if isinstance(x, torch.Tensor):
                assert not x.is_cuda and x.is_contiguous()
                return x.data_ptr()
            return x.ctypes.data

        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        n = pos.shape[0]
        if out is None:
            v = np.empty((n, self.Lreal), dtype=np.float32)
            g = None if values_only else np.empty((n, 3, self.Lreal), dtype=np.float32)
            lp = None if values_only else np.empty((n, self.Lreal), dtype=np.float32)
        else:
            v, g, lp = out
        nw = 0
        optr = None
        if offsets is not None:
            if isinstance(offsets, np.ndarray):
                offsets = np.ascontiguousarray(offsets, dtype=np.int32)
            nw = offsets.shape[0] - 1
            optr = P(ptr(offsets))
        _check(self._lib.blip_eval_host(self._h, P(ptr(pos)), n, optr, nw, P(ptr(v)),
                                        P(ptr(g)) if g is not None else None,
                                        P(ptr(lp)) if lp is not None else None), "blip_eval_host")
        return v, g, lp

    def eval_ratio(self, pos, inv_cols, offsets=None, with_values=False, sort=0, stream=None,
                   values_out=None):
        """Fused ratio (``blip_eval_ratio``): returns (ratio [E][5], values or
        None).  ``inv_cols``: CUDA float32 [E][n_orb], column j of the inverse
        Slater matrix for electron j; ``values_out``: a preallocated
        [E][n_orb] float32 CUDA tensor for the new rows (implies
        with_values)."""
        import torch
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()):
            raise TypeError("pos must be a contiguous CUDA float64 tensor")
        if not (inv_cols.is_cuda and inv_cols.dtype == torch.float32 and inv_cols.is_contiguous()):
            raise TypeError("inv_cols must be a contiguous CUDA float32 tensor")
        n = pos.shape[0]
        ratio = torch.empty((n, 5), dtype=torch.float32, device=pos.device)
        if values_out is not None:
            if not (values_out.is_cuda and values_out.dtype == torch.float32 and
                    values_out.is_contiguous() and values_out.numel() >= n * self.Lreal):
                raise TypeError("values_out must be a contiguous CUDA float32 tensor of E x n_orb")
            vals = values_out
        else:
            vals = torch.empty((n, self.Lreal), dtype=torch.float32, device=pos.device) \
                if with_values else None
        nw = 0 if offsets is None else offsets.shape[0] - 1
        _check(self._lib.blip_eval_ratio(self._h, P(pos.data_ptr()), n,
                                         P(offsets.data_ptr()) if offsets is not None else None,
                                         nw, P(inv_cols.data_ptr()), P(ratio.data_ptr()),
                                         P(vals.data_ptr()) if vals is not None else None,
                                         int(sort), _stream_ptr(stream)), "blip_eval_ratio")
        return ratio, vals

    def probe_gather(self, pos, out=None, store=True, stream=None):
        """Measurement probe (``blip_probe_gather``): the row loads (and, if
        ``store``, the output stores) of an evaluation of ``pos`` without its
        arithmetic.  ``out``: outputs from ``alloc_outputs`` (written with
        meaningless contents)."""
        import torch
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()):
            raise TypeError("pos must be a contiguous CUDA float64 tensor")
        n = pos.shape[0]
        v = g = lp = None
        if store:
            v, g, lp = out if out is not None else self.alloc_outputs(n, False, pos.device)
        _check(self._lib.blip_probe_gather(self._h, P(pos.data_ptr()), n,
                                           P(v.data_ptr()) if v is not None else None,
                                           P(g.data_ptr()) if g is not None else None,
                                           P(lp.data_ptr()) if lp is not None else None,
                                           1 if store else 0, _stream_ptr(stream)),
               "blip_probe_gather")

    def status(self):
        s = ctypes.c_int(0)
        _check(self._lib.blip_status(self._h, ctypes.byref(s)), "blip_status")
        return s.value

    def info(self):
        a = (ctypes.c_longlong * 8)()
        _check(self._lib.blip_info(self._h, a), "blip_info")
        keys = ["rows", "row_stride", "Lreal", "elem_bytes", "table_bytes", "storage",
                "sm_count", "variant"]
        return dict(zip(keys, [int(x) for x in a]))

    def set_kpoints(self, kfrac, koffs):
        """Bloch k-points (``blip_set_kpoints``): kfrac [n_k][3] in
        reciprocal-lattice units, koffs [n_k + 1] complex-orbital offsets.
        ``kfrac=None`` clears them."""
        if kfrac is None:
            _check(self._lib.blip_set_kpoints(self._h, 0, None, None), "blip_set_kpoints")
            return
        kf = np.ascontiguousarray(kfrac, dtype=np.float64).reshape(-1, 3)
        ko = np.ascontiguousarray(koffs, dtype=np.int32)
        _check(self._lib.blip_set_kpoints(self._h, kf.shape[0], P(kf.ctypes.data),
                                          P(ko.ctypes.data)), "blip_set_kpoints")

    def set_l2_residency(self, fraction):
        """Keep a share of the table resident in L2 (``blip_set_l2_residency``);
        0 turns it off.  Applies to launches on non-default streams."""
        _check(self._lib.blip_set_l2_residency(self._h, float(fraction)), "blip_set_l2_residency")

    def set_kernel(self, variant=1, chunks=1, warps=8, sort=0):
        _check(self._lib.blip_set_kernel(self._h, variant, chunks, warps, sort), "blip_set_kernel")

    def autotune(self, pos, offsets=None, values_only=False, out=None, stream=None):
        n = pos.shape[0]
        v, g, lp = out if out is not None else self.alloc_outputs(n, values_only, pos.device)
        chosen = (ctypes.c_int * 4)()
        nw = 0 if offsets is None else offsets.shape[0] - 1
        _check(self._lib.blip_autotune(self._h, P(pos.data_ptr()), n,
                                       P(offsets.data_ptr()) if offsets is not None else None, nw,
                                       P(v.data_ptr()), P(g.data_ptr()) if g is not None else None,
                                       P(lp.data_ptr()) if lp is not None else None,
                                       _stream_ptr(stream), chosen), "blip_autotune")
        return tuple(chosen)

    def graph(self, pos, out, per_launch, offsets=None):
        """Capture an evaluation into a CUDA graph (``blip_graph_create``)."""
        v, g, lp = out
        h = P()
        nw = 0 if offsets is None else offsets.shape[0] - 1
        _check(self._lib.blip_graph_create(self._h, P(pos.data_ptr()), pos.shape[0],
                                           P(offsets.data_ptr()) if offsets is not None else None,
                                           nw, P(v.data_ptr()),
                                           P(g.data_ptr()) if g is not None else None,
                                           P(lp.data_ptr()) if lp is not None else None,
                                           int(per_launch), ctypes.byref(h)), "blip_graph_create")
        return BlipGraph(self, h)

    @staticmethod
    def as_complex(x):
        """View interleaved float32 outputs of a complex table as complex64."""
        import torch
        if isinstance(x, torch.Tensor):
            return torch.view_as_complex(x.reshape(*x.shape[:-1], -1, 2))
        return x.view(np.complex64)


def probe_l2_read(buf, reps, stream=None):
    """Measurement aid (``blip_probe_l2_read``): read the CUDA tensor ``buf``
    ``reps`` times through L2 in one launch."""
    if not (buf.is_cuda and buf.is_contiguous()):
        raise TypeError("buf must be a contiguous CUDA tensor")
    _check(lib().blip_probe_l2_read(P(buf.data_ptr()), buf.numel() * buf.element_size(),
                                    int(reps), _stream_ptr(stream)), "blip_probe_l2_read")


def sm_update(dinv, rows, cols, work=None, stream=None):
    """Sherman-Morrison row update of a batch of inverses (``blip_sm_update``).

    dinv: CUDA float32 [W][n][n] (updated in place); rows: CUDA float32
    [W][n]; cols: CUDA int32 [W] (-1 = no update).  Returns the work buffer
    ([W][2n]: w = psi' Dinv, then the old column j)."""
    import torch
    W, n = dinv.shape[0], dinv.shape[1]
    for x, dt in ((dinv, torch.float32), (rows, torch.float32), (cols, torch.int32)):
        if not (x.is_cuda and x.dtype == dt and x.is_contiguous()):
            raise TypeError("sm_update expects contiguous CUDA tensors (float32, float32, int32)")
    if work is None:
        work = torch.empty((W, 2 * n), dtype=torch.float32, device=dinv.device)
    _check(lib().blip_sm_update(W, n, P(dinv.data_ptr()), P(rows.data_ptr()), P(cols.data_ptr()),
                                P(work.data_ptr()), _stream_ptr(stream)), "blip_sm_update")
    return work


class BlipGraph:
    def __init__(self, table, h):
        self._t = table
        self._h = h

    def launch(self, stream=None):
        _check(self._t._lib.blip_graph_launch(self._h, _stream_ptr(stream)), "blip_graph_launch")

    def close(self):
        if self._h is not None and self._h.value:
            self._t._lib.blip_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
