"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle under a rigorous per-output error bound.

Bound (FP32 path): |o_gpu - o_ref| <= TAU32 * C_o, where
C_o = sum_s |W_o(s)| |a_{l,s}| is computed by the oracle for every output
(``absmag``).  TAU32 = 8e-6 ~ (64 + 70) * 2^-24 covers the FP32 rounding of
the offset t, of the weights (a few operations each) and of the 64-term FP32
accumulation, plus the FP64 -> FP32 rounding of the coefficients.

Quantised tables add the coefficient rounding: |delta a| <= u |a| with
u = 2^-8 (BF16) or 2^-11 (FP16), plus an FP16 subnormal term
2^-25 * s_l * sum_s |W_o(s)| for coefficients below 2^-14 * s_l.
"""
from __future__ import annotations

import functools

import numpy as np

import blip_inputs as bi
import oracle

TAU32 = 8e-6
U_Q = {1: 2.0 ** -8, 2: 2.0 ** -11, 4: 2.0 ** -8}   # storage kind -> unit roundoff


@functools.lru_cache(maxsize=4)
def cached_table(name, **kw):
    w = bi.workload(name, **dict(kw))
    return w, w.table()


def gpu_eval(table, pos_np, offsets=None, values_only=False):
    """Evaluate on the GPU through the C ABI; return numpy arrays."""
    import torch
    pos = torch.from_numpy(np.ascontiguousarray(pos_np, dtype=np.float64)).cuda()
    offs = None if offsets is None else torch.from_numpy(np.asarray(offsets, dtype=np.int32)).cuda()
    v, g, lp = table.eval(pos, offs, values_only=values_only)
    torch.cuda.synchronize()
    out = [v.cpu().numpy()]
    if not values_only:
        out += [g.cpu().numpy(), lp.cpu().numpy()]
    return out


def sum_abs_weights(grid, lattice, pos, norm=0):
    """sum_s |W_o(s)| per electron and output kind (oracle, table of ones)."""
    ones = np.ones(tuple(grid) + (1,))
    _, _, _, mag = oracle.eval_stencil(grid, lattice, ones, pos, norm=norm, absmag=True)
    return mag[:, :, 0]                                   # [E][5]


def compare(grid, lattice, coeffs, pos, gpu_out, storage=0, norm=0, scales=None, sample=None):
    """Check GPU outputs against the oracle for electrons ``sample`` (all if
    None).  Returns a dict of error statistics; raises AssertionError if any
    output breaks its bound."""
    idx = np.arange(len(pos)) if sample is None else np.asarray(sample)
    p = np.asarray(pos)[idx]
    v, g, lp, mag = oracle.eval_stencil(grid, lattice, coeffs, p, norm=norm, absmag=True)
    cplx = np.iscomplexobj(coeffs)
    if cplx:
        v, g, lp = (x.view(np.float64) for x in (v, g, lp))
    ref = [v, g.reshape(len(idx), 3, -1), lp]
    mags = [mag[:, 0], mag[:, 1:4], mag[:, 4]]
    tau = TAU32 + U_Q.get(storage, 0.0)
    sub = None
    if storage == 2:        # FP16 subnormal floor
        sw = sum_abs_weights(grid, lattice, p, norm)
        s = np.asarray(scales)[None, :]
        sub = [2.0 ** -25 * sw[:, 0:1] * s, 2.0 ** -25 * sw[:, 1:4, None] * s[:, None, :],
               2.0 ** -25 * sw[:, 4:5] * s]
    stats = {}
    names = ["value", "grad", "lap"]
    for k, name in enumerate(names):
        got = np.asarray(gpu_out[k])[idx].astype(np.float64)
        err = np.abs(got - ref[k])
        bound = tau * mags[k] + 1e-30
        if sub is not None:
            bound = bound + sub[k]
        ratio = err / bound
        stats[name] = {
            "max_abs": float(np.nanmax(err)),
            "rms_abs": float(np.sqrt(np.nanmean(err ** 2))),
            "max_rel_to_C": float(np.nanmax(err / (mags[k] + 1e-300))),
            "max_rel": float(np.nanmax(err / (np.abs(ref[k]) + 1e-3 * np.abs(ref[k]).max()))),
            "max_bound_ratio": float(np.nanmax(ratio)),
        }
        bad = ~(ratio <= 1.0)
        if bad.any():
            where = np.argwhere(bad)
            rows = sorted(set(int(i) for i in where[:, 0]))
            cols = sorted(set(int(i) for i in where[:, -1]))
            raise AssertionError(
                f"{name}: {int(bad.sum())} outputs break the bound; worst ratio "
                f"{float(np.nanmax(ratio)):.3g}; electrons {rows[:12]} of {len(p)}, "
                f"components {cols[:12]}; first bad: got {got[tuple(where[0])]!r} "
                f"ref {ref[k][tuple(where[0])]!r}")
    return stats


def kinetic_error_bound(values, laps, bound_v, bound_l, blocks):
    """First-order bound on |T_L(gpu) - T_L(ref)| from elementwise output
    bounds.  With X = D^{-1} Lap,
        dT = -1/2 [tr(D^{-1} dLap) - tr(D^{-1} dD X)],
    so |dT| <= 1/2 [sum |D^{-1}|^T * B_lap + sum |X D^{-1}|^T * B_val]
    (elementwise products summed), per spin block."""
    total = 0.0
    for j0, j1 in blocks:
        m = j1 - j0
        D = np.asarray(values[j0:j1, :m], dtype=np.float64)
        Lp = np.asarray(laps[j0:j1, :m], dtype=np.float64)
        Di = np.linalg.inv(D)
        X = Di @ Lp
        total += 0.5 * (np.sum(np.abs(Di).T * bound_l[j0:j1, :m])
                        + np.sum(np.abs(X @ Di).T * bound_v[j0:j1, :m]))
    return total
