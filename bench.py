#!/usr/bin/env python
"""Benchmark: orbital x electron evaluations per second (value + gradient +
Laplacian) of the periodic cubic-blip path on GB300.

Default workload: the quasi-simultaneous precision batch on the TiO2-shaped
table (tetragonal 17.4 x 17.4 x 11.2 bohr, 72 x 72 x 48 grid, 768 real
orbitals): 1,024 walkers x 1,536 trial moves (Gaussian, sigma 0.3 bohr) in
one launch per step, FP32 storage for the headline value.  A step is one
blip_eval of the batch; L2 is flushed (512 MB write, then 512 MB read so no
dirty lines remain) between steps outside the per-step CUDA-event window.
Beside it the line carries BF16 and FP16 storage on the same positions
(throughput, error against the FP64 oracle on sampled electrons, and the
Slater-only kinetic-energy error per primitive cell of two walkers), the
values-only and fused-ratio paths, the batch sweep of 256 walkers x
b in {1, 8, 32, 128, 1536} for FP32 and BF16, and the 1,536-electron
single-walker launch (all at once and one electron per launch).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import blip_inputs as bi  # noqa: E402

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the evaluation kernel on this workload, from ncu, keyed by the SHA-256 of
# the evaluation-path code it was measured on (kernel_hash) and by the
# kernel (variant, chunks); reported as null once those sources change.
# Filled from the committed summaries under profiles/.
NCU_TRAFFIC = {
    # (kernel source hash, workload, storage, electrons): {(variant, chunks): bytes}
    ("33f210082c611060", "tio2", "f32", 1536): {(11, 1): 276002560 + 13652480,
                                                (9, 1): 275730688 + 12409344,
                                                (3, 2): 274905344 + 11279616},
    # captured with 128 orbitals, scaled x6 to 768 (rows and outputs grow
    # in proportion to the orbital count)
    ("33f210082c611060", "tio2_batch", "f32", 393216): {(8, 4): 6 * (156558592 + 947191552)},
    # tensor-core kernel: captured on the electrons of a slab (a_1 < 1/8) of
    # the batch at the same density (196,327 electrons), scaled by electrons
    # to the full batch (outputs dominate: traffic grows in proportion)
    ("fbf8723eb9be50ef", "tio2_precision", "f32", 1572864): {
        (12, 1): (321207552 + 2954819072) * 1572864 // 196327},
}

# the metric and its unit, identical in every arm of the benchmark
METRIC = "orbital\u00b7electron evals/s (val+grad+lap), % HBM roofline; BF16 vs FP32 at err"
UNIT = "orbital*electron evals/s (val+grad+lap)"

STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "c64": 3, "bf16pair": 4}
DTYPE = {"f32": "f32", "bf16": "bf16", "f16": "f16", "c64": "f32", "bf16pair": "bf16"}
ELEM_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "c64": 4, "bf16pair": 2}   # per real component


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tio2_precision",
                    choices=["tio2", "tio2_batch", "tio2_precision", "cubic16",
                             "tio2_super_complex", "sm_update"])
    ap.add_argument("--batch", type=int, default=1536, help="electrons per walker (tio2_batch)")
    ap.add_argument("--walkers", type=int, default=0, help="override walker count")
    ap.add_argument("--orbitals", type=int, default=0,
                    help="override the orbital count (smaller profiling cases)")
    ap.add_argument("--storage", default="f32", choices=list(STORAGE))
    ap.add_argument("--kernel", default="auto", help="auto | variant,chunks,warps,sort")
    ap.add_argument("--step", default="eval", choices=["eval", "ratio"],
                    help="the timed step: the evaluation (blip_eval) or the fused ratio "
                         "(blip_eval_ratio, cell order, seeded N(0,1) inverse columns)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the access-pattern probe and the SGEMM peak")
    ap.add_argument("--warm", action="store_true",
                    help="no L2 flush between steps (tables that fit in L2)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--slab", type=float, default=0.0,
                    help="keep only the electrons with fractional a_1 coordinate below this "
                         "(a smaller case at the same density, for profiling captures)")
    ap.add_argument("--sweep", default="1,8,32,128,1536",
                    help="batch sizes of the 256-walker sweep extra ('' for none)")
    return ap.parse_args()


def make_workload(args, rank):
    kw = {}
    if args.workload == "tio2_batch":
        kw["batch"] = args.batch
    if args.walkers:
        kw["n_walkers"] = args.walkers
    if args.orbitals:
        kw["n_orb"] = args.orbitals
    w = bi.workload(args.workload, **kw)
    from paper_1204_1121_gb300 import replicas
    w.pos_seed = replicas.weak_seed(w.pos_seed, rank)   # each rank: its own walkers
    return w


def describe(w, args, E):
    d = {"workload": f"{w.name}: cell {np.diag(w.lattice).tolist()} bohr, grid "
                     f"{'x'.join(map(str, w.grid))}, {w.n_orb} "
                     f"{'complex' if w.is_complex else 'real'} orbitals, {E} positions per step"
                     + (f" ({w.n_walkers} walkers)" if w.n_walkers > 1 else " (all at once)"),
         "electrons": E, "orbitals": w.n_orb, "storage": args.storage,
         "l2": "warm (no flush between steps)" if args.warm else
               "flushed between steps (512 MB write + 512 MB read, outside the event window)",
         "positions": "uniform in cell" if w.uniform_n else "walker configs + N(0,0.3^2) moves"}
    if args.slab > 0:
        d["slab"] = f"electrons with fractional a_1 coordinate below {args.slab} only"
    if getattr(args, "step", "eval") == "ratio":
        d["step"] = ("blip_eval_ratio in cell order: sum_l {psi, grad, lap}_l c_j[l] with "
                     "seeded N(0,1) columns c_j (5 floats per electron out)")
    return d


def touched_sites(grid, lattice, pos):
    """Distinct grid sites whose coefficients a launch must read (the 4x4x4
    stencils of all positions), for the compulsory-traffic model."""
    n = np.array(grid)
    ainv = np.linalg.inv(np.asarray(lattice, dtype=np.float64).T)
    u = pos @ ainv.T
    u -= np.floor(u)
    u[u >= 1.0] = 0.0
    base = np.floor(u * n).astype(np.int64) % n
    mark = np.zeros(int(np.prod(n)), dtype=bool)
    for kx in range(4):
        ix = (base[:, 0] - 1 + kx) % n[0]
        for ky in range(4):
            iy = (base[:, 1] - 1 + ky) % n[1]
            for kz in range(4):
                iz = (base[:, 2] - 1 + kz) % n[2]
                mark[(ix * n[1] + iy) * n[2] + iz] = True
    return int(mark.sum())


def _code_only(text):
    """Source text without comments and with whitespace runs collapsed, so
    that comment edits keep the hash."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


# sources outside the evaluation path: the Sherman-Morrison update and the
# two fused-ratio kernels
_NOT_EVAL_PATH = ("blip_sm.cu", "blip_ratio.cu", "blip_ratio_tc.cu")


def kernel_hash():
    """SHA-256 (16 hex digits) of the code (comments aside) of every CUDA
    source of the evaluation path (all of the library but the
    Sherman-Morrison update and the fused-ratio kernels)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1204_1121_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f not in _NOT_EVAL_PATH:
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                h.update(f.encode() + b"\0" + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def sgemm_tflops(n=8192, reps=5):
    """Measured FP32 (CUDA-core) throughput of this GPU: cuBLAS SGEMM n^3 with
    TF32 off, best of `reps` CUDA-event timings.  Reported beside the FP32
    peak derived from unit counts and the clock."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.randn((n, n), generator=g, device="cuda")
        b = torch.randn((n, n), generator=g, device="cuda")
        c = torch.empty((n, n), device="cuda")
        for _ in range(2):
            torch.matmul(a, b, out=c)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def tensor_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("bf16_tflops"):
            return d["bf16_tflops"], "measured"
    return 1900.0, "fallback"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_baseline(w, tab, pos, seconds):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample."""
    import oracle
    cores = os.cpu_count() or 1
    E = len(pos)
    t0 = time.perf_counter()
    oracle.eval_stencil(w.grid, w.lattice, tab, pos[: min(E, 256)], threads=cores)
    probe = time.perf_counter() - t0
    per_e = probe / min(E, 256)
    n = int(max(64, min(E, seconds / max(per_e, 1e-9))))
    t0 = time.perf_counter()
    oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
    per_pass = time.perf_counter() - t0
    reps = max(1, min(2000, int(seconds / max(per_pass, 1e-9))))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
    dt = time.perf_counter() - t0
    Lr = w.n_orb
    # one core too (the kind of baseline the paper's 30x figure used): a
    # sample of about a tenth of the time above
    n1 = max(16, min(n, int(0.1 * seconds / max(per_e * cores, 1e-9))))
    t1 = time.perf_counter()
    oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n1], threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": n * reps * Lr / dt, "unit": UNIT,
            "cores": cores, "kind": "oracle",
            "sample": f"first {n} of {E} positions x {reps} repeats, FP64, {cores} threads, "
                      f"{dt:.1f} s",
            "single_core": {"value": n1 * Lr / dt1, "cores": 1,
                            "sample": f"first {n1} of {E} positions, FP64, 1 thread, "
                                      f"{dt1:.1f} s"}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import oracle
    w = make_workload(args, 0)
    tab = w.table()
    pos, offs = w.positions()
    cores = os.cpu_count() or 1
    E = len(pos)
    # bound each step to about 1.5 s of wall time
    t0 = time.perf_counter()
    oracle.eval_stencil(w.grid, w.lattice, tab, pos[: min(E, 256)], threads=cores)
    per_e = (time.perf_counter() - t0) / min(E, 256)
    n = int(max(16, min(E, 1.5 / max(per_e, 1e-9))))
    for _ in range(args.warmup):
        oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = n * w.n_orb / (ms / 1e3)
    unit = UNIT
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, args, E),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} of {E} positions per step, FP64, {cores} threads"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_sm(args):
    """Sherman-Morrison inverse updates: 256 walkers x one accepted move each,
    n = 768 (one spin of the 1,536-electron TiO2 cell).  HBM-bound: the
    inverse is read and written once, 8 n^2 bytes per walker update."""
    import torch
    import paper_1204_1121_gb300 as pb
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    W = args.walkers or 256
    n = 768
    g = torch.Generator(device="cuda").manual_seed(7)
    dinv = torch.randn((W, n, n), generator=g, device="cuda") * 0.05
    dinv += torch.eye(n, device="cuda")
    rows = torch.randn((W, n), generator=g, device="cuda")
    cols = torch.arange(W, dtype=torch.int32, device="cuda") % n
    work = torch.empty((W, 2 * n), device="cuda")
    # L2 flush as in the evaluation benchmark: write 512 MB, then read
    # another 512 MB, so no dirty lines are charged to the update
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    flush_rd = torch.ones(512 * 1024 * 1024 // 4, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(max(3, args.warmup)):
        pb.sm_update(dinv, rows, cols, work)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    sleep = getattr(torch.cuda, "_sleep", None)
    if sleep is not None:              # the host enqueues every step first
        sleep(int(2.0e9 * (0.05 + 0.002 * args.steps)))
    for k in range(args.steps):
        flush.fill_(float(k))
        flush_rd.sum()
        evs[k][0].record(stream)
        pb.sm_update(dinv, rows, cols, work)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    bytes_alg = W * (8.0 * n * n + 16.0 * n)
    peak, kind = measured_peaks()
    ach = bytes_alg / (ms / 1e3) / 1e9
    line = {"metric": "walker inverse updates/s (Sherman-Morrison, n=768)", "value": W / (ms / 1e3),
            "unit": "updates/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sm_update: {W} walkers x 1 accepted move, n = {n}",
                       "l2": "flushed between steps (512 MB write + 512 MB read, outside the event window)"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": None,
                         "algorithmic_bytes_per_launch": bytes_alg},
            "gpu_launches": 2 * args.steps}
    print(json.dumps(line))
    return 0


class Stepper:
    """Timing of repeated launches: L2 flush between launches (512 MB
    written, then 512 MB read, so no dirty lines are charged to the next
    launch), a device-side hold so that the host enqueues every launch
    before the first one starts, CUDA events around each launch on the
    launching stream."""

    def __init__(self, warm_l2, stream):
        import torch
        self.torch = torch
        self.warm = warm_l2
        self.stream = stream
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        self.flush_rd = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2(self, k):
        if self.warm:                  # warm L2: the table stays cached between steps
            return
        self.flush.fill_(float(k))
        self.flush_rd.sum()

    def hold(self, steps, per_step_s=0.002):
        # a device-side wait (torch's spin kernel) ahead of timed launches:
        # the host enqueues them all while it runs, so a host stall cannot
        # leave the GPU idle inside a step's CUDA-event window; it runs
        # before the first event, outside every window
        sleep = getattr(self.torch.cuda, "_sleep", None)
        if sleep is not None:
            sleep(int(2.0e9 * (0.05 + per_step_s * steps)))

    def time(self, fn, K, warmup=3):
        """Per-launch times (ms) of K launches of fn()."""
        torch = self.torch
        for k in range(warmup):
            self.flush_l2(k)
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        torch.cuda.synchronize()
        self.hold(K)
        for k in range(K):
            self.flush_l2(k)
            evs[k][0].record(self.stream)
            fn()
            evs[k][1].record(self.stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]


def launch_model(mode, E, Lr, U, b_c):
    """Algorithmic bytes and FP32 FLOPs of one launch.  mode: 'full' (value,
    gradient, Laplacian: 20 L B and 640 FLOP per eval), 'vonly' (4 L B, 128
    FLOP), 'ratio' (the inverse columns read, 4 L B, five floats written per
    electron, 650 FLOP per eval).  Table bytes: the U touched rows once."""
    out = {"full": 20.0 * Lr * E, "vonly": 4.0 * Lr * E,
           "ratio": 4.0 * Lr * E + 20.0 * E}[mode]
    fl = {"full": 640.0, "vonly": 128.0, "ratio": 650.0}[mode] * Lr * E
    return U * Lr * b_c + out + 24.0 * E, fl


def tensor_products(kernel, storage):
    """16-bit tensor-core products per algorithmic FMA of the tensor-core
    kernel (variant 12): weights in two parts against a 16-bit table (2), or
    against an FP32 table's two FP16 planes less the lo x lo term (3); 0 for
    the CUDA-core kernels."""
    if kernel is None or int(kernel[0]) != 12:
        return 0
    return 3 if storage in ("f32", "c64") else 2


def roofline(bytes_alg, flops, ms, sms, products=0):
    """The binding roofline of one launch: HBM (measured copy bandwidth) or
    the arithmetic pipe the kernel contracts on: the FP32 FMA pipe (SMs x
    128 lanes x 2 FLOP x 2.07 GHz) for the CUDA-core kernels; for the
    tensor-core kernel the measured dense BF16 tensor peak (burst) with the
    algorithmic FLOPs times the 16-bit products each FMA takes."""
    peak, peak_kind = measured_peaks()
    f32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    t_hbm = bytes_alg / (peak * 1e9)
    hbm_ach = bytes_alg / (ms / 1e3) / 1e9
    alu_ach = flops / (ms / 1e3) / 1e12
    if products:
        tc_peak, tc_kind = tensor_peak()
        work = flops * products
        t_cmp = work / (tc_peak * 1e12)
        cmp = {"bound": "tensor", "achieved": work / (ms / 1e3) / 1e12, "peak": tc_peak,
               "unit": "TFLOP/s", "frac": work / (ms / 1e3) / 1e12 / tc_peak,
               "peak_kind": f"{tc_kind} dense BF16 tensor throughput (burst); "
                            f"{products} 16-bit products per FMA"}
    else:
        t_cmp = flops / (f32_peak * 1e12)
        cmp = {"bound": "alu", "achieved": alu_ach, "peak": f32_peak, "unit": "TFLOP/s",
               "frac": alu_ach / f32_peak,
               "peak_kind": f"FP32 FMA: {sms} SMs x 128 lanes x 2 FLOP x 2.07 GHz"}
    if t_hbm >= t_cmp:
        r = {"bound": "hbm", "achieved": hbm_ach, "peak": peak, "unit": "GB/s",
             "frac": hbm_ach / peak, "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"}
    else:
        r = cmp
    r.update({"algorithmic_bytes_per_launch": bytes_alg, "fp32_flop_per_launch": flops,
              "hbm_frac": hbm_ach / peak, "alu_frac": alu_ach / f32_peak,
              "roof_time_us": 1e6 * max(t_hbm, t_cmp)})
    if products:
        r["tensor_frac"] = cmp["frac"]
    return r


def sample_idx(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, size=k)]))


def error_stats(w, tab, pos, idx, rows):
    """Max and RMS error of GPU outputs ``rows`` (values, grads, laps at
    electrons idx) against the FP64 oracle, absolute and relative to the
    rounding scale C_o = sum_s |W_o(s)| |a_ls|."""
    import oracle
    v, g, lp, mag = oracle.eval_stencil(w.grid, w.lattice, tab, pos[idx], absmag=True)
    refs = [v, g, lp]
    mags = [mag[:, 0], mag[:, 1:4], mag[:, 4]]
    out = {}
    for name, got, ref, m in zip(("value", "grad", "lap"), rows, refs, mags):
        err = np.abs(np.asarray(got, dtype=np.float64) - ref)
        out[name] = {"max_abs": float(err.max()), "rms_abs": float(np.sqrt(np.mean(err ** 2))),
                     "max_rel_to_C": float((err / (m + 1e-300)).max()),
                     "ref_rms": float(np.sqrt(np.mean(ref ** 2)))}
    return out


def kinetic_errors(w, tab, pos, vals, laps, n_walk=2, per=1536):
    """|T_L(gpu) - T_L(oracle)| / 64 per walker (Slater-only local kinetic
    energy, two spins of per/2 electrons, 64 primitive cells per walker)."""
    import oracle
    h = per // 2
    blocks = [(0, h), (h, per)]
    out = []
    for wk in range(n_walk):
        p0 = pos[per * wk:per * (wk + 1)]
        rv, _, rl = oracle.eval_stencil(w.grid, w.lattice, tab, p0)
        T_ref, conds = oracle.kinetic.local_kinetic(rv, rl, blocks)
        T_gpu, _ = oracle.kinetic.local_kinetic(vals[per * wk:per * (wk + 1)],
                                                laps[per * wk:per * (wk + 1)], blocks)
        out.append({"T_ref": T_ref, "err_per_cell": abs(T_gpu - T_ref) / 64.0,
                    "cond": max(conds)})
    return out


def main():
    args = parse()
    if args.workload == "sm_update":
        return run_sm(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1204_1121_gb300 as pb
    from paper_1204_1121_gb300 import replicas

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = make_workload(args, rank)
    if w.is_complex and args.storage in ("f32", "bf16", "f16"):
        args.storage = "c64"
    spectral = bool(w.extra.get("spectral"))
    tab = w.table(device="cuda") if spectral else w.table()
    pos, offs = w.positions()
    if args.slab > 0:
        # the electrons of a slab of the cell (one walker of what is left)
        u = pos @ np.linalg.inv(np.asarray(w.lattice, dtype=np.float64))
        pos = np.ascontiguousarray(pos[(u[:, 0] - np.floor(u[:, 0])) < args.slab])
        offs = np.array([0, len(pos)], dtype=np.int32)
        args.no_extra = True
    E = len(pos)
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=STORAGE[args.storage])
    if spectral:                       # the FP64 device copy is no longer needed
        del tab
        tab = None
        torch.cuda.empty_cache()
    info = t.info()
    sms = info["sm_count"]
    Lr = info["Lreal"]
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    out = t.alloc_outputs(E)
    stream = torch.cuda.current_stream()
    if args.step == "ratio":
        # the ratio picks its kernel by density (tensor cores for dense batches)
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        cols = torch.randn((E, Lr), generator=g, device="cuda", dtype=torch.float32)
        chosen = (12, 1, 1, 1) if 2 * E >= int(np.prod(w.grid)) else (0, 0, 0, 1)
    elif args.kernel == "auto":
        chosen = t.autotune(dpos, doffs, out=out)
    else:
        v_, c_, w_, s_ = (int(x) for x in args.kernel.split(","))
        t.set_kernel(v_, c_, w_, s_)
        chosen = (v_, c_, w_, s_)
    st_ = Stepper(args.warm, stream)

    def step():
        if args.step == "ratio":
            t.eval_ratio(dpos, cols, doffs, sort=1)
        else:
            t.eval(dpos, doffs, out=out)

    for k in range(max(3, args.warmup)):
        st_.flush_l2(k)
        step()
    torch.cuda.synchronize()
    st = t.status()

    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    st_.hold(K)
    for k in range(K):
        st_.flush_l2(k)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    per = [a.elapsed_time(b) for a, b in evs]
    ms = replicas.max_over_ranks(statistics.mean(per))
    ms_median = replicas.max_over_ranks(statistics.median(per))
    evals = E * w.n_orb
    value = world * evals / (ms / 1e3)

    # roofline of the evaluation kernel (the dominant kernel of the step)
    U = touched_sites(w.grid, w.lattice, pos)
    b_c = ELEM_BYTES[args.storage]
    bytes_alg, flops = launch_model("ratio" if args.step == "ratio" else "full", E, Lr, U, b_c)
    roof = roofline(bytes_alg, flops, ms, sms, tensor_products(chosen, args.storage))
    kh = kernel_hash()
    roof["traffic"] = NCU_TRAFFIC.get((kh, w.name, args.storage, E), {}).get(tuple(chosen[:2])) \
        if args.step == "eval" else None
    roof.update({"touched_sites": U, "kernel_source_hash": kh,
                 "gather_model_GBps": (E * 64 * Lr * b_c + 20 * Lr * E) / (ms / 1e3) / 1e9})
    if not args.no_probe and roof["bound"] == "hbm" and E * Lr * 20 > 4e9:
        # the output stream's own ceiling: a plain write of the gradient
        # buffer (12 of the launch's 20 L bytes per electron), timed alike
        g = out[1]
        wms = statistics.mean(st_.time(lambda: g.fill_(0.5), max(3, K // 4)))
        roof["hbm_write_probe_GBps"] = g.numel() * 4 / (wms / 1e3) / 1e9
        roof["frac_of_write_probe"] = roof["achieved"] / roof["hbm_write_probe_GBps"]
    if roof["bound"] == "alu" and not args.no_probe:
        sg = sgemm_tflops()
        roof["fp32_sgemm_tflops"] = sg
        roof["frac_of_sgemm"] = roof["achieved"] / sg
    if roof["bound"] == "alu" and clocks and clocks.get("sm_mhz"):
        # the same fraction at the SM clock sampled during the timed region
        roof["frac_at_sampled_clock"] = roof["frac"] * 2070.0 / clocks["sm_mhz"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "ms_median": ms_median,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.storage], "data": "synthetic",
            "config": describe(w, args, E), "roofline": roof, "clocks": clocks,
            "gpu_launches": K * (6 if chosen[3] else 1), "kernel_choice": list(chosen),
            "status": st, "wall_s_timed_region": wall}

    if not args.no_e2e:
        # end to end through the host-buffer entry point: positions from
        # page-locked host memory, evaluation, all outputs back to page-locked
        # host memory, every step (blip_eval_host)
        try:
            hp = torch.from_numpy(pos).pin_memory()
            ho = torch.from_numpy(offs).pin_memory()
            hv = torch.empty((E, Lr), dtype=torch.float32).pin_memory()
            hg = torch.empty((E, 3, Lr), dtype=torch.float32).pin_memory()
            hl = torch.empty((E, Lr), dtype=torch.float32).pin_memory()
            for _ in range(2):
                t.eval_host(hp, ho, out=(hv, hg, hl))
            tt = []
            for _ in range(K):
                t0 = time.perf_counter()
                t.eval_host(hp, ho, out=(hv, hg, hl))
                tt.append(time.perf_counter() - t0)
            e_ms = replicas.max_over_ranks(1e3 * statistics.mean(tt))
            line["e2e"] = {"value": world * evals / (e_ms / 1e3), "unit": UNIT,
                           "h2d_bytes_per_step": int(hp.numel() * 8 + ho.numel() * 4),
                           "d2h_bytes_per_step": int((hv.numel() + hg.numel() + hl.numel()) * 4),
                           "ms_per_step": e_ms,
                           "api": "blip_eval_host with page-locked host buffers (the kernel "
                                  "reads the positions and writes the outputs across the "
                                  "host link)"}
            del hv, hg, hl
        except RuntimeError as ex:      # host memory: state it in the line
            line["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None,
                           "d2h_bytes_per_step": None,
                           "unavailable": f"page-locked host buffers of the full outputs "
                                          f"({20 * E * Lr / 1e9:.1f} GB): {str(ex)[:120]}"}

    if not args.no_extra and rank == 0 and tab is not None and w.name == "tio2_precision":
        extras_precision(args, pb, w, tab, pos, dpos, doffs, t, out, st_, line, sms, chosen, ms)
    if not args.no_extra and rank == 0 and tab is not None and w.name in ("tio2_precision",
                                                                           "tio2"):
        extras_single_walker(args, pb, w, tab, t, st_, line, sms, stream)
    if not args.no_extra and rank == 0 and w.name == "tio2_precision":
        extras_l2(args, pb, line, sms)

    if w.is_complex:
        line["real_equivalent_value"] = 2 * value
    if rank == 0 and not args.no_cpu_baseline and tab is not None:
        line["cpu_baseline"] = cpu_baseline(w, tab, pos, args.cpu_seconds)

    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _timed_entry(ms_list, E, Lr, U, b_c, mode, sms, chosen=None, storage="f32"):
    ms = statistics.mean(ms_list)
    bytes_alg, flops = launch_model(mode, E, Lr, U, b_c)
    r = roofline(bytes_alg, flops, ms, sms, tensor_products(chosen, storage))
    d = {"us": 1e3 * ms, "evals_per_s": E * Lr / (ms / 1e3), "bound": r["bound"],
         "frac": r["frac"], "hbm_frac": r["hbm_frac"], "alu_frac": r["alu_frac"],
         "roof_us": r["roof_time_us"]}
    if chosen is not None:
        d["kernel"] = list(chosen)
    return d


def extras_precision(args, pb, w, tab, pos, dpos, doffs, t32, out, st_, line, sms, chosen32,
                     ms32):
    """BF16 / FP16 storage on the same positions, errors against the FP64
    oracle, kinetic-energy error per primitive cell, values-only and fused
    ratio paths, and the 256-walker batch sweep."""
    import torch
    E = len(pos)
    K = args.steps
    Lr = t32.info()["Lreal"]
    U = line["roofline"]["touched_sites"]
    idx = sample_idx(E, 62, 1)
    prec = {}
    tables = {"f32": t32}
    for storage in ("f32", "bf16", "f16"):
        if storage == "f32":
            t = t32
            ent = _timed_entry([ms32], E, Lr, U, 4, "full", sms, chosen32, "f32")
            t.eval(dpos, doffs, out=out)          # the outputs again (the write probe used them)
            torch.cuda.synchronize()
        else:
            t = pb.BlipTable(w.grid, w.lattice, tab, storage=STORAGE[storage])
            ch = t.autotune(dpos, doffs, out=out)
            ent = _timed_entry(st_.time(lambda: t.eval(dpos, doffs, out=out), K), E, Lr, U,
                               ELEM_BYTES[storage], "full", sms, ch, storage)
            t.eval(dpos, doffs, out=out)
            torch.cuda.synchronize()
        rows = [out[0][idx].cpu().numpy(), out[1][idx].cpu().numpy(), out[2][idx].cpu().numpy()]
        ent["errors"] = error_stats(w, tab, pos, idx, rows)
        ent["errors"]["sample"] = f"{len(idx)} electrons (seeded) of {E}, all {Lr} orbitals"
        ent["kinetic"] = kinetic_errors(w, tab, pos, out[0][:3072].cpu().numpy(),
                                        out[2][:3072].cpu().numpy())
        ent["status"] = t.status()
        prec[storage] = ent
        tables[storage] = t
    prec["bf16_over_f32_throughput"] = prec["bf16"]["evals_per_s"] / prec["f32"]["evals_per_s"]
    prec["f16_over_f32_throughput"] = prec["f16"]["evals_per_s"] / prec["f32"]["evals_per_s"]
    prec["tolerance"] = ("paper: ~1e-3 hartree per primitive cell (64 cells per 1,536-electron "
                         "walker); kinetic = Slater-only local kinetic energy of walkers 0, 1")
    line["precision"] = prec
    del tables["f16"]

    # values only (the paper's GPU workload) and the fused ratio
    vo = {}
    for storage in ("f32", "bf16"):
        t = tables[storage]
        o1 = (out[0], None, None)
        ch = t.autotune(dpos, doffs, values_only=True, out=o1)
        vo[storage] = _timed_entry(st_.time(lambda: t.eval(dpos, doffs, values_only=True, out=o1),
                                            K), E, Lr, U, ELEM_BYTES[storage], "vonly", sms, ch,
                                   storage)
    line["values_only"] = vo
    cols = out[1].view(-1)[:E * Lr].view(E, Lr)          # any float data will do for timing
    ra = {}
    for storage in ("f32", "bf16"):
        t = tables[storage]
        # sort 1: cell order, the tensor cores for this dense batch (the
        # ratio kernel with the columns as an operand; with the new rows
        # requested, the evaluation kernel's ratio epilogue); sort 2: cell
        # order on the CUDA cores
        ms_l = st_.time(lambda: t.eval_ratio(dpos, cols, doffs, sort=1), max(3, K // 2))
        ent = _timed_entry(ms_l, E, Lr, U, ELEM_BYTES[storage], "ratio", sms, (12, 1, 1, 1),
                           storage)
        ent["sort"] = 1
        ent["kernel_name"] = "blip_ratio_tc (orbital sum on the tensor cores, columns as operand)"
        vals = out[0].view(-1)[:E * Lr].view(E, Lr)
        ms_v = st_.time(lambda: t.eval_ratio(dpos, cols, doffs, sort=1, values_out=vals),
                        max(3, K // 4))
        wv = _timed_entry(ms_v, E, Lr, U, ELEM_BYTES[storage], "ratio", sms, (12, 1, 1, 1),
                          storage)
        ent["with_new_rows"] = {"us": wv["us"], "evals_per_s": wv["evals_per_s"],
                                "kernel_name": "blip_eval_tc ratio epilogue (also writes psi rows)"}
        ms_c = st_.time(lambda: t.eval_ratio(dpos, cols, doffs, sort=2), max(3, K // 4))
        core = _timed_entry(ms_c, E, Lr, U, ELEM_BYTES[storage], "ratio", sms)
        ent["cuda_cores_sorted"] = {k: core[k] for k in ("us", "evals_per_s", "bound", "frac")}
        ent["status"] = t.status()
        ra[storage] = ent
    line["ratio"] = ra

    # 256 walkers x b electrons per walker per launch, FP32 and BF16
    sweep = []
    for b in [int(x) for x in args.sweep.split(",") if x.strip()]:
        wb = bi.workload("tio2_batch", batch=b)
        pb_, ob = wb.positions()
        Eb = len(pb_)
        db, dob = torch.from_numpy(pb_).cuda(), torch.from_numpy(ob).cuda()
        ob_ = (out[0][:Eb], out[1][:Eb], out[2][:Eb])
        Ub = touched_sites(wb.grid, wb.lattice, pb_)
        for storage in ("f32", "bf16"):
            t = tables[storage]
            ch = t.autotune(db, dob, out=ob_)
            ent = _timed_entry(st_.time(lambda: t.eval(db, dob, out=ob_), K), Eb, Lr, Ub,
                               ELEM_BYTES[storage], "full", sms, ch, storage)
            ent.update({"b": b, "E": Eb, "storage": storage})
            # values only (the paper's own GPU workload), autotuned for it
            ov = (out[0][:Eb], None, None)
            chv = t.autotune(db, dob, values_only=True, out=ov)
            vo = _timed_entry(st_.time(lambda: t.eval(db, dob, values_only=True, out=ov),
                                       max(3, K // 2)), Eb, Lr, Ub, ELEM_BYTES[storage],
                              "vonly", sms, chv, storage)
            ent["values_only"] = {k: vo[k] for k in ("us", "evals_per_s", "bound", "frac", "kernel")}
            sweep.append(ent)
    line["batch_sweep"] = sweep


def extras_l2(args, pb, line, sms):
    """A table that fits in L2: the TiO2 primitive cell with 64 k-points
    (15 MB complex64) for 256 walkers x 128 moves drawn in the 4 x 4 x 4
    supercell, on a stream of its own: warm (nothing between launches), and
    with an L2 flush between launches (standing in for the rest of a Monte
    Carlo step) without and with the table's L2 access-policy window; beside
    the L2 read bandwidth of blip_probe_l2_read on a 48 MB buffer."""
    import torch
    w = bi.workload("tio2_kpoints")
    tab = w.table()
    pos, offs = w.positions()
    E = len(pos)
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=STORAGE["c64"])
    t.set_kpoints(w.extra["kfrac"], w.extra["koffs"])
    s = torch.cuda.Stream()
    warm, cold = Stepper(True, s), Stepper(False, s)
    K = args.steps
    Lr = t.info()["Lreal"]
    res = {"workload": "tio2_kpoints: primitive cell 4.35 x 4.35 x 2.8 bohr, grid 18x18x12, "
                       "64 k-points x 6 complex orbitals (15 MB complex64), "
                       f"{E} electrons (256 walkers x 128 moves in the supercell)",
           "table_bytes": t.info()["table_bytes"]}
    with torch.cuda.stream(s):
        dpos = torch.from_numpy(pos).cuda()
        doffs = torch.from_numpy(offs).cuda()
        out = t.alloc_outputs(E)
        ch = t.autotune(dpos, doffs, out=out, stream=s)
        ev = lambda: t.eval(dpos, doffs, out=out, stream=s)
        times = {"warm": statistics.mean(warm.time(ev, K)),
                 "flushed_window_off": statistics.mean(cold.time(ev, K))}
        t.set_l2_residency(1.0)
        times["flushed_window_on"] = statistics.mean(cold.time(ev, K))
        t.set_l2_residency(0.0)
        buf = torch.ones(12 * 1024 * 1024, device="cuda")           # 48 MB
        reps = 50
        pms = statistics.mean(warm.time(lambda: pb.probe_l2_read(buf, reps, stream=s), 5))
    s.synchronize()
    l2_gbs = buf.numel() * 4 * reps / (pms / 1e3) / 1e9
    gather = 64.0 * Lr * 4 * E                  # stencil rows, served by L2 when resident
    outb = 20.0 * Lr * E
    peak, _ = measured_peaks()
    f32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    roof = {"l2": gather / (l2_gbs * 1e9), "hbm": outb / (peak * 1e9),
            "alu": 640.0 * Lr * E / (f32_peak * 1e12)}
    bound = max(roof, key=roof.get)
    for name, ms in times.items():
        res[name] = {"us": 1e3 * ms, "evals_per_s": E * w.n_orb / (ms / 1e3),
                     "l2_GBps": gather / (ms / 1e3) / 1e9, "bound": bound,
                     "frac": roof[bound] / (ms / 1e3)}
    res.update({"kernel": list(ch), "l2_read_probe_GBps": l2_gbs,
                "roof_us": {k: 1e6 * v for k, v in roof.items()}})
    line["l2_resident"] = res
    t.close()


def extras_single_walker(args, pb, w, tab, t, st_, line, sms, stream):
    """The 1,536-electron single walker (uniform positions) on the same FP32
    table: all electrons in one launch (with the access-pattern probe), and
    one electron per launch (a CUDA graph of 1,536 launches)."""
    import torch
    if w.name == "tio2":
        w1, t1 = w, t
    else:
        w1 = bi.workload("tio2")
        t1 = t if t.storage == 0 else pb.BlipTable(w1.grid, w1.lattice, tab, storage=0)
    pos1, _ = w1.positions()
    E = len(pos1)
    K = args.steps
    Lr = t1.info()["Lreal"]
    d1 = torch.from_numpy(pos1).cuda()
    o1 = t1.alloc_outputs(E)
    ch = t1.autotune(d1, out=o1) if args.kernel == "auto" else tuple(
        int(x) for x in args.kernel.split(","))
    U1 = touched_sites(w1.grid, w1.lattice, pos1)
    ms_l = st_.time(lambda: t1.eval(d1, out=o1), K)
    ent = _timed_entry(ms_l, E, Lr, U1, 4, "full", sms, ch)
    ms = statistics.mean(ms_l)
    if not args.no_probe and ch[3] == 0:
        # the access pattern's own time (blip_probe_gather): the evaluation's
        # item walk, FP64 geometry, row loads and output stores without the
        # weights and FMAs (input order: the ceiling of unsorted launches)
        g_ms = statistics.mean(st_.time(lambda: t1.probe_gather(d1, out=o1, store=False), K))
        gs_ms = statistics.mean(st_.time(lambda: t1.probe_gather(d1, out=o1, store=True), K))
        bytes_alg, _ = launch_model("full", E, Lr, U1, 4)
        peak, _ = measured_peaks()
        ent["pattern_ceiling"] = {
            "gather_us": 1e3 * g_ms, "gather_store_us": 1e3 * gs_ms,
            "kernel_frac_of_ceiling": gs_ms / ms,
            "ceiling_frac_of_copy": bytes_alg / (gs_ms / 1e3) / 1e9 / peak}
    # one electron per launch (particle-by-particle order), 1,536 kernel
    # nodes in one CUDA graph
    one_choice = list(ch)
    if args.kernel == "auto":
        one_choice = list(t1.autotune(d1[:1].contiguous(), out=tuple(x[:1] for x in o1)))
    g = t1.graph(d1, o1, 1)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    st_.hold(reps, per_step_s=0.01)
    a.record(stream)
    for _ in range(reps):
        g.launch()
    b.record(stream)
    torch.cuda.synchronize()
    oms = a.elapsed_time(b) / reps
    ent["one_at_a_time"] = {"evals_per_s": E * w1.n_orb / (oms / 1e3), "ms_per_step": oms,
                            "us_per_electron": 1e3 * oms / E,
                            "how": "CUDA graph of 1,536 single-electron launches",
                            "kernel": one_choice}
    g.close()
    ent["workload"] = "tio2: 1 walker, 1,536 uniform positions, FP32"
    line["single_walker"] = ent


if __name__ == "__main__":
    sys.exit(main())
