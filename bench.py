#!/usr/bin/env python
"""Benchmark: orbital x electron evaluations per second (value + gradient +
Laplacian) of the periodic cubic-blip path on GB300.

Default workload: the TiO2-shaped table (tetragonal 17.4 x 17.4 x 11.2 bohr,
72 x 72 x 48 grid, 768 real orbitals, FP32 storage) evaluated at 1,536
uniform positions all at once (one batched launch per step).  A step is one
blip_eval of the batch; L2 is flushed (512 MB write, then 512 MB read so no
dirty lines remain) between steps outside the per-step CUDA-event window.

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
}

STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "c64": 3, "bf16pair": 4}
ELEM_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "c64": 4, "bf16pair": 2}   # per real component


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tio2",
                    choices=["tio2", "tio2_batch", "tio2_precision", "cubic16",
                             "tio2_super_complex", "sm_update"])
    ap.add_argument("--batch", type=int, default=1536, help="electrons per walker (tio2_batch)")
    ap.add_argument("--walkers", type=int, default=0, help="override walker count")
    ap.add_argument("--orbitals", type=int, default=0,
                    help="override the orbital count (smaller profiling cases)")
    ap.add_argument("--storage", default="f32", choices=list(STORAGE))
    ap.add_argument("--kernel", default="auto", help="auto | variant,chunks,warps,sort")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the access-pattern probe and the SGEMM peak")
    ap.add_argument("--warm", action="store_true",
                    help="no L2 flush between steps (tables that fit in L2)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
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


def kernel_hash():
    """SHA-256 (16 hex digits) of the code (comments aside) of every CUDA
    source of the evaluation path (all of the library but the
    Sherman-Morrison update)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1204_1121_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f != "blip_sm.cu":
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
    return {"value": n * reps * Lr / dt, "unit": "orbital*electron evals/s (val+grad+lap)",
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
    # bound each step to about 2 s of wall time
    t0 = time.perf_counter()
    oracle.eval_stencil(w.grid, w.lattice, tab, pos[: min(E, 256)], threads=cores)
    per_e = (time.perf_counter() - t0) / min(E, 256)
    n = int(max(16, min(E, 2.0 / max(per_e, 1e-9))))
    for _ in range(args.warmup):
        oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.eval_stencil(w.grid, w.lattice, tab, pos[:n], threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = n * w.n_orb / (ms / 1e3)
    unit = "orbital*electron evals/s (val+grad+lap)"
    line = {"impl": "reference", "metric": "orbital*electron evals/s (val+grad+lap)",
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
    E = len(pos)
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=STORAGE[args.storage])
    if spectral:                       # the FP64 device copy is no longer needed
        del tab
        tab = None
        torch.cuda.empty_cache()
    info = t.info()
    dpos = torch.from_numpy(pos).cuda()
    doffs = torch.from_numpy(offs).cuda()
    out = t.alloc_outputs(E)
    stream = torch.cuda.current_stream()
    if args.kernel == "auto":
        chosen = t.autotune(dpos, doffs, out=out)
    else:
        v_, c_, w_, s_ = (int(x) for x in args.kernel.split(","))
        t.set_kernel(v_, c_, w_, s_)
        chosen = (v_, c_, w_, s_)
    # L2 flush between steps: write 512 MB, then read another 512 MB so the
    # L2 is left holding clean lines (no write-back charged to the next step)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_rd = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2(k):
        if args.warm:                  # warm L2: the table stays cached between steps
            return None
        flush.fill_(float(k))
        return flush_rd.sum()

    def step():
        t.eval(dpos, doffs, out=out)

    def hold_queue(steps):
        # a device-side wait (torch's spin kernel, 50 ms + 2 ms per step)
        # ahead of timed launches: the host enqueues them all while it runs,
        # so a host stall cannot leave the GPU idle inside a step's CUDA-event
        # window; it runs before the first event, outside every window
        sleep = getattr(torch.cuda, "_sleep", None)
        if sleep is not None:
            sleep(int(2.0e9 * (0.05 + 0.002 * steps)))

    for k in range(max(3, args.warmup)):
        flush_l2(k)
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
    hold_queue(K)
    for k in range(K):
        flush_l2(k)
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

    # roofline of the evaluation kernel (the only kernel in the step)
    U = touched_sites(w.grid, w.lattice, pos)
    Lr = info["Lreal"]
    bytes_alg = U * Lr * ELEM_BYTES[args.storage] + 20 * Lr * E + 24 * E
    peak, peak_kind = measured_peaks()
    kh = kernel_hash()
    rec = NCU_TRAFFIC.get((kh, w.name, args.storage, E), {}).get(tuple(chosen[:2]))
    # FP32 FMA peak from unit counts and clock: SMs x 128 FP32 lanes x 2 FLOP
    # x 2.07 GHz (maximum SM clock)
    sms = info["sm_count"]
    f32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    flops = 640.0 * Lr * E
    t_hbm = bytes_alg / (peak * 1e9)
    t_alu = flops / (f32_peak * 1e12)
    hbm_ach = bytes_alg / (ms / 1e3) / 1e9
    alu_ach = flops / (ms / 1e3) / 1e12
    if t_hbm >= t_alu:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": peak, "unit": "GB/s",
                "frac": hbm_ach / peak, "traffic": rec,
                "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"}
    else:
        roof = {"bound": "alu", "achieved": alu_ach, "peak": f32_peak, "unit": "TFLOP/s",
                "frac": alu_ach / f32_peak, "traffic": rec,
                "peak_kind": f"FP32 FMA: {sms} SMs x 128 lanes x 2 FLOP x 2.07 GHz"}
        if not args.no_probe:
            sg = sgemm_tflops()
            roof["fp32_sgemm_tflops"] = sg
            roof["frac_of_sgemm"] = alu_ach / sg
    roof.update({"algorithmic_bytes_per_launch": bytes_alg, "touched_sites": U,
                 "fp32_flop_per_launch": flops, "kernel_source_hash": kh,
                 "hbm_frac": hbm_ach / peak, "alu_frac": alu_ach / f32_peak,
                 "roof_time_us": 1e6 * max(t_hbm, t_alu),
                 "gather_model_GBps": (E * 64 * Lr * ELEM_BYTES[args.storage] + 20 * Lr * E)
                                      / (ms / 1e3) / 1e9})

    line = {"metric": "orbital*electron evals/s (val+grad+lap)", "value": value,
            "unit": "orbital*electron evals/s", "n_gpus": world, "steps": K,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "ms_median": ms_median,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": describe(w, args, E), "roofline": roof, "clocks": clocks,
            "gpu_launches": K * (6 if chosen[3] else 1), "kernel_choice": list(chosen),
            "status": st,
            "wall_s_timed_region": wall}

    if not args.no_probe and args.storage in ("f32", "c64") and chosen[3] == 0:
        # the access pattern's own time (blip_probe_gather): the evaluation's
        # item walk, FP64 geometry, row loads and output stores without the
        # weights and FMAs, timed like the steps above (the probe walks the
        # batch in input order, so it is the ceiling of unsorted launches)
        def probe_ms(store):
            for k in range(3):
                flush_l2(k)
                t.probe_gather(dpos, out=out, store=store)
            pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(K)]
            hold_queue(K)
            for k in range(K):
                flush_l2(k)
                pe[k][0].record(stream)
                t.probe_gather(dpos, out=out, store=store)
                pe[k][1].record(stream)
            torch.cuda.synchronize()
            return statistics.mean(a.elapsed_time(b) for a, b in pe)
        g_ms, gs_ms = probe_ms(False), probe_ms(True)
        line["pattern_ceiling"] = {
            "gather_us": 1e3 * g_ms, "gather_store_us": 1e3 * gs_ms, "kernel_us": 1e3 * ms,
            "kernel_frac_of_ceiling": gs_ms / ms,
            "ceiling_frac_of_copy": bytes_alg / (gs_ms / 1e3) / 1e9 / peak,
            "what": "blip_probe_gather on the same positions (input order): geometry, the 64 row "
                    "loads per item and (gather_store) the output stores, without the arithmetic"}

    if not args.no_e2e:
        # end to end through the host-buffer entry point: H2D positions,
        # evaluation, D2H of all outputs, per step
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
        line["e2e"] = {"value": world * evals / (e_ms / 1e3), "unit": "orbital*electron evals/s",
                       "h2d_bytes_per_step": int(hp.numel() * 8 + ho.numel() * 4),
                       "d2h_bytes_per_step": int((hv.numel() + hg.numel() + hl.numel()) * 4),
                       "ms_per_step": e_ms,
                       "api": "blip_eval_host with page-locked host buffers (the kernel reads the "
                              "positions and writes the outputs across the host link)"}

    if not args.no_extra and args.workload == "tio2" and rank == 0:
        # one electron per launch (particle-by-particle order), 1,536 kernel
        # nodes in one CUDA graph
        o1 = t.alloc_outputs(E)
        one_choice = list(chosen)
        if args.kernel == "auto":      # tune the one-electron launch too
            one_choice = list(t.autotune(dpos[:1].contiguous(), out=tuple(x[:1] for x in o1)))
        g = t.graph(dpos, o1, 1)
        for _ in range(2):
            g.launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        hold_queue(reps)
        a.record(stream)
        for _ in range(reps):
            g.launch()
        b.record(stream)
        torch.cuda.synchronize()
        oms = a.elapsed_time(b) / reps
        line["one_at_a_time"] = {"value": evals / (oms / 1e3), "ms_per_step": oms,
                                 "us_per_electron": 1e3 * oms / E,
                                 "how": "CUDA graph of 1,536 single-electron launches",
                                 "kernel_choice": one_choice}
        g.close()

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


if __name__ == "__main__":
    sys.exit(main())
