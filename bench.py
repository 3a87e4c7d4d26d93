#!/usr/bin/env python
"""Benchmark of the tracer-advection hot path on GB300.

Workload (one bench "step" = one tracker_advance call = the whole hot path:
cell split, block keys, re-binning (counting sort), stencil gather + separable
contraction, fused RK2 update, re-binned after every RK2 step):

    256^3 float32 velocity field (divergence-free random Fourier modes,
    |k| <= 85, E(k) ~ k^-5/3), 2^20 uniform tracers with float64 positions,
    spline kernel I = 6 (m = 2), 100 RK2 steps of dt = 5e-3.

Metric: particle-steps/s (particles x RK2 steps per second), whole job.
Multi-GPU: replicas (each rank advances its own tracer set in its own copy of
the field; no data-path collective), weak scaling.

``--impl reference`` times the FP64 CPU oracle on the host cores on the same
workload (bounded particle sample per step); it is the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, KMAX, NP, I, M, DT, INNER = 256, 85, 1 << 20, 6, 2, 5e-3, 100
SEED_FIELD, SEED_POS = 1001, 2
WORKLOAD = (f"{N}^3 fp32 velocity |k|<={KMAX}, 2^20 uniform tracers (fp64 positions), spline I={I} m={M}, "
            f"{INNER} RK2 steps dt={DT}, re-binned every step")
METRIC, UNIT = "particle-steps/s", "particle-steps/s"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--inner", type=int, default=INNER, help="RK2 steps per bench step (workload: 100)")
    ap.add_argument("--no-variants", action="store_true", help="skip the float64 and split-bf16 forms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "block", "column", "direct"],
                    help="step kernel of the headline workload (default: auto, the tracker's timed choice)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (precision, batching, differentiation, small, sparse)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5, 6, 7],
                    help="2: the headline workload (default); 1 small, 3 precision, 4 batching, 5 adjoint, "
                         "6 the paper's sparse tracer density, 7 the step tuner's table against density")
    ap.add_argument("--sparse-n", type=int, default=1024, help="grid of config 6 (1.5e-3 tracers per cell)")
    ap.add_argument("--direct-block", type=int, default=0,
                    help="with --step-kernel direct: the binning block edge of the direct path (0: default)")
    ap.add_argument("--halo-copy", default="auto", choices=["auto", "async", "tma"],
                    help="the block kernel's halo staging (config 3; default: the tracker's choice)")
    ap.add_argument("--c3-n", type=int, default=1024, help="grid of config 3 (smaller grids for profiling)")
    ap.add_argument("--c3-np-log2", type=int, default=27, help="log2 of the tracer count of config 3")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device):
    """The largest x over the ranks of the initialised process group (x itself
    without one); device: where the collective's tensor lives (cuda for nccl,
    cpu for gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ws, ms):
    """Whole-job throughput: every rank's units (replicas: the same count on
    each rank) over the slowest rank's time in milliseconds."""
    return units_per_rank * ws / (ms * 1e-3)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def field_and_particles(with_f64=False):
    """The headline workload's float32 field and tracers (and the float64 field
    the float32 one was rounded from, for the error against the truth)."""
    import numpy as np

    import synth

    f64 = synth.velocity_field_np(N, KMAX, SEED_FIELD)
    field = f64.astype(np.float32)
    pos = synth.uniform_particles_np(NP, SEED_POS)
    return (field, pos, f64) if with_f64 else (field, pos)


STEP_KERNELS = {"column": ("k_column<6,5,RK2> (float32 field)", "k_column_rk2_f32_i6",
                            ("column_kernel.cuh", "column_i6.cu", "block_kernel.cuh", "internal.cuh", "coeffs.inc")),
                "block": ("k_block<float,6,5,RK2,F32>", "k_block_rk2_f32_i6",
                          ("block_kernel.cuh", "block_i6.cu", "internal.cuh", "coeffs.inc")),
                "direct": ("k_direct<float,6,5,RK2,F32>", "k_direct_rk2_f32_i6",
                           ("block_kernel.cuh", "direct_i6.cu", "internal.cuh", "coeffs.inc"))}


def kernel_source_sha(kind="column"):
    """Hash of the sources of the step kernel the headline workload runs."""
    h = hashlib.sha256()
    for f in STEP_KERNELS[kind][2]:
        with open(os.path.join(ROOT, "paper_2107_01104_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_record(sha, kind="column"):
    """The committed ncu summary of the step kernel (profiles/traffic.json), if it matches the source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(STEP_KERNELS[kind][1])
    if not e or e.get("source_sha") != sha:
        return {}
    return e


def ncu_traffic(sha, kind="column"):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it matches the source."""
    return ncu_record(sha, kind).get("dram_bytes_per_launch")


def sync_flags(tr, trk, notes):
    """Wait for the tracker; a CFL flag (a particle moved more than one cell in
    one stage, computed exactly through the slow path) is recorded, not fatal."""
    try:
        tr.sync()
    except trk.TrackerError as e:
        if e.status != trk.TRK_ECFL:
            raise
        notes["cfl_slow_path_used"] = True


def oracle_cost(f64, pos):
    """Seconds per particle-step of the oracle on this host (calibrated on a
    sample large enough that its fixed per-call cost does not dominate)."""
    import oracle

    n = 256
    while True:
        t0 = time.perf_counter()
        oracle.advance(f64, pos[:, :n], DT, 2, oracle.SPLINE, I, M)
        el = time.perf_counter() - t0
        if el > 0.5 or n >= NP:
            return el / (n * 2)
        n = min(NP, n * 8)


def cpu_baseline(field, pos, seconds):
    """The oracle as it stands, on this host's cores, on a bounded particle sample."""
    import numpy as np

    import oracle

    f64 = field.astype(np.float64)
    cal = oracle_cost(f64, pos)
    n = int(max(512, min(NP, seconds / max(cal, 1e-9) / INNER)))
    t0 = time.perf_counter()
    oracle.advance(f64, pos[:, :n], DT, INNER, oracle.SPLINE, I, M)
    el = time.perf_counter() - t0
    return {"value": n * INNER / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} of the {NP} tracers x {INNER} RK2 steps ({el:.1f} s)"}


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle

    oracle.build()
    field, pos = field_and_particles()
    f64 = field.astype(np.float64)
    # bounded sample per step, sized so the whole run stays within a few minutes
    cal = oracle_cost(f64, pos)
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    n = int(max(256, min(NP, per_step_s / max(cal, 1e-9) / args.inner)))
    p = pos[:, :n].copy()
    for _ in range(args.warmup):
        p = oracle.advance(f64, p, DT, args.inner, oracle.SPLINE, I, M)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p = oracle.advance(f64, p, DT, args.inner, oracle.SPLINE, I, M)
    el = time.perf_counter() - t0
    value = n * args.inner * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_particles": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{n} tracers x {args.inner} RK2 steps per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GB300 arm: timing helpers
# --------------------------------------------------------------------------
def _events():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def timed(fn, stream, dev_index, min_s=0.5, max_reps=50, min_reps=3):
    """ms per call of fn, timed with CUDA events on `stream` over enough calls to
    last about min_s (sized from one untimed call), with the SM clocks sampled
    by nvidia-smi during the timed calls: (ms, reps, clocks)."""
    import torch

    e0, e1 = _events()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    one = max(e0.elapsed_time(e1), 1e-3)
    reps = int(min(max_reps, max(min_reps, math.ceil(min_s * 1e3 / one))))
    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.15)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, reps, clocks.stop()


def profiled(tr, trk, fn, reps=1):
    """Device time per call of each kernel class of tracker tr over `reps`
    calls of fn (event-bracketed launches; the tracker replays no CUDA graph
    while it records): {'step'|'bin'|'other': (ms per call, launches per call)}."""
    import torch

    torch.cuda.synchronize()
    trk.tracker_profile(tr.h, True)
    for _ in range(reps):
        fn()
    prof = trk.tracker_profile_read(tr.h)
    trk.tracker_profile(tr.h, False)
    return {k: (v[0] / reps, v[1] / reps) for k, v in prof.items()}


def hbm_roofline(alg_bytes, kernel_ms, label, alg_def, **extra):
    """HBM roofline of one kernel launch (or one call's kernels): algorithmic
    bytes over device time against the measured copy bandwidth."""
    peak, kind = measured_peaks()
    ach = alg_bytes / (kernel_ms * 1e-3) / 1e9
    d = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "kernel": label,
         "alg_bytes": alg_bytes, "kernel_ms": kernel_ms, "alg_def": alg_def, "peak_kind": kind}
    d.update(extra)
    return d


def fma_bound(fmas, kernel_ms, fma_per_s, what):
    """FMA-bound fraction: the contraction's FMAs over device time against the probed FMA rate."""
    ach = fmas / (kernel_ms * 1e-3)
    return {"achieved_fma_per_s": ach, "peak_fma_per_s": fma_per_s, "frac": ach / fma_per_s,
            "fmas": fmas, "peak_def": f"tracker_probe_fma ({what}) on this GPU, same run"}


def kernel_name(trk, tr):
    return {trk.TRK_STEP_BLOCK: "block", trk.TRK_STEP_COLUMN: "column",
            trk.TRK_STEP_DIRECT: "direct"}.get(tr.last_step_kernel(), "?")


def interp_error(trk, tr, field64, pos_sample, I_, M_, family=None):
    """Interpolated u at a tracer sample against the oracle on the float64
    field (the truth): max and rms error over the field rms."""
    import numpy as np
    import torch

    import oracle

    family = trk.TRK_SPLINE if family is None else family
    p = torch.from_numpy(np.ascontiguousarray(pos_sample)).cuda()
    got = tr.interpolate(p, out_dtype=torch.float64).cpu().numpy()
    ref = oracle.interp(field64, pos_sample, family, I_, M_)
    rms = float(np.sqrt(np.mean(field64 ** 2)))
    d = got - ref
    return {"max_err_over_rms": float(np.abs(d).max()) / rms, "rms_err_over_rms": float(np.sqrt(np.mean(d ** 2))) / rms,
            "vs": "oracle on the float64 field", "sample": int(pos_sample.shape[1])}


FMA_RK2_I6 = 2 * 3 * (I ** 3 + I ** 2 + I)    # separable contraction, two stages, three components


# --------------------------------------------------------------------------
# GB300 arm: the headline workload
# --------------------------------------------------------------------------
def run_gb300(args):
    import numpy as np
    import torch

    import paper_2107_01104_gb300 as trk
    from paper_2107_01104_gb300 import build as lib_build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    dev_index = torch.cuda.current_device()
    if rank == 0:
        lib_build.build()
    if ws > 1:
        dist.barrier()
    trk.load_library()

    field, pos, field64 = field_and_particles(with_f64=True)
    tr = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
    tr.set_step_kernel({"auto": trk.TRK_STEP_AUTO, "block": trk.TRK_STEP_BLOCK,
                        "column": trk.TRK_STEP_COLUMN, "direct": trk.TRK_STEP_DIRECT}[args.step_kernel])
    if args.step_kernel == "direct" and args.direct_block:
        tr.set_tuning(step_kernel=trk.TRK_STEP_DIRECT, direct_block=args.direct_block)
    tr.set_field(torch.from_numpy(field).to(dev))
    p = torch.from_numpy(pos).to(dev)
    stream = torch.cuda.current_stream()

    def barrier_sync():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    notes = {"cfl_slow_path_used": False}
    for _ in range(args.warmup):
        tr.advance(p, DT, args.inner, trk.TRK_RK2)
    sync_flags(tr, trk, notes)
    notes["tuning"] = tr.tuning()     # the launch shape the tuner chose in the first warm-up call

    # ---------------- device-timed region (the step pairs replay from CUDA graphs) ----------------
    clocks = ClockSampler(dev_index)
    barrier_sync()
    clocks.start()
    time.sleep(0.2)
    launches0 = tr.launch_count
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(args.steps):
        tr.advance(p, DT, args.inner, trk.TRK_RK2)
    e1.record(stream)
    barrier_sync()
    clk = clocks.stop()
    launches = tr.launch_count - launches0
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dev)
    sync_flags(tr, trk, notes)
    value = job_value(NP * args.inner * args.steps, ws, ms)

    # ---------------- per-kernel times: a separate, profiled pass ----------------
    psteps = max(1, min(args.steps, 3))
    barrier_sync()
    prof = profiled(tr, trk, lambda: tr.advance(p, DT, args.inner, trk.TRK_RK2), reps=psteps)
    sync_flags(tr, trk, notes)

    # ---------------- roofline of the step kernel ----------------
    step_ms, step_n = prof["step"]
    avg_launch_s = step_ms * 1e-3 / max(step_n, 1)
    field_bytes = 3 * N ** 3 * 4
    alg_bytes = field_bytes + 52 * NP                 # field once + fp64 positions read and written + key
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    kind = kernel_name(trk, tr)
    kernel_label = STEP_KERNELS[kind][0]
    if kind == "direct":   # node loads through the texture object (most of the rows) or plain loads
        notes["direct_node_loads"] = "texture" if tr.field_texture() else "plain"
        kernel_label = kernel_label[:-1] + (",NM_TEX4>" if tr.field_texture() else ",NM_VEC4>")
    sha = kernel_source_sha(kind)
    gather_bytes = NP * 2 * I ** 3 * 3 * 4            # two stencil gathers per RK2 step, float32
    sm_mhz = clk.get("sm_mhz") or 1900.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    smem_peak = nsm * 128 * sm_mhz * 1e6 / 1e9
    fma32 = trk.tracker_probe_fma(trk.TRK_DTYPE_F32)
    fma64 = trk.tracker_probe_fma(trk.TRK_DTYPE_F64)

    # ---------------- error of the timed form against the oracle ----------------
    rng = np.random.default_rng(0)
    sample = rng.choice(NP, 4096, replace=False)
    error = interp_error(trk, tr, field64, pos[:, sample], I, M)
    import oracle

    few = sample[:256]
    q = torch.from_numpy(np.ascontiguousarray(pos[:, few])).to(dev)
    tr.advance(q, DT, args.inner, trk.TRK_RK2)
    ref = oracle.advance(field.astype(np.float64), pos[:, few], DT, args.inner, oracle.SPLINE, I, M)
    error["positions_after_one_step_call"] = {
        "max_abs_err": float(np.abs(q.cpu().numpy() - ref).max()), "rk2_steps": args.inner, "sample": len(few),
        "vs": "oracle on the stored float32 values (same input)", "cell_width": 2 * math.pi / N}
    sync_flags(tr, trk, notes)

    # ---------------- end-to-end through the public API ----------------
    host = torch.from_numpy(pos).pin_memory()
    back = torch.empty_like(host).pin_memory()
    barrier_sync()
    w0, w1 = _events()
    w0.record(stream)
    for _ in range(args.steps):
        p.copy_(host, non_blocking=True)
        tr.advance(p, DT, args.inner, trk.TRK_RK2)
        back.copy_(p, non_blocking=True)
    w1.record(stream)
    barrier_sync()
    e2e_ms = w0.elapsed_time(w1)
    e2e_ms = max_over_ranks(e2e_ms, dev)
    e2e = {"value": job_value(NP * args.inner * args.steps, ws, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": host.numel() * 8,
           "d2h_bytes_per_step": back.numel() * 8}

    # ---------------- other forms of the same workload ----------------
    variants = {}
    if not args.no_variants:
        variants.update(precision_variants(trk, dev, stream, dev_index, field, field64, pos, sample, fma64, args))
        variants.update(ab_variants(trk, tr, dev, stream, dev_index, pos, args))
    tr.close()
    del p, host, back
    torch.cuda.empty_cache()

    configs = {}
    if not args.no_configs and ws == 1:
        for name, fn in (("1_small_plain", config1_block), ("3_precision", config3_block),
                         ("4_batching", config4_block), ("5_differentiation", config5_block),
                         ("6_sparse_paper_density", config6_block)):
            configs[name] = fn(trk, dev, stream, dev_index, args, {"fp32": fma32, "fp64": fma64})
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(field, pos, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "np": NP, "kernel": f"spline I={I} m={M}", "scheme": "RK2",
                       "dt": DT, "rk2_steps_per_bench_step": args.inner, "field_storage": "f32",
                       "positions": "f64", "l2": "inputs larger than L2 (201 MB field vs 129 MB L2)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": ncu_traffic(sha, kind), "kernel": kernel_label,
                         "l2_hit_rate": ncu_record(sha, kind).get("l2_hit_rate"),
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                         "launches_timed": step_n, "peak_kind": peak_kind, "source_sha": sha},
            "fma_roofline": {**fma_bound(NP * FMA_RK2_I6, avg_launch_s * 1e3, fma32, "float32"),
                             "fma_per_particle_step": FMA_RK2_I6},
            "smem_roofline": {"achieved": gather_bytes / avg_launch_s / 1e9, "peak": smem_peak, "unit": "GB/s",
                              "frac": gather_bytes / avg_launch_s / 1e9 / smem_peak,
                              "gather_bytes_per_launch": gather_bytes,
                              "path": "shared memory" if kind != "direct" else
                              ("L1 (gathers: texture and load/store data paths)" if notes.get("direct_node_loads") ==
                               "texture" else "L1 (global gathers)"),
                              "peak_def": "SMs x 128 B/clk (the L1 / shared-memory data path) x median SM clock under load"},
            "phase_ms_per_step": {"step_kernel": step_ms / args.inner, "binning": prof["bin"][0] / args.inner,
                                  "other": prof["other"][0] / args.inner, "profiled_calls": psteps,
                                  "note": "event-bracketed launches without graph replay"},
            "error": error,
            "fma_peaks_probed": {"fp32_fma_per_s": fma32, "fp64_fma_per_s": fma64,
                                 "fp64_fma_per_clk_per_sm": fma64 / (nsm * sm_mhz * 1e6),
                                 "fp32_fma_per_clk_per_sm": fma32 / (nsm * sm_mhz * 1e6)},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "variants": variants, "configs": configs,
            "notes": notes, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def precision_variants(trk, dev, stream, dev_index, field, field64, pos, sample, fma64, args):
    """The headline workload with the field stored as float64 (the paper's
    plain form) and as split-bf16 pairs: rate, HBM roofline of the step kernel,
    FMA-bound fraction (float64), error against the oracle, clocks."""
    import torch

    out = {}
    for name, storage, inner, esz in (("f64", trk.TRK_F64, 10, 8), ("bf16x2", trk.TRK_BF16X2, args.inner, 4)):
        tv = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=M, storage=storage)
        tv.set_field(torch.from_numpy(field64 if storage == trk.TRK_F64 else field).to(dev))
        pv = torch.from_numpy(pos).to(dev)
        for _ in range(3):
            tv.advance(pv, DT, inner, trk.TRK_RK2)
        ms, reps, clk = timed(lambda: tv.advance(pv, DT, inner, trk.TRK_RK2), stream, dev_index, min_s=0.8)
        prof = profiled(tv, trk, lambda: tv.advance(pv, DT, inner, trk.TRK_RK2))
        kms = prof["step"][0] / inner
        alg = 3 * N ** 3 * esz + 52 * NP
        d = {"value": NP * inner / (ms * 1e-3), "unit": UNIT, "rk2_steps_per_call": inner, "calls_timed": reps,
             "kernel": kernel_name(trk, tv), "step_kernel_ms": kms, "binning_ms": prof["bin"][0] / inner,
             "roofline": hbm_roofline(alg, kms, kernel_name(trk, tv), f"field 3 N^3 x {esz} B + 52 B per particle-step"),
             "error": interp_error(trk, tv, field64, pos[:, sample], I, M), "clocks": clk}
        if storage == trk.TRK_F64:
            d["fma_roofline"] = {**fma_bound(NP * FMA_RK2_I6, kms, fma64, "float64"),
                                 "fma_per_particle_step": FMA_RK2_I6}
        out[name] = d
        tv.close()
        del pv
        torch.cuda.empty_cache()
    return out


def ab_variants(trk, tr, dev, stream, dev_index, pos, args):
    """Adams-Bashforth of orders 2 and 4 (one field evaluation per step) on the
    headline tracker, history full when the timed calls start."""
    import torch

    out = {}
    for name, scheme in (("ab2", trk.TRK_AB2), ("ab4", trk.TRK_AB4)):
        k = scheme + 1
        pv = torch.from_numpy(pos).to(dev)
        hist = torch.zeros((k - 1, 3, NP), dtype=torch.float32, device=dev)
        tr.advance(pv, DT, k - 1, scheme, rhs=hist, history_valid=0)
        call = lambda: tr.advance(pv, DT, args.inner, scheme, rhs=hist, history_valid=k - 1)  # noqa: E731
        call()
        ms, reps, clk = timed(call, stream, dev_index, min_s=0.8)
        prof = profiled(tr, trk, call)
        kms = prof["step"][0] / args.inner
        alg = 3 * N ** 3 * 4 + NP * (52 + 24 * (k - 1))
        out[name] = {"value": NP * args.inner / (ms * 1e-3), "unit": UNIT, "ab_steps_per_call": args.inner,
                     "calls_timed": reps, "field_storage": "f32", "kernel": kernel_name(trk, tr),
                     "step_kernel_ms": kms, "binning_ms": prof["bin"][0] / args.inner,
                     "roofline": hbm_roofline(alg, kms, kernel_name(trk, tr),
                                              f"field once + 52 B + {24 * (k - 1)} B history per particle-step"),
                     "clocks": clk}
        del pv, hist
    return out


# --------------------------------------------------------------------------
# the other configurations (single GPU)
# --------------------------------------------------------------------------
def config1_block(trk, dev, stream, dev_index, args, fma):
    """32^3 float64 field |k| <= 8, 1e4 tracers, Lagrange I=4: interpolation and
    one RK2 step dt=1e-3 per call (launch-bound small case), against the oracle."""
    import numpy as np
    import torch

    import oracle
    import synth

    field = synth.velocity_field_np(32, 8, 1000)
    pos = synth.uniform_particles_np(10_000, 1)
    t = trk.Tracker(32, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F64)
    t.set_field(torch.from_numpy(field).to(dev))
    p0 = torch.from_numpy(pos).to(dev)
    u = t.interpolate(p0, out_dtype=torch.float64)
    p1 = p0.clone()
    t.advance(p1, 1e-3, 1)
    t.sync()
    err_u = float(np.abs(u.cpu().numpy() - oracle.interp(field, pos, oracle.LAGRANGE, 4, 0)).max())
    err_x = float(np.abs(p1.cpu().numpy() - oracle.advance(field, pos, 1e-3, 1, oracle.LAGRANGE, 4, 0)).max())
    p = p0.clone()

    def call():
        t.interpolate(p, out_dtype=torch.float64)
        t.advance(p, 1e-3, 1)

    ms, reps, clk = timed(call, stream, dev_index, min_s=0.3, max_reps=200)
    t.close()
    return {"metric": "particle-steps/s", "value": 10_000 / (ms * 1e-3), "unit": "particle-steps/s",
            "ms_per_call": ms, "calls_timed": reps, "dtype": "f64",
            "workload": "32^3 f64 velocity |k|<=8, 1e4 tracers, Lagrange I=4, interpolate + one RK2 step dt=1e-3",
            "error": {"u_max_abs": err_u, "x_max_abs": err_x, "vs": "oracle, same float64 field",
                      "bar": "1e-12 x max|u| (u), 1e-13 (positions)"},
            "roofline": None, "note": "launch-bound (a few kernels for 1e4 tracers): no roofline", "clocks": clk}


def config3_block(trk, dev, stream, dev_index, args, fma):
    """1024^3, u (3) + grad u (9, spectral), float32 and split bf16 storage,
    2^27 tracers, spline I = 8: interpolation rate, HBM roofline of the
    interpolation kernel, FMA-bound fraction, error against the oracle on a
    1e5-tracer subsample (the float64 field is made one component at a time
    on the GPU and only the subsample's stencil nodes are gathered)."""
    import numpy as np
    import torch

    import oracle
    import synth

    N3, NPART, I8, M8 = args.c3_n, 1 << args.c3_np_log2, 8, 3
    KM, NSUB = N3 // 3, min(100_000, NPART)
    pos = synth.uniform_particles_torch(NPART, 3, device=dev)
    sub = pos[:, :NSUB].cpu().numpy()
    cell, frac = oracle.split(sub, N3)
    rel = np.arange(1 - I8 // 2, I8 // 2 + 1)
    c1 = (cell[0][:, None] + rel[None, :]) % N3
    c2 = (cell[1][:, None] + rel[None, :]) % N3
    c3 = (cell[2][:, None] + rel[None, :]) % N3
    idx = ((c3[:, :, None, None] * N3 + c2[:, None, :, None]) * N3 + c1[:, None, None, :]).reshape(NSUB, -1)
    idx_t = torch.from_numpy(idx).to(dev)
    f12 = torch.empty((12, N3, N3, N3), dtype=torch.float32, device=dev)
    truth = np.empty((12, NSUB))
    rms = np.empty(12)
    t0 = time.perf_counter()
    for i, comp in enumerate(synth.velocity_components_torch(N3, KM, 1002, device=dev)):
        f12[i] = comp.to(torch.float32)
        rms[i] = float(torch.sqrt(torch.mean(comp * comp)))
        st = comp.reshape(-1)[idx_t].cpu().numpy()
        del comp
        truth[i] = oracle.interp_stencil(frac, st.reshape(NSUB, 1, I8, I8, I8), oracle.SPLINE, I8, M8)[0]
    prep_s = time.perf_counter() - t0
    del idx_t
    torch.cuda.empty_cache()
    rms_u, rms_g = float(np.sqrt(np.mean(rms[:3] ** 2))), float(np.sqrt(np.mean(rms[3:] ** 2)))
    out = {"workload": f"{N3}^3 u (3) + grad u (9, spectral), |k|<={KM}, 2^{args.c3_np_log2} uniform tracers "
                       f"(fp64 positions), spline I=8 m=3, interpolation; error vs the fp64 oracle on {NSUB} tracers",
           "metric": "particles/s", "unit": "particles/s", "prep_s": prep_s}
    for sname, storage in (("f32", trk.TRK_F32), ("bf16x2", trk.TRK_BF16X2)):
        for C in (3, 12):
            t = trk.Tracker(N3, family=trk.TRK_SPLINE, I=I8, m=M8, storage=storage)
            t.set_halo_copy({"auto": trk.TRK_HALO_AUTO, "async": trk.TRK_HALO_ASYNC,
                             "tma": trk.TRK_HALO_TMA}[args.halo_copy])
            t.set_field(f12[:C])
            o = torch.empty((C, NPART), dtype=torch.float32, device=dev)
            call = lambda: t.interpolate(pos, out=o)  # noqa: E731
            call()                                    # AUTO: times the block and the direct kernel once
            ms, reps, clk = timed(call, stream, dev_index, min_s=0.6, max_reps=10)
            prof = profiled(t, trk, call)
            kms = prof["step"][0]
            err = o[:, :NSUB].double().cpu().numpy() - truth[:C]
            alg = C * N3 ** 3 * 4 + NPART * (24 + 4 * C)
            fmas = NPART * C * (I8 ** 3 + I8 ** 2 + I8)
            key = f"{sname}_{'u' if C == 3 else 'u+grad'}"
            kname = kernel_name(trk, t)
            out[key] = {"value": NPART / (ms * 1e-3), "ms_per_call": ms, "calls_timed": reps, "kernel": kname,
                        "kernel_ms": kms, "binning_ms": prof["bin"][0], "other_ms": prof["other"][0],
                        "roofline": hbm_roofline(alg, kms, kname, f"field {C} N^3 x 4 B + (24 + 4 C) B per particle"),
                        "fma_roofline": fma_bound(fmas, kms, fma["fp32"], "float32"),
                        "error": {"u_rms_err_over_rms": float(np.sqrt(np.mean(err[:3] ** 2))) / rms_u,
                                  "u_max_err_over_rms": float(np.abs(err[:3]).max()) / rms_u,
                                  "vs": "oracle on the float64 field", "sample": NSUB},
                        "clocks": clk}
            if C == 12:
                out[key]["error"]["grad_rms_err_over_rms"] = float(np.sqrt(np.mean(err[3:] ** 2))) / rms_g
                out[key]["error"]["grad_max_err_over_rms"] = float(np.abs(err[3:]).max()) / rms_g
            t.close()
            del o
            torch.cuda.empty_cache()
    del f12, pos
    torch.cuda.empty_cache()
    out["value"] = out["f32_u"]["value"]
    return out


def config4_block(trk, dev, stream, dev_index, args, fma):
    """512^3 float32 u, 8 sets 1e3 .. 2e7 tracers, I cycling 4/6/8, 3 or 9
    outputs, 50 AB2 steps per call, one persistent launch per step."""
    import numpy as np
    import torch

    import oracle
    import synth

    N4, dt, steps = 512, 2e-3, 50
    u = synth.velocity_field_torch(N4, 170, 1003, out_dtype=torch.float32)
    t = trk.Tracker(N4, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(u)
    sizes = [1000, 10_000, 30_000, 100_000, 1_000_000, 3_000_000, 10_000_000, 20_000_000]
    pos0, sets = [], []
    for s, n in enumerate(sizes):
        I_ = (4, 6, 8)[s % 3]
        p0 = synth.uniform_particles_torch(n, 10 + s, device=dev)
        pos0.append(p0)
        sets.append(dict(pos=p0.clone(), rhs=torch.zeros((3, n), dtype=torch.float32, device=dev),
                         out=torch.zeros((9 if s % 2 else 3, n), dtype=torch.float32, device=dev),
                         family=trk.TRK_SPLINE, I=I_, m=I_ // 2 - 1, deriv=s % 2))
    total = sum(sizes)
    # error: one 50-step call from the initial positions, 16 tracers per set against the oracle
    t.advance_batched(sets, dt, steps, history_valid=False)
    try:
        t.sync()
    except trk.TrackerError as e:
        if e.status != trk.TRK_ECFL:
            raise
    fs = u.double().cpu().numpy()
    del u
    rng = np.random.default_rng(0)
    errs = []
    for s, S in enumerate(sets):
        ix = rng.choice(sizes[s], 16, replace=False)
        x0 = pos0[s][:, ix].cpu().numpy()
        ref, _ = oracle.advance(fs, x0, dt, steps, S["family"], S["I"], S["m"], scheme=oracle.AB2)
        errs.append(float(np.abs(S["pos"][:, ix].cpu().numpy() - ref).max()))
    del fs
    call = lambda: t.advance_batched(sets, dt, steps, history_valid=True)  # noqa: E731
    l0 = t.launch_count
    ms, reps, clk = timed(call, stream, dev_index, min_s=1.0, max_reps=5)
    launches = (t.launch_count - l0) / (reps + 1)
    prof = profiled(t, trk, call)
    kms = prof["step"][0] / steps
    outs = sum(n * (9 if s % 2 else 3) * 4 for s, n in enumerate(sizes))
    alg = 3 * N4 ** 3 * 4 + total * 72 + outs
    t.close()
    del sets, pos0
    return {"metric": "particle-steps/s", "value": total * steps / (ms * 1e-3), "unit": "particle-steps/s",
            "ms_per_call": ms, "calls_timed": reps, "gpu_launches_per_call": launches,
            "workload": "512^3 fp32 u |k|<=170, 8 sets (1e3..2e7, sum 3.414e7), I cycling 4/6/8, 3- or 9-component "
                        "outputs, 50 AB2 steps per call, one persistent launch per step under a CUDA graph",
            "step_kernel_ms": kms, "binning_ms_per_step": prof["bin"][0] / steps,
            "roofline": hbm_roofline(alg, kms, "k_batched", "u field once (3 N^3 x 4 B) + 72 B per particle "
                                     "(positions r/w 48, AB2 history r/w 24) + 4 B per output value, per step"),
            "error": {"max_abs_pos_err_per_set": errs, "steps": steps, "sample_per_set": 16,
                      "vs": "oracle AB2 on the stored float32 values (same input)"},
            "clocks": clk}


def config5_block(trk, dev, stream, dev_index, args, fma):
    """256^3 float32 u, 2^22 tracers, spline I=6, 20 RK2 steps, loss sum |X_T|^2,
    backward by the discrete adjoint with checkpoints every 5 steps: forward
    and backward rates, each with the HBM roofline of its whole phase, and the
    position gradient of a tracer sample against the oracle."""
    import numpy as np
    import torch

    import oracle
    import synth

    N5, n, dt, steps = 256, 1 << 22, 5e-3, 20
    field = synth.velocity_field_np(N5, 85, 1004).astype(np.float32)
    t = trk.Tracker(N5, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).to(dev))
    p0 = synth.uniform_particles_torch(n, 5, device=dev)
    gf = torch.zeros((3, N5, N5, N5), dtype=torch.float64, device=dev)
    x = p0.clone()
    lam = torch.empty_like(p0)

    def fwd():
        x.copy_(p0)
        t.advance(x, dt, steps)

    def bwd():
        t.adjoint(p0, lam, dt, steps, 5, grad_field=gf)

    fwd()
    torch.mul(x, 2.0, out=lam)
    gpos, _ = t.adjoint(p0, lam, dt, steps, 5, grad_field=gf)
    try:
        t.sync()
    except trk.TrackerError as e:
        if e.status != trk.TRK_ECFL:
            raise
    ix = np.random.default_rng(0).choice(n, 256, replace=False)
    ps = p0[:, ix].cpu().numpy()
    fs = field.astype(np.float64)
    posT = oracle.advance(fs, ps, dt, steps, oracle.SPLINE, 6, 2)
    gref, _ = oracle.adjoint_rk2(fs, ps, 2 * posT, dt, steps, oracle.SPLINE, 6, 2, with_field=False)
    g = gpos.cpu().numpy()[:, ix]
    rel_err = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
    fms, freps, fclk = timed(fwd, stream, dev_index, min_s=0.6, max_reps=20)
    bms, breps, bclk = timed(bwd, stream, dev_index, min_s=1.0, max_reps=10)
    field_b = 3 * N5 ** 3 * 4
    K = 5
    nseg = (steps + K - 1) // K
    # forward: one field sweep + 52 B per particle per step
    f_alg = steps * (field_b + 52 * n)
    # backward: the recomputed forward steps ((nseg - 1) K to lay the checkpoints, then
    # steps - nseg inside the segments) and, per step, the adjoint sweep: field once,
    # X (24 B), lambda in and out (48 B), and the float64 field gradient read and written
    recomputed = (nseg - 1) * K + (steps - nseg)
    b_alg = recomputed * (field_b + 52 * n) + steps * (field_b + 72 * n + 2 * 3 * N5 ** 3 * 8)
    t.close()
    return {"metric": "particle-steps/s", "value": n * steps / ((fms + bms) * 1e-3), "unit": "particle-steps/s",
            "workload": "256^3 fp32 u |k|<=85, 2^22 tracers, spline I=6 m=2, 20 RK2 steps, loss sum |X_T|^2, "
                        "backward by the discrete adjoint with checkpoints every 5 steps",
            "forward": {"ms": fms, "calls_timed": freps, "particle_steps_per_s": n * steps / (fms * 1e-3),
                        "roofline": hbm_roofline(f_alg, fms, "forward call (all kernels)",
                                                 "per step: field once + 52 B per particle"),
                        "clocks": fclk},
            "backward": {"ms": bms, "calls_timed": breps, "particle_steps_per_s": n * steps / (bms * 1e-3),
                         "roofline": hbm_roofline(b_alg, bms, "backward call (all kernels)",
                                                  "recomputed forward steps + per step: field once, 72 B per particle, "
                                                  "float64 field gradient read and written"),
                         "clocks": bclk},
            "error": {"grad_pos_rel_err": rel_err, "sample": len(ix), "bar": 1e-6,
                      "vs": "oracle adjoint on the stored float32 values (same input)"}}


def config6_block(trk, dev, stream, dev_index, args, fma, Ns=None):
    """The paper's production density, 1.5e-3 tracers per grid cell, on a
    1024^3 float32 field (spline I = 6, RK2, 20 steps per call): the automatic
    choice is the direct path.  Roofline of the step kernel: per particle-step
    one stencil of I^3 nodes x 3 components x 4 B (stencils of different
    tracers do not overlap at this density; the stage-2 stencil is the same
    cell's, or one cell away sharing all but I^2 of its nodes, so one stencil
    is the compulsory part) plus 52 B of particle state."""
    import torch

    import synth

    Ns = Ns or args.sparse_n
    ns, inner = int(1.5e-3 * Ns ** 3), 20
    dt = DT * 256 / Ns                      # the same CFL number as the 256^3 workload
    field = synth.velocity_field_torch(Ns, Ns // 3, 1006, device=dev, out_dtype=torch.float32)
    t = trk.Tracker(Ns, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
    t.set_field(field)
    del field
    p = synth.uniform_particles_torch(ns, 7, device=dev)
    notes = {"cfl_slow_path_used": False}
    call = lambda: t.advance(p, dt, inner, trk.TRK_RK2)  # noqa: E731
    for _ in range(2):
        call()
    sync_flags(t, trk, notes)
    kind = kernel_name(trk, t)
    if kind == "direct":
        notes["direct_node_loads"] = "texture" if t.field_texture() else "plain"
    ms, reps, clk = timed(call, stream, dev_index, min_s=0.6, max_reps=20)
    prof = profiled(t, trk, call)
    sync_flags(t, trk, notes)
    step_ms, step_n = prof["step"]
    launch_ms = step_ms / max(step_n, 1)
    alg = ns * (I ** 3 * 3 * 4 + 52)
    rec = sparse_ncu_record(kind)
    per_particle = rec.get("dram_bytes_per_particle")
    t.close()
    del p
    return {"metric": "particle-steps/s", "value": ns * inner / (ms * 1e-3), "unit": "particle-steps/s",
            "workload": f"{Ns}^3 fp32 velocity |k|<={Ns // 3}, {ns} uniform tracers (1.5e-3 per cell, the paper's "
                        f"density), spline I={I} m={M}, {inner} RK2 steps dt={dt} per call, re-binned every step",
            "ms_per_step": ms / inner, "calls_timed": reps, "kernel": kind,
            "roofline": hbm_roofline(alg, launch_ms, kind, "one stencil x I^3 x 3 x 4 B + 52 B state per particle-step",
                                     traffic=per_particle * ns if per_particle else None,
                                     l2_hit_rate=rec.get("l2_hit_rate")),
            "phase_ms_per_step": {"step_kernel": step_ms / inner, "binning": prof["bin"][0] / inner},
            "clocks": clk, "notes": notes}


def sparse_ncu_record(kind):
    """The committed ncu summary of the sparse direct step kernel (captured on a
    smaller grid at the same density; the traffic of this kernel grows with the
    particle count), if it matches the source."""
    if kind != "direct":
        return {}
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        e = json.load(fh).get("k_direct_rk2_f32_i6_sparse")
    if not e or e.get("source_sha") != kernel_source_sha("direct"):
        return {}
    return e


def tuner_table(trk, dev, stream, dev_index, args, fma):
    """The step tuner against tracer density (256^3 float32 field, spline I = 6,
    RK2 and AB2, dt = 5e-3): per density, the ms per step of every candidate
    launch shape fixed, and the one the tuner picks on its own (first call of
    24 steps)."""
    import torch

    import synth

    Nt = 256
    field = torch.from_numpy(synth.velocity_field_np(Nt, 85, 1001).astype("float32")).to(dev)
    rows = []
    cands = [("column seg 4", dict(step_kernel=trk.TRK_STEP_COLUMN, column_segment=4)),
             ("column seg 8", dict(step_kernel=trk.TRK_STEP_COLUMN, column_segment=8)),
             ("column seg 16", dict(step_kernel=trk.TRK_STEP_COLUMN, column_segment=16)),
             ("block (tensor-copy halo)", dict(step_kernel=trk.TRK_STEP_BLOCK, halo_copy=trk.TRK_HALO_TMA)),
             ("block (cp.async halo)", dict(step_kernel=trk.TRK_STEP_BLOCK, halo_copy=trk.TRK_HALO_ASYNC)),
             ("direct edge 8", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=8)),
             ("direct edge 16", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=16)),
             ("direct edge 32", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=32)),
             ("direct edge 8, 128 per CTA", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=8, direct_particles=128)),
             ("direct edge 16, 128 per CTA", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=16,
                                                   direct_particles=128)),
             ("direct edge 8, 64 per CTA", dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=8, direct_particles=64))]
    names = {trk.TRK_STEP_COLUMN: "column", trk.TRK_STEP_BLOCK: "block", trk.TRK_STEP_DIRECT: "direct"}
    for scheme, sname in ((trk.TRK_RK2, "RK2"), (trk.TRK_AB2, "AB2")):
        for dens in (1.5e-3, 1 / 64, 1 / 32, 1 / 16, 1 / 8, 1 / 4, 1 / 2):
            n = int(dens * Nt ** 3)
            pos0 = synth.uniform_particles_torch(n, 8, device=dev)
            row = {"scheme": sname, "per_cell": dens, "np": n, "ms_per_step": {}}
            for label, tun in [("tuner", None)] + cands:
                t = trk.Tracker(Nt, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
                if tun is not None:
                    t.set_tuning(**tun)
                t.set_field(field)
                p = pos0.clone()
                rhs = torch.zeros((3, n), dtype=torch.float32, device=dev) if scheme == trk.TRK_AB2 else None
                t.advance(p, DT, 24, scheme, rhs=rhs)       # the tuner's first call (timed candidates)
                if tun is None:
                    info = t.tuning()
                    row["tuner_pick"] = {"kernel": names.get(info["step_kernel"], "?"),
                                         "direct_block": info["direct_block"],
                                         "direct_particles": info["direct_particles"],
                                         "column_segment": info["column_segment"], "source": info["source"]}
                ms, _, _ = timed(lambda: t.advance(p, DT, 20, scheme, rhs=rhs, history_valid=scheme != trk.TRK_RK2),
                                 stream, dev_index, min_s=0.2, max_reps=10)
                row["ms_per_step"][label] = ms / 20
                try:
                    t.sync()
                except trk.TrackerError as e:
                    if e.status != trk.TRK_ECFL:
                        raise
                t.close()
            rows.append(row)
            del pos0
            torch.cuda.empty_cache()
    return {"value": 0.0, "workload": "tuner table: 256^3 fp32, spline I=6, RK2 and AB2 against density", "rows": rows}


def run_single_config(args):
    """--config N: one configuration on its own, printed as one JSON line."""
    import torch

    import paper_2107_01104_gb300 as trk
    from paper_2107_01104_gb300 import build as lib_build

    torch.cuda.set_device(0)
    lib_build.build()
    trk.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    fma = {"fp32": trk.tracker_probe_fma(trk.TRK_DTYPE_F32), "fp64": trk.tracker_probe_fma(trk.TRK_DTYPE_F64)}
    fn = {1: config1_block, 3: config3_block, 4: config4_block, 5: config5_block, 6: config6_block,
          7: tuner_table}[args.config]
    d = fn(trk, dev, stream, 0, args, fma)
    line = {"metric": d.get("metric", METRIC), "value": d["value"], "unit": d.get("unit", UNIT), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": d.get("dtype", "f32"), "data": "synthetic",
            "config": {"workload": d.get("workload", f"config {args.config}")}, "result": d}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 2:
        run_gb300(args)
    else:
        run_single_config(args)


if __name__ == "__main__":
    main()
