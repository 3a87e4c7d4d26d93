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
                    help="step kernel of the headline workload (default: the column kernel)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5, 6],
                    help="2: the headline workload (default); 1 small, 3 precision, 4 batching, 5 adjoint, "
                         "6 the paper's sparse tracer density")
    ap.add_argument("--sparse-n", type=int, default=1024, help="grid of config 6 (1.5e-3 tracers per cell)")
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
def field_and_particles():
    import numpy as np

    import synth

    field = synth.velocity_field_np(N, KMAX, SEED_FIELD).astype(np.float32)
    pos = synth.uniform_particles_np(NP, SEED_POS)
    return field, pos


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
# GB300 arm
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
    if rank == 0:
        lib_build.build()
    if ws > 1:
        dist.barrier()
    trk.load_library()

    field, pos = field_and_particles()
    tr = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
    tr.set_step_kernel({"auto": trk.TRK_STEP_AUTO, "block": trk.TRK_STEP_BLOCK,
                        "column": trk.TRK_STEP_COLUMN, "direct": trk.TRK_STEP_DIRECT}[args.step_kernel])
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

    # ---------------- device-timed region (the step pairs replay from CUDA graphs) ----------------
    clocks = ClockSampler(torch.cuda.current_device())
    barrier_sync()
    clocks.start()
    time.sleep(0.2)
    launches0 = tr.launch_count
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
    # (tracker_profile records events around every launch, which turns the
    # graph replay off; the headline value above is not taken from it)
    psteps = max(1, min(args.steps, 3))
    barrier_sync()
    trk.tracker_profile(tr.h, True)
    for _ in range(psteps):
        tr.advance(p, DT, args.inner, trk.TRK_RK2)
    barrier_sync()
    prof = trk.tracker_profile_read(tr.h)
    trk.tracker_profile(tr.h, False)
    sync_flags(tr, trk, notes)

    # ---------------- roofline of the step kernel ----------------
    step_ms, step_n = prof["step"]
    avg_launch_s = step_ms * 1e-3 / max(step_n, 1)
    field_bytes = 3 * N ** 3 * 4
    alg_bytes = field_bytes + 52 * NP                 # field once + fp64 positions read and written + key
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    kind = {trk.TRK_STEP_BLOCK: "block", trk.TRK_STEP_COLUMN: "column",
            trk.TRK_STEP_DIRECT: "direct"}[tr.last_step_kernel()]
    kernel_label = STEP_KERNELS[kind][0]
    if kind == "direct":   # node loads through the texture object (three quarters of the rows) or plain loads
        notes["direct_node_loads"] = "texture" if tr.field_texture() else "plain"
        kernel_label = kernel_label[:-1] + (",NM_TEX4>" if tr.field_texture() else ",NM_VEC4>")
    sha = kernel_source_sha(kind)
    gather_bytes = NP * 2 * I ** 3 * 3 * 4            # two stencil gathers per RK2 step, float32
    sm_mhz = clk.get("sm_mhz") or 1900.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    smem_peak = nsm * 128 * sm_mhz * 1e6 / 1e9
    # separable contraction: per stage and component I^3 + I^2 + I FMAs (x1 sums, then x2, then x3)
    fma_per_ps = 2 * 3 * (I ** 3 + I ** 2 + I)
    fp32_peak = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12      # TFLOP/s, FP32 SIMT FMA

    # ---------------- end-to-end through the public API ----------------
    host = torch.from_numpy(pos).pin_memory()
    back = torch.empty_like(host).pin_memory()
    barrier_sync()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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

    # ---------------- other precision forms of the same workload ----------------
    variants = {}
    if not args.no_variants:
        for name, storage, inner in (("f64", trk.TRK_F64, 5), ("bf16x2", trk.TRK_BF16X2, args.inner)):
            tv = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=M, storage=storage)
            tv.set_field(torch.from_numpy(field).to(dev))
            pv = torch.from_numpy(pos).to(dev)
            tv.advance(pv, DT, 1, trk.TRK_RK2)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            reps = 2
            for _ in range(reps):
                tv.advance(pv, DT, inner, trk.TRK_RK2)
            v1.record(stream)
            torch.cuda.synchronize()
            vms = v0.elapsed_time(v1)
            variants[name] = {"value": NP * inner * reps / (vms * 1e-3), "unit": UNIT, "rk2_steps": inner * reps}
            tv.close()
        # Adams-Bashforth of orders 2 and 4 (one field evaluation per step), f32 field,
        # history already full when the timed steps start
        for name, scheme in (("ab2", trk.TRK_AB2), ("ab4", trk.TRK_AB4)):
            k = scheme + 1
            pv = torch.from_numpy(pos).to(dev)
            hist = torch.zeros((k - 1, 3, NP), dtype=torch.float32, device=dev)
            tr.advance(pv, DT, k - 1, scheme, rhs=hist, history_valid=0)
            tr.advance(pv, DT, args.inner, scheme, rhs=hist, history_valid=k - 1)
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            v0.record(stream)
            for _ in range(reps):
                tr.advance(pv, DT, args.inner, scheme, rhs=hist, history_valid=k - 1)
            v1.record(stream)
            torch.cuda.synchronize()
            vms = v0.elapsed_time(v1)
            variants[name] = {"value": NP * args.inner * reps / (vms * 1e-3), "unit": UNIT,
                              "ab_steps": args.inner * reps, "field_storage": "f32"}
            del pv, hist
        variants["sparse_1024"] = sparse_variant(trk, dev, stream, measured_peaks())

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
            "fma_roofline": {"achieved": NP * fma_per_ps * 2 / avg_launch_s / 1e12, "peak": fp32_peak,
                             "unit": "TFLOP/s", "frac": NP * fma_per_ps * 2 / avg_launch_s / 1e12 / fp32_peak,
                             "fma_per_particle_step": fma_per_ps,
                             "peak_def": "SMs x 128 FP32 FMA/clk x 2 FLOP x median SM clock under load"},
            "smem_roofline": {"achieved": gather_bytes / avg_launch_s / 1e9, "peak": smem_peak, "unit": "GB/s",
                              "frac": gather_bytes / avg_launch_s / 1e9 / smem_peak,
                              "gather_bytes_per_launch": gather_bytes,
                              "path": "shared memory" if kind != "direct" else
                              ("L1 (gathers: texture and load/store data paths)" if tr.field_texture()
                               else "L1 (global gathers)"),
                              "peak_def": "SMs x 128 B/clk (the L1 / shared-memory data path) x median SM clock under load"},
            "phase_ms_per_step": {"step_kernel": step_ms / psteps, "binning": prof["bin"][0] / psteps,
                                  "other": prof["other"][0] / psteps, "profiled_steps": psteps,
                                  "note": "event-bracketed launches without graph replay"},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "variants": variants, "notes": notes,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    tr.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# other configurations (single GPU; one JSON line each, same keys)
# --------------------------------------------------------------------------
def sparse_variant(trk, dev, stream, peaks):
    """The paper's production density, 1.5e-3 tracers per grid cell, on a 1024^3
    float32 field (spline I = 6, RK2): the automatic choice is the direct path.
    Its roofline counts, per particle and stage, one stencil of I^3 nodes x 3
    components x 4 B (no overlap between stencils at this density) plus 52 B of
    particle state per step."""
    import torch

    import synth

    Ns, ns = 1024, int(1.5e-3 * 1024 ** 3)
    dt = DT * 256 / Ns                      # the same CFL number as the 256^3 workload
    field = synth.velocity_field_torch(Ns, Ns // 3, 1006, device=dev, out_dtype=torch.float32)
    tv = trk.Tracker(Ns, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
    tv.set_field(field)
    del field
    kernel = tv.step_kernel_for(ns)
    pv = torch.from_numpy(synth.uniform_particles_np(ns, 7)).to(dev)
    steps = 20
    tv.advance(pv, dt, steps, trk.TRK_RK2)
    torch.cuda.synchronize()
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    tv.advance(pv, dt, steps, trk.TRK_RK2)
    v1.record(stream)
    torch.cuda.synchronize()
    ms = v0.elapsed_time(v1) / steps
    alg = ns * (2 * I ** 3 * 3 * 4 + 52)
    tv.close()
    del pv
    torch.cuda.empty_cache()
    gbs = alg / (ms * 1e-3) / 1e9
    return {"value": ns / (ms * 1e-3), "unit": UNIT, "N": Ns, "np": ns, "per_cell": 1.5e-3, "scheme": "RK2",
            "kernel": {trk.TRK_STEP_DIRECT: "direct", trk.TRK_STEP_COLUMN: "column",
                       trk.TRK_STEP_BLOCK: "block"}[kernel],
            "ms_per_step": ms, "dt": dt, "alg_bytes_per_step": alg, "achieved_gbs": gbs, "hbm_frac": gbs / peaks[0],
            "note": "whole step incl. binning; alg bytes = 2 stencils x I^3 x 3 x 4 B + 52 B state per particle"}


def _events():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _line(metric, value, unit, args, ms_step, workload, extra, dtype="f32", hib=True):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": ms_step, "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
         "data": "synthetic", "config": {"workload": workload}}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run_config1(args):
    """32^3 float64 field |k| <= 8, 1e4 tracers, Lagrange I=4, one RK2 step (launch-bound small case)."""
    import torch

    import paper_2107_01104_gb300 as trk
    import synth

    field = synth.velocity_field_np(32, 8, 1000)
    pos = synth.uniform_particles_np(10_000, 1)
    t = trk.Tracker(32, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F64)
    t.set_field(torch.from_numpy(field).cuda())
    p0 = torch.from_numpy(pos).cuda()
    p = p0.clone()
    for _ in range(args.warmup):
        t.advance(p, 1e-3, 1)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        t.interpolate(p, out_dtype=torch.float64)
        t.advance(p, 1e-3, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    _line("particle-steps/s", 10_000 / (ms * 1e-3), "particle-steps/s", args, ms,
          "32^3 f64 velocity |k|<=8, 1e4 tracers, Lagrange I=4, interpolate + one RK2 step dt=1e-3",
          {"note": "launch-bound (about 13 kernels for 1e4 particles)"}, dtype="f64")


def run_config3(args):
    """1024^3, u (3) + grad u (9, spectral), float32 and split bf16 storage, 2^27 tracers, I = 8."""
    import numpy as np
    import torch

    import oracle
    import paper_2107_01104_gb300 as trk
    import synth

    N, KM, NPART, NSUB, I8, M8 = 1024, 340, 1 << 27, 100_000, 8, 3
    dev = torch.device("cuda")
    pos = synth.uniform_particles_torch(NPART, 3, device=dev)
    sub = pos[:, :NSUB].cpu().numpy()
    cell, frac = oracle.split(sub, N)
    rel = np.arange(1 - I8 // 2, I8 // 2 + 1)
    c1 = (cell[0][:, None] + rel[None, :]) % N
    c2 = (cell[1][:, None] + rel[None, :]) % N
    c3 = (cell[2][:, None] + rel[None, :]) % N
    idx = ((c3[:, :, None, None] * N + c2[:, None, :, None]) * N + c1[:, None, None, :]).reshape(NSUB, -1)
    idx_t = torch.from_numpy(idx).to(dev)
    f12 = torch.empty((12, N, N, N), dtype=torch.float32, device=dev)
    stencil = np.empty((NSUB, 12, I8 ** 3), np.float64)
    for i, comp in enumerate(synth.velocity_components_torch(N, KM, 1002, device=dev)):
        f12[i] = comp.to(torch.float32)
        stencil[:, i, :] = comp.reshape(-1)[idx_t].cpu().numpy()
        del comp
    del idx_t
    torch.cuda.empty_cache()
    truth = oracle.interp_stencil(frac, stencil.reshape(NSUB, 12, I8, I8, I8), oracle.SPLINE, I8, M8)
    del stencil
    rms_u = float(np.sqrt(np.mean(truth[:3] ** 2)))
    rms_g = float(np.sqrt(np.mean(truth[3:] ** 2)))
    results, roof = {}, None
    peak, peak_kind = measured_peaks()
    for sname, storage in (("f32", trk.TRK_F32), ("bf16x2", trk.TRK_BF16X2)):
        for C in (3, 12):
            t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I8, m=M8, storage=storage)
            t.set_field(f12[:C])
            out = torch.empty((C, NPART), dtype=torch.float32, device=dev)
            for _ in range(max(1, args.warmup)):
                t.interpolate(pos, out=out)
            torch.cuda.synchronize()
            trk.tracker_profile(t.h, True)
            e0, e1 = _events()
            reps = max(1, min(args.steps, 3))
            e0.record()
            for _ in range(reps):
                t.interpolate(pos, out=out)
            e1.record()
            torch.cuda.synchronize()
            prof = trk.tracker_profile_read(t.h)
            trk.tracker_profile(t.h, False)
            ms = e0.elapsed_time(e1) / reps
            err = out[:, :NSUB].double().cpu().numpy() - truth[:C]
            key = f"{sname}_{'u' if C == 3 else 'u+grad'}"
            results[key] = {"particles_per_s": NPART / (ms * 1e-3), "ms": ms,
                            "kernel_ms": prof["step"][0] / reps, "binning_ms": prof["bin"][0] / reps,
                            "rms_err_u_over_rms_u": float(np.sqrt(np.mean(err[:3] ** 2))) / rms_u}
            if C == 12:
                results[key]["rms_err_grad_over_rms_grad"] = float(np.sqrt(np.mean(err[3:] ** 2))) / rms_g
            if storage == trk.TRK_F32 and C == 3:
                alg = 3 * N ** 3 * 4 + NPART * 36
                ach = alg / (prof["step"][0] / reps * 1e-3) / 1e9
                kname = {trk.TRK_STEP_DIRECT: "k_direct<float,8,7,INTERP,F32>",
                         trk.TRK_STEP_BLOCK: "k_block<float,8,7,INTERP,F32>"}.get(t.last_step_kernel(), "?")
                roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": None, "kernel": kname, "alg_bytes_per_launch": alg,
                        "peak_kind": peak_kind}
            results[key]["kernel"] = {trk.TRK_STEP_DIRECT: "direct", trk.TRK_STEP_BLOCK: "block"}.get(
                t.last_step_kernel(), "?")
            t.close()
            del out
            torch.cuda.empty_cache()
    head = results["f32_u"]
    _line("particles/s", head["particles_per_s"], "particles/s", args, head["ms"],
          "1024^3 u (3) + grad u (9, spectral), fp32 and split-bf16 storage, |k|<=340, 2^27 tracers, spline I=8 m=3,"
          " interpolation; error vs the fp64 oracle on 1e5 tracers", {"results": results, "roofline": roof})


def run_config4(args):
    """512^3 float32 u, 8 sets 1e3..2e7 tracers, I cycling 4/6/8, 3 or 9 outputs, 50 AB2 steps per call."""
    import torch

    import paper_2107_01104_gb300 as trk
    import synth

    N, dt, steps = 512, 2e-3, 50
    dev = torch.device("cuda")
    u = synth.velocity_field_torch(N, 170, 1003, out_dtype=torch.float32)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(u)
    del u
    sizes = [1000, 10_000, 30_000, 100_000, 1_000_000, 3_000_000, 10_000_000, 20_000_000]
    sets = []
    for s, n in enumerate(sizes):
        I = (4, 6, 8)[s % 3]
        sets.append(dict(pos=synth.uniform_particles_torch(n, 10 + s, device=dev),
                         rhs=torch.zeros((3, n), dtype=torch.float32, device=dev),
                         out=torch.zeros((9 if s % 2 else 3, n), dtype=torch.float32, device=dev),
                         family=trk.TRK_SPLINE, I=I, m=I // 2 - 1, deriv=s % 2))
    total = sum(sizes)
    for _ in range(args.warmup):
        t.advance_batched(sets, dt, steps, history_valid=True)
    torch.cuda.synchronize()
    l0 = t.launch_count
    trk.tracker_profile(t.h, True)
    trk.tracker_profile(t.h, False)   # graph replay stays on (profiling would disable it)
    e0, e1 = _events()
    e0.record()
    for _ in range(args.steps):
        t.advance_batched(sets, dt, steps, history_valid=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    _line("particle-steps/s", total * steps / (ms * 1e-3), "particle-steps/s", args, ms,
          "512^3 fp32 u |k|<=170, 8 sets (1e3..2e7, sum 3.414e7), I cycling 4/6/8, 3- or 9-component outputs,"
          " 50 AB2 steps per call, one persistent launch per step under a CUDA graph",
          {"gpu_launches": t.launch_count - l0, "per_set_path": "direct or halo, chosen by timing"})


def run_config6(args):
    """The paper's production density, 1.5e-3 tracers per grid cell, on an N^3
    float32 field (default 1024^3), spline I = 6, 20 RK2 steps per call; the
    automatic choice is the direct path.  Roofline of the step kernel in
    algorithmic bytes: per particle and stage one stencil of I^3 x 3 x 4 B
    (stencils do not overlap at this density) plus 52 B of particle state."""
    import torch

    import paper_2107_01104_gb300 as trk
    import synth

    Ns = args.sparse_n
    ns, inner = int(1.5e-3 * Ns ** 3), 20
    dt = DT * 256 / Ns                      # the same CFL number as the 256^3 workload
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    field = synth.velocity_field_torch(Ns, Ns // 3, 1006, device=dev, out_dtype=torch.float32)
    t = trk.Tracker(Ns, family=trk.TRK_SPLINE, I=I, m=M, storage=trk.TRK_F32)
    t.set_field(field)
    del field
    kind = {trk.TRK_STEP_DIRECT: "direct", trk.TRK_STEP_COLUMN: "column",
            trk.TRK_STEP_BLOCK: "block"}[t.step_kernel_for(ns)]
    p = synth.uniform_particles_torch(ns, 7, device=dev)
    notes = {"cfl_slow_path_used": False}
    for _ in range(args.warmup):
        t.advance(p, dt, inner, trk.TRK_RK2)
    sync_flags(t, trk, notes)
    if kind == "direct":
        notes["direct_node_loads"] = "texture" if t.field_texture() else "plain"
    l0 = t.launch_count
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(args.steps):
        t.advance(p, dt, inner, trk.TRK_RK2)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = t.launch_count - l0
    ms = e0.elapsed_time(e1) / (args.steps * inner)
    trk.tracker_profile(t.h, True)
    t.advance(p, dt, inner, trk.TRK_RK2)
    torch.cuda.synchronize()
    prof = trk.tracker_profile_read(t.h)
    trk.tracker_profile(t.h, False)
    sync_flags(t, trk, notes)
    step_ms, step_n = prof["step"]
    launch_s = step_ms * 1e-3 / max(step_n, 1)
    alg = ns * (2 * I ** 3 * 3 * 4 + 52)
    peak, peak_kind = measured_peaks()
    achieved = alg / launch_s / 1e9
    rec = sparse_ncu_record(kind)
    per_particle = rec.get("dram_bytes_per_particle")
    _line("particle-steps/s", ns / (ms * 1e-3), "particle-steps/s", args, ms * inner,
          f"{Ns}^3 fp32 velocity |k|<={Ns // 3}, {ns} uniform tracers (1.5e-3 per cell, the paper's density), "
          f"spline I={I} m={M}, {inner} RK2 steps dt={dt} per call, re-binned every step",
          {"roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": per_particle * ns if per_particle else None, "kernel": kind,
                        "l2_hit_rate": rec.get("l2_hit_rate"),
                        "alg_bytes_per_launch": alg, "avg_launch_ms": launch_s * 1e3, "peak_kind": peak_kind,
                        "alg_def": "2 stencils x I^3 x 3 x 4 B + 52 B state per particle-step"},
           "phase_ms_per_step": {"step_kernel": step_ms / inner, "binning": prof["bin"][0] / inner},
           "gpu_launches": launches, "notes": notes})


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


def run_config5(args):
    """256^3 float32 u, 2^22 tracers, spline I=6, 20 RK2 steps, adjoint with checkpoints every 5."""
    import numpy as np
    import torch

    import paper_2107_01104_gb300 as trk
    import synth

    N, n, dt, steps = 256, 1 << 22, 5e-3, 20
    dev = torch.device("cuda")
    field = synth.velocity_field_np(N, 85, 1004).astype(np.float32)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).to(dev))
    p0 = synth.uniform_particles_torch(n, 5, device=dev)
    gf = torch.zeros((3, N, N, N), dtype=torch.float64, device=dev)
    x = p0.clone()
    for _ in range(args.warmup):
        x.copy_(p0)
        t.advance(x, dt, steps)
        t.adjoint(p0, 2 * x, dt, steps, 5, grad_field=gf)
    torch.cuda.synchronize()
    fwd = bwd = 0.0
    for _ in range(args.steps):
        x.copy_(p0)
        a0, a1 = _events()
        b1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        t.advance(x, dt, steps)
        a1.record()
        t.adjoint(p0, 2 * x, dt, steps, 5, grad_field=gf)
        b1.record()
        torch.cuda.synchronize()
        fwd += a0.elapsed_time(a1)
        bwd += a1.elapsed_time(b1)
    fwd /= args.steps
    bwd /= args.steps
    _line("particle-steps/s", n * steps / ((fwd + bwd) * 1e-3), "particle-steps/s", args, fwd + bwd,
          "256^3 fp32 u |k|<=85, 2^22 tracers, spline I=6 m=2, 20 RK2 steps, loss sum |X_T|^2, backward by the"
          " discrete adjoint (field scatter-add + position Jacobians) with checkpoints every 5 steps",
          {"forward": {"ms": fwd, "particle_steps_per_s": n * steps / (fwd * 1e-3)},
           "backward": {"ms": bwd, "particle_steps_per_s": n * steps / (bwd * 1e-3)}})


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 2:
        run_gb300(args)
    else:
        import torch

        from paper_2107_01104_gb300 import build as lib_build

        torch.cuda.set_device(0)
        lib_build.build()
        {1: run_config1, 3: run_config3, 4: run_config4, 5: run_config5, 6: run_config6}[args.config](args)


if __name__ == "__main__":
    main()
