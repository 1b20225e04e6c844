"""Benchmark: spinor-steps/s of the split-operator massless-Dirac solve on GB300.

Workload (default): the Landau-Zener-Stueckelberg scan -- a 2048x2048 momentum
grid on [-10,10]^2 eV, 20-cycle sin^2 x-linear pulse, 1e5 time steps, seeded
(omega, E0) samples; each benchmark step is one whole solve of one sample
(evolve all steps, fused projection, density reduction), FP32-mixed.  The
FP64 solve of the same workload is timed beside it.  Inputs are synthetic.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1607_03062_gb300 import workloads as W  # noqa: E402

METRIC = "spinor-steps/s"
N_SAMPLES = 8
# FP32 lanes per SM and SMs of a GB300; nominal FP64 rate 1.25 TFLOP/s.
SMS = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_FLOPS = 1.25e12
SM_MAX_MHZ_NOMINAL = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=2048)
    ap.add_argument("--time-steps", type=int, default=100_000)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 leg")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serving", action="store_true", help="skip the request-loop leg")
    ap.add_argument("--serving-requests", type=int, default=256)
    ap.add_argument("--serving-load", type=float, default=0.8,
                    help="offered load as a fraction of the measured solve throughput")
    ap.add_argument("--serving-chunk", type=int, default=2000)
    ap.add_argument("--no-small-grid", action="store_true", help="skip the 64x64 latency leg")
    ap.add_argument("--no-magnus4", action="store_true", help="skip the fourth-order leg")
    ap.add_argument("--no-strang", action="store_true", help="skip the STRANG_XY leg")
    ap.add_argument("--no-projection", action="store_true",
                    help="skip the standalone-projection (HBM) leg")
    ap.add_argument("--projection-grid", type=int, default=4096)
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture, with the
# SHA-256 of the kernel source the counters were taken on; a different source
# means the counters are stale and the traffic is reported as null.
KERNEL_TRAFFIC = {
    "evolve_strip_kernel": {"bytes": 95.11e6,
                            "source_sha256": "74889d15ce1ba2e7c4751818ff356b4b99ed59e4886b167b6c79eeb474c6e413"},
}


def kernel_source_sha256():
    """SHA-256 over the strip kernel's translation unit (dsp_strip.cu and the headers
    it includes)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("dsp_strip.cu", "dsp_device.cuh", "dsp_internal.h", "dsp_df.cuh"):
        with open(os.path.join(ROOT, "paper_1607_03062_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(name):
    rec = KERNEL_TRAFFIC.get(name)
    if not rec or rec["bytes"] is None or rec["source_sha256"] != kernel_source_sha256():
        return None
    return rec["bytes"]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tan_norm_degree(group):
    """Degree of the (1 + y)^(-1/2) series that normalises a tan-normalised group of G
    steps: the lowest whose first omitted term stays below 1e-14 for y <= 1.05 x
    0.27^2 / G (the group angle of EXACT and STRANG_XY)."""
    y = 1.05 * 0.27 * 0.27 / group
    c, yk = 1.0, 1.0
    for k in range(1, 16):
        c *= (2 * k - 1) / (2 * k)
        yk *= y
        if c * yk <= 1e-14:
            return k - 1
    return 15


def tan_chain_ops(group):
    """FP32 lane instructions per spinor-step of a tan-normalised group of G steps,
    past the step's coefficients: the chain (0 for the first step, 6 for the second,
    9 for each further one) and, once per group, y = det W - 1 (5), its series (DF),
    the scaled entries (5) and the compensated update (28): 9 + (26 + DF) / G."""
    return 9 + (26.0 + tan_norm_degree(group)) / group


def ops_mixed(dc, ds, group=2, strips=False, tdeg=0):
    """FP32 lane instructions per spinor-step of the FP32-mixed EXACT path.  Steps one
    at a time (G = 1): dt P (4) + theta^2 (2) + dc + ds + q (2) + the update (12) and
    Fast2Sum (12) = 32 + dc + ds.  Tan-normalised groups: dt P (4) + theta^2 (2) +
    tan(theta)/theta - 1 (tdeg) + tau (2) + tan_chain_ops; at tdeg = 1 the product
    c1 theta^2 is formed from fl(c1 P_x) and fl(fl(c1 P_y) P_y) (2 + 1) and one
    multiply-add: 4 + 4 + 2.  On row strips the momentum work of a step is shared:
    each thread forms dt P_x (and at tdeg = 1 fl(c1 P_x)) once for its 4 spinors (2
    or 3 scalar ops: 0.5 or 0.75 per spinor) and reads dt P_y and fl(dt P_y^2) (or
    fl(fl(c1 P_y) P_y)) from the strip's row table: 4.5 (tdeg = 1: 6.25) fewer per
    spinor-step (the table itself, a few operations per row and step for 1024
    spinors, is left out)."""
    if group == 1:
        return 32 + dc + ds - (4.5 if strips else 0.0)
    if tdeg == 1:
        return 10 + tan_chain_ops(group) - (6.25 if strips else 0.0)
    return 8 + tdeg + tan_chain_ops(group) - (4.5 if strips else 0.0)


def ops_magnus4(dc, ds, group=1, strips=False, tdeg=0):
    """FP32 lane instructions per spinor-step of the MAGNUS4 path.  Single steps: 4 (Pbar)
    + 2 (n_z) + 3 (|n|^2) + dc + ds + 3 (q, q_z) + 16 ((U - I) psi + lo) + 12 (Fast2Sum)
    = 40 + dc + ds.  Tan-normalised groups of G: 4 (Pbar) + 2 (n_z) + 3 (|n|^2) + tdeg
    (tan|n|/|n| - 1) + 3 (tau, t_z) per step, then the chain: 1 to start it (-t_z), 13
    per further step, and once per group y = det W - 1 (5), its series (DF), the scaled
    entries (5) and the compensated update (28): 12 + tdeg + 13 + (26 + DF) / G.  On row
    strips dt Pbar_y and -fl(dt Pbar_y D_x) come from the strip's row table and dt
    Pbar_x is formed once per thread for its 4 spinors: 4.5 fewer per spinor-step."""
    save = 4.5 if strips else 0.0
    if group == 1:
        return 40 + dc + ds - save
    return 12 + tdeg + 13 + (26.0 + tan_norm_degree(group)) / group - save


def ops_strang(dc, ds, group=1, strips=False, tdeg=0):
    """FP32 lane instructions per spinor-step of the STRANG_XY path.  Steps one at a
    time: dt P (4) + P_x^2, P_y^2 (2) + 2 dc + 2 ds (cos - 1 and sin/theta - 1 of both)
    + 5 (sin 2a, sin b, cos b sin 2a, m) + 28 (update, Fast2Sum); on row strips the
    P_y parts come from the strip's row table and the P_x parts are formed once per
    thread for its 4 spinors: 3 per spinor + (4 + dc + ds) / 4.  Tan-normalised
    groups: dt P (4) + squares (2) + tan b, tan 2a (tdeg + 1 each) + sec 2a - 1 (tdeg)
    + tau_r (1) = 9 + 3 tdeg, on row strips 1 per spinor + (4 + 2 tdeg) / 4 per thread;
    then tan_chain_ops."""
    if group == 1:
        coef = 3 + (4 + dc + ds) / 4.0 if strips else 11 + 2 * (dc + ds)
        return coef + 28
    coef = 1 + (4 + 2 * tdeg) / 4.0 if strips else 9 + 3 * tdeg
    return coef + tan_chain_ops(group)


def ops_fp64(dc, ds, strips=False):
    """FP64 instructions per spinor-step of the FP64 EXACT step: dt P (2) + the small parts
    m = cos(theta) - 1 and s1 = sin(theta)/theta - 1 (evaluated in double-float FP32
    arithmetic, series degrees dc and ds; 2 FP64 adds to bring them to double) + q (2) +
    the update (12) = 18, whatever the degrees.  On row strips dt P_x is formed once per
    thread for its 4 spinors (0.25 each) and dt P_y comes from the strip's row table:
    16.25.  The FP32 instructions of the series (about 300 per spinor-step at degrees
    (5, 5)) issue beside them and are not counted against the FP64 peak."""
    return 16.25 if strips else 18.0


def launches_per_solve(n, strips, sms, ctas_per_sm=2):
    """Kernel launches of one dsp_solve of an n x n grid: the evolve launch (on row
    strips, split in two when the library runs the last wave of CTAs in 2-row strips,
    by the same rule as its split_last_wave: 4-row strips of 256 columns, the strip
    kernel's 2 CTAs per SM) and the density finalize."""
    evolve = 1
    if strips:
        ncb, nstrips = n // 256, (n + 3) // 4
        slots = sms * ctas_per_sm
        rem = (ncb * nstrips) % slots
        if rem:
            k = min(nstrips, (rem + ncb - 1) // ncb)
            tail_tiles = ncb * ((n - 4 * (nstrips - k) + 1) // 2)
            if tail_tiles <= slots and nstrips > k:
                evolve = 2
    return evolve + 1


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1607_03062_gb300 import binding as B
    from paper_1607_03062_gb300 import build as Bd

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        Bd.build()
    if world > 1:
        dist.barrier()
    B.lib()

    n = args.grid
    nsteps = args.time_steps
    cfgs = [W.config_lzs_2048(s, n=n, steps=nsteps) for s in range(N_SAMPLES)]
    tables = [B.sample_pulse(c["pulse"], nsteps) for c in cfgs]
    g0 = cfgs[0]["grid"]
    stream = torch.cuda.current_stream()
    st_ptr = stream.cuda_stream

    def make(prec):
        nbytes = B.state_bytes(n, n, prec)
        state = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        mdt = torch.float64 if prec == "fp64" else torch.float32
        mp = torch.empty((n, n), dtype=mdt, device="cuda")
        h = B.create_grid(n, n, g0["px"], g0["py"], prec, "exact", 1, st_ptr, state.data_ptr(),
                          nbytes)
        return h, state, mp

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    kept = {}  # (precision, sample) -> host |c+|^2 map, for the accuracy check
    dens_by = {}  # (precision, sample) -> density

    strips_seen = []

    def timed_solves(prec, warm, steps, sample_offset, keep_sample=None):
        h, state, mp = make(prec)
        dens = []
        times = []
        ops = []
        for k in range(warm + steps):
            s = (sample_offset + k * world + rank) % N_SAMPLES
            a_mid, a_in, a_out, dt = tables[s]
            B.set_pulse(h, a_mid, dt, a_in, a_out)
            flush.fill_(float(k))  # evict the previous solve from L2
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.solve(h, mp.data_ptr(), want_density=False)
            e1.record(stream)
            torch.cuda.synchronize()
            if s == keep_sample and (prec, s) not in kept:
                kept[(prec, s)] = mp.double().cpu().numpy()
            if (prec, s) not in dens_by:
                dens_by[(prec, s)] = B.reduce_density(h)
            if k >= warm:
                times.append(e0.elapsed_time(e1) / 1e3)
                dens.append(B.reduce_density(h))
                info = B.get_info(h)
                strips_seen.append(bool(info["row_strips"]))
                if prec == "fp64":
                    ops.append(ops_fp64(info["cos_degree"], info["sinc_degree"],
                                        bool(info["row_strips"])))
                else:
                    ops.append(ops_mixed(info["cos_degree"], info["sinc_degree"],
                                         info["group_steps"], bool(info["row_strips"]),
                                         info["tan_degree"]))
        B.destroy_grid(h)
        del state, mp
        return times, dens, ops

    sampler = ClockSampler(local)
    # ---- FP32-mixed (headline) ----
    sampler.start()
    t_mixed, d_mixed, o_mixed = timed_solves("fp32_mixed", args.warmup, args.steps, 0,
                                             keep_sample=0)
    clocks = sampler.stop()
    tot = sum(t_mixed)
    if world > 1:
        t = torch.tensor([tot], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    work_per_solve = float(n) * n * nsteps
    value = work_per_solve * args.steps * world / tot
    strips_used = bool(strips_seen) and all(strips_seen)

    # ---- FP64 ----
    fp64 = None
    if not args.no_fp64:
        # sample 0 first (its map is checked against the oracle below)
        t64, d64, o64 = timed_solves("fp64", args.fp64_warmup, args.fp64_steps, 0,
                                     keep_sample=0)
        tt = sum(t64)
        if world > 1:
            t = torch.tensor([tt], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tt = float(t.item())
        fp64 = {"value": work_per_solve * args.fp64_steps * world / tt, "unit": METRIC,
                "ms_per_step": 1e3 * tt / args.fp64_steps, "steps": args.fp64_steps,
                "warmup": args.fp64_warmup}
        # density of the same samples in both precisions
        rels = [abs(dens_by[("fp32_mixed", smp)] - v) / v for (p_, smp), v in dens_by.items()
                if p_ == "fp64" and ("fp32_mixed", smp) in dens_by and v > 0]
        fp64["density_rel_diff_vs_fp32_mixed"] = max(rels) if rels else None

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    h = B.create_grid(n, n, g0["px"], g0["py"], "fp32_mixed", "exact", 1, st_ptr)
    # the caller's host map in pinned memory, as a serving loop would hold it
    host_map = torch.empty((n, n), dtype=torch.float32, pin_memory=True).numpy()
    e2e_t = []
    # the samples of the device-timed steps (k = warmup .. warmup + steps - 1), after one
    # untimed solve, so that e2e and the headline average the same work
    for i, k in enumerate([args.warmup] + list(range(args.warmup, args.warmup + args.steps))):
        s = (k * world + rank) % N_SAMPLES
        a_mid, a_in, a_out, dt = tables[s]
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.solve_host(h, a_mid, dt, a_in, a_out, host_map)
        t1 = time.perf_counter()
        if i >= 1:
            e2e_t.append(t1 - t0)
    B.destroy_grid(h)
    e2e_tot = sum(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_tot], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e = {"value": work_per_solve * args.steps * world / e2e_tot, "unit": METRIC,
           # the FP32 pulse table the host builds and the projection nodes (hi/lo
           # float pairs of every column and row)
           "h2d_bytes_per_step": 8 * nsteps + 8 * (n + n),
           "d2h_bytes_per_step": 4 * n * n + 16,
           "note": "dsp_solve_host: host midpoint table in, host |c+|^2 map (pinned) and density out"}

    # ---- the other step schemes on the same workload ----
    magnus = None
    if not args.no_magnus4:
        magnus = scheme_leg(args, cfgs, st_ptr, world, rank, "magnus4")
    strang = None
    if not args.no_strang:
        strang = scheme_leg(args, cfgs, st_ptr, world, rank, "strang_xy")

    # ---- small grid: sequential vs time-parallel solve latency ----
    small = None
    if not args.no_small_grid and rank == 0:
        small = small_grid_leg(st_ptr)

    # ---- serving: continuous batching vs one request at a time ----
    serving = None
    if not args.no_serving and rank == 0:
        serving = serving_leg(args, value / world, st_ptr)

    # ---- standalone projection of a state on the device (HBM-bound) ----
    projection = None
    if not args.no_projection and rank == 0:
        projection = projection_leg(args, st_ptr)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the evolve kernel (FP32 pipe) ----
    peaks = load_peaks()
    # achieved = algorithmic FP32 instructions of each timed launch / its event time
    achieved = statistics.mean(o * work_per_solve / t for o, t in zip(o_mixed, t_mixed)) / 1e12
    kernel_name = "evolve_strip_kernel" if strips_used else "evolve_mixed_kernel"
    peak = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "Tinst/s (FP32 lane instructions)", "frac": achieved / peak,
            "traffic": kernel_traffic(kernel_name), "kernel": kernel_name,
            "ops_per_spinor_step": o_mixed,
            "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz (unit counts x max SM clock)"}
    roof["ceiling_spinor_steps_per_s"] = peak * 1e12 / statistics.mean(o_mixed)
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (SMS * FP32_LANES_PER_SM *
                                                     clocks["sm_mhz"] * 1e6 / 1e12)
    if fp64:
        a64 = statistics.mean(o * work_per_solve / t for o, t in zip(o64, t64)) / 1e12
        fp64["roofline"] = {"bound": "alu", "achieved": a64,
                            "peak": FP64_NOMINAL_FLOPS / 2 / 1e12,
                            "unit": "T FP64 inst/s", "frac": a64 / (FP64_NOMINAL_FLOPS / 2 / 1e12),
                            "ops_per_spinor_step": o64,
                            "peak_basis": "nominal 1.25 TFLOP/s FP64 = 0.625 T DFMA/s"}

    # ---- CPU baseline: the oracle on a bounded sample ----
    cpu = None
    accuracy = None
    if not args.no_cpu_baseline:
        cpu, accuracy = cpu_baseline(cfgs[0], args.cpu_seconds, nsteps,
                                     {p: m for (p, smp), m in kept.items() if smp == 0})

    # The order of the keys is deliberate: the figures a reader checks first
    # (headline, e2e, roofline, CPU baseline, clocks) lead, the long legs follow,
    # and the FP64 leg closes the line.
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded pulses; no dataset)",
        "config": {"workload": f"lzs_scan_{n}x{n}_{nsteps}_steps_fp32_mixed",
                   "grid": [n, n], "p_range_eV": [-10, 10], "time_steps": nsteps,
                   "pulse": "20-cycle sin^2, x-linear, (omega, E0) ~ U[0.5,3] x U[0.2,6], seed 1607",
                   "samples_rotated": N_SAMPLES, "scheme": "exact midpoint exponential",
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world} (independent samples per rank)"},
        "gpu_launches": args.steps * launches_per_solve(
            n, strips_used, torch.cuda.get_device_properties(local).multi_processor_count),
        "e2e": e2e,
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
        "arithmetic": "FP32 spinor stored compensated (hi + lo); momentum p + A from an FP32 "
                      "hi/lo p and one error-fed FP32 A per step; FP64 initial state; "
                      "double-float projection; FP64 density",
        "density_first_step": d_mixed[0] if d_mixed else None,
        "serving": serving, "small_grid": small, "magnus4": magnus, "strang_xy": strang,
        "projection": projection, "accuracy_vs_oracle": accuracy, "fp64": fp64,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# Fourth-order Magnus leg
# ------------------------------------------------------------------------------------------

SCHEME_LEGS = {
    "magnus4": ("magnus4 (fourth order, 2 Gauss points/step)", ops_magnus4),
    "strang_xy": ("strang_xy (sigma_x / sigma_y split of each step)", ops_strang),
}


def scheme_leg(args, cfgs, stream, world, rank, scheme, warm=1, reps=2):
    """The same 2048^2 x 1e5-step solves with another step scheme, FP32-mixed, in
    step groups like EXACT: the fourth-order Magnus step (two Gauss-point samples
    per step) or the sigma_x / sigma_y split.  Instructions per spinor-step from
    ops_magnus4 / ops_strang."""
    import torch

    from paper_1607_03062_gb300 import binding as B

    n = args.grid
    g0 = cfgs[0]["grid"]
    nbytes = B.state_bytes(n, n, "fp32_mixed")
    state = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    mp = torch.empty((n, n), dtype=torch.float32, device="cuda")
    label, ops_fn = SCHEME_LEGS[scheme]
    sample = B.sample_pulse_gauss if scheme == "magnus4" else B.sample_pulse
    h = B.create_grid(n, n, g0["px"], g0["py"], "fp32_mixed", scheme, 1, stream,
                      state.data_ptr(), nbytes)
    times, ops = [], []
    for k in range(warm + reps):
        c = cfgs[(k * world + rank) % len(cfgs)]
        a, a_in, a_out, dt = sample(c["pulse"], args.time_steps)
        B.set_pulse(h, a, dt, a_in, a_out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        B.solve(h, mp.data_ptr(), want_density=False)
        e1.record()
        torch.cuda.synchronize()
        if k >= warm:
            times.append(e0.elapsed_time(e1) / 1e3)
            info = B.get_info(h)
            ops.append(ops_fn(info["cos_degree"], info["sinc_degree"], info["group_steps"],
                              bool(info["row_strips"]), info["tan_degree"]))
    B.destroy_grid(h)
    work = float(n) * n * args.time_steps
    achieved = statistics.mean(o * work / t for o, t in zip(ops, times)) / 1e12
    peak = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    return {"value": work * reps / sum(times), "unit": METRIC, "ms_per_step": 1e3 * statistics.mean(times),
            "steps": reps, "warmup": warm, "scheme": label,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                         "unit": "Tinst/s (FP32 lane instructions)", "ops_per_spinor_step": ops}}


# ------------------------------------------------------------------------------------------
# Small-grid leg
# ------------------------------------------------------------------------------------------

def small_grid_leg(stream, reps=5, warm=3):
    """64x64 on [-4,4]^2, 5-cycle sin^2 pulse, 2000 steps: four 1024-point tiles,
    far too few to fill the GPU.  Latency of one solve, sequential (dsp_solve) vs
    time-parallel (dsp_solve_segmented, automatic segment count), CUDA events."""
    import torch

    from paper_1607_03062_gb300 import binding as B

    cfg = W.config_sin2_64()
    g = cfg["grid"]
    a_mid, a_in, a_out, dt = B.sample_pulse(cfg["pulse"], cfg["steps"])
    out = {"workload": "sin2_64x64_2000_steps", "spinor_steps": 64 * 64 * cfg["steps"]}
    for prec in ("fp64", "fp32_mixed"):
        grid = B.Grid(g["nx"], g["ny"], g["px"], g["py"], prec)
        res = {}
        for mode in ("sequential", "segmented"):
            times = []
            for k in range(warm + reps):
                grid.set_pulse(a_mid, dt, a_in, a_out)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                if mode == "sequential":
                    B.solve(grid.h, grid.map.data_ptr(), want_density=False)
                else:
                    B.solve_segmented(grid.h, 0, grid.map.data_ptr(), want_density=False)
                e1.record()
                torch.cuda.synchronize()
                if k >= warm:
                    times.append(e0.elapsed_time(e1))
            res[mode + "_ms"] = statistics.median(times)
        res["speedup"] = res["sequential_ms"] / res["segmented_ms"]
        out[prec] = res
        grid.close()
    return out


# ------------------------------------------------------------------------------------------
# Standalone projection leg
# ------------------------------------------------------------------------------------------

def projection_leg(args, stream, reps=10, warm=3):
    """dsp_project of a state already on the device (a launch with no steps), on
    the 4096^2 two-colour grid after 512 steps, in both precisions: the
    projection kernel reads the 32-byte state of every point and writes its map
    value (4 bytes FP32-mixed, 8 bytes FP64), plus one double per 256-point
    granule of the density sum.  Algorithmic bytes / CUDA-event time of the
    launch, against the measured HBM copy bandwidth; the inputs are larger than
    L2 (the state alone is 537 MB, four times the 129 MB L2), so no flush."""
    import torch

    from paper_1607_03062_gb300 import binding as B

    n = args.projection_grid
    steps = 512  # the two-colour pulse in 512 steps: theta_max ~ 1.4 (< pi)
    cfg = W.config_two_colour_4096(n=n, steps=steps)
    g = cfg["grid"]
    tab = B.sample_pulse(cfg["pulse"], steps)
    hbm = load_peaks().get("hbm_gbs")
    out = {"workload": f"two_colour_{n}x{n}, state after {steps} steps", "points": n * n,
           "peak_gbs": hbm, "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy), of measured"}
    for prec, map_bytes in (("fp32_mixed", 4), ("fp64", 8)):
        grid = B.Grid(g["nx"], g["ny"], g["px"], g["py"], prec)
        grid.set_pulse(tab[0], tab[3], tab[1], tab[2])
        grid.evolve(steps)
        times = []
        for k in range(warm + reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            B.project(grid.h, grid.map.data_ptr())
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            if k >= warm:
                times.append(e0.elapsed_time(e1) / 1e3)
        grid.close()
        parts = (n * n + 255) // 256
        alg = n * n * (32 + map_bytes) + 8 * parts
        t = statistics.median(times)
        gbs = alg / t / 1e9
        out[prec] = {"us": round(t * 1e6, 2), "algorithmic_bytes": alg,
                     "bytes_per_point": 32 + map_bytes, "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / hbm, 3) if hbm else None}
    return out


# ------------------------------------------------------------------------------------------
# Serving leg
# ------------------------------------------------------------------------------------------

def serving_leg(args, solve_rate, stream):
    """256 seeded Poisson requests through the library's continuous-batching server
    vs the same requests one at a time (FIFO, each alone); at an offered load of
    args.serving_load x the measured solve throughput (latency), and with every
    request submitted at t = 0 (throughput at saturation)."""
    from paper_1607_03062_gb300 import serve

    probe = W.serving_requests(count=args.serving_requests, seed=1607, rate_hz=1.0)
    mean_work = float(np.mean([r["grid"]["nx"] * r["grid"]["ny"] * r["steps"] for r in probe]))
    rate = args.serving_load * solve_rate / mean_work
    reqs = serve.prepare(W.serving_requests(count=args.serving_requests, seed=1607, rate_hz=rate))
    budget = 64 << 30
    out = {"requests": len(reqs), "rate_hz": round(rate, 3), "offered_load": args.serving_load,
           "chunk_steps": args.serving_chunk}
    legs = {"batched": dict(max_active=48, chunk_steps=args.serving_chunk),
            "one_at_a_time": dict(max_active=1, chunk_steps=1 << 40)}
    for name, kw in legs.items():
        for mode, realtime in (("poisson", True), ("saturated", False)):
            r = serve.run(reqs, hbm_budget_bytes=budget, stream=stream, realtime=realtime, **kw)
            out[f"{name}_{mode}"] = {"p50_s": round(r["p50_s"], 4), "p99_s": round(r["p99_s"], 4),
                                     "throughput": float(f"{r['throughput']:.4g}"),
                                     "max_active": r["max_active_seen"]}
    out["throughput_ratio_saturated"] = (out["batched_saturated"]["throughput"] /
                                         out["one_at_a_time_saturated"]["throughput"])
    return out


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ------------------------------------------------------------------------------------------

def oracle_rate(cfg, n_points, nsteps, seed=5, nthreads=0):
    """Times the oracle on n_points seeded points of the grid; returns
    (spinor-steps/s, seconds, flat indices, |c+|^2 at those points)."""
    from oracle import oracle
    g = cfg["grid"]
    a_mid, a_in, a_out, dt = oracle.pulse_table(cfg["pulse"], nsteps)
    idx = W.sample_points(g["nx"], g["ny"], n_points, seed=seed)
    xs = oracle.grid_nodes(*g["px"], g["nx"])
    ys = oracle.grid_nodes(*g["py"], g["ny"])
    t0 = time.perf_counter()
    r = oracle.solve_points(xs[idx % g["nx"]], ys[idx // g["nx"]], a_mid, dt, a_in, a_out,
                            nthreads=nthreads)
    el = time.perf_counter() - t0
    return n_points * nsteps / el, el, idx, r["cplus2"]


def cpu_baseline(cfg, seconds, nsteps, gpu_maps=None):
    """The oracle as it stands on a seeded subset of the grid sized to ~`seconds`;
    the same points also give the GPU maps' error against the FP64 oracle."""
    from oracle import oracle
    cores = oracle.max_threads()
    rate = oracle_rate(cfg, 256, nsteps)[0]
    pts = int(max(256, min(cfg["grid"]["nx"] ** 2, rate * seconds / nsteps)))
    rate, el, idx, ref = oracle_rate(cfg, pts, nsteps)
    sample = (f"{pts} seeded points of the {cfg['grid']['nx']}^2 grid x {nsteps} steps "
              f"(sample 0), {el:.1f} s, FP64, OpenMP over points")
    base = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample}
    one = oracle_rate(cfg, 256, nsteps, seed=9, nthreads=1)
    base["single_core"] = {"value": one[0], "unit": METRIC, "cores": 1,
                           "sample": f"256 seeded points x {nsteps} steps, {one[1]:.1f} s"}
    acc = None
    if gpu_maps:
        acc = {"points": sample, "max_oracle_cplus2": float(ref.max())}
        for prec, m in gpu_maps.items():
            got = m.ravel()[idx]
            acc[prec] = {"max_abs_err_cplus2": float(np.abs(got - ref).max()),
                         "sampled_density_rel_err": float(abs(got.sum() - ref.sum()) / ref.sum())}
        if "fp32_mixed" in gpu_maps and "fp64" in gpu_maps:
            # every point of the grid: FP32-mixed against the FP64 kernel's map (which
            # meets the oracle to ~1e-13 on the points above)
            err = np.abs(gpu_maps["fp32_mixed"] - gpu_maps["fp64"]).ravel()
            acc["fp32_mixed_vs_fp64_every_point"] = {
                "points": int(err.size), "max_abs_err_cplus2": float(err.max()),
                "p99_9_abs_err_cplus2": float(np.quantile(err, 0.999))}
    return base, acc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n, nsteps = args.grid, args.time_steps
    cfg = W.config_lzs_2048(0, n=n, steps=nsteps)
    from oracle import oracle
    oracle.build()
    cores = oracle.max_threads()
    per_step_s = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    rate = oracle_rate(cfg, 256, nsteps)[0]
    pts = int(max(64, min(n * n, rate * per_step_s / nsteps)))
    times = []
    for k in range(args.warmup + args.steps):
        el = oracle_rate(cfg, pts, nsteps, seed=100 + k)[1]
        if k >= args.warmup:
            times.append(el)
    tot = sum(times)
    value = pts * nsteps * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded pulses; no dataset)",
            "config": {"workload": f"lzs_scan_{n}x{n}_{nsteps}_steps_fp32_mixed", "grid": [n, n],
                       "time_steps": nsteps},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{pts} seeded points x {nsteps} steps per step"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
