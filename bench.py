#!/usr/bin/env python
"""Throughput benchmark of the Hermite block-step engine (acc/jerk/snap interactions/s).

Default workload (the largest configuration, run on one GPU): a Plummer sphere
of N = 8,388,608 particles with Salpeter masses on [0.1, 100] (seed 5), Henon
units, eps = 1e-4, eta = 0.45, dt_max = 1/16, mixed precision (FP32 pair
arithmetic in packed f32x2 instructions, double-single position differences,
compensated sums, FP64 state, predictor, corrector and time steps).  The
start-up (hg_init: every particle active at t = 0, 7.0e13 pair evaluations) is
set-up, timed and reported apart.  One step = one graph-replayed block step
(next-block selection fused into the FP64 prediction, evaluation, j-split
reduction, FP64 correction with the new time steps); value = sum of m * N
over the timed block steps per second of device time.  The energy (the
paper's synchronisation-time diagnostic) is not part of a step: no
synchronisation time (a multiple of dt_max) is reached within a few block steps
at this N, and an FP64-pair energy of 2^23 particles costs tens of minutes.

Beside the line: the mixed kernel against the FP64 kernel on a seeded subset of
4096 particles at this N (same state; errors and both kernels' rates); both
paths integrated from t = 0 to 1/8 on the N = 65536 Plummer sphere with
FP64-pair energies for both (|dE/E| of each, "mixed vs FP64 at stated
|dE/E|"); the measured FP32 / FP64 FMA peaks; the CPU oracle on a bounded
sample; an end-to-end figure through the C ABI with host buffers; the
evaluation kernel's roofline; sampled SM clocks and the kernel launch count.

--impl reference times the CPU oracle (plain single-threaded C) on a bounded
sample of the same workload.  Under torchrun each rank runs its own replica
(seed + rank) on its own GPU: weak scaling, no collective on the data path.
--mode selects the other configurations (one JSON line each).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

PROCESS_T0 = time.perf_counter()   # the whole run's wall clock, reported beside the device-timed line

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "acc/jerk/snap interactions/s and % FP32 peak; mixed vs FP64 GPU at stated |ΔE/E|"
FLOPS_F32 = 77     # FP32 adds + muls of the pair law per interaction (FMA = 2 flops; rsqrt not counted)
FLOPS_F64 = 77     # the same count for the FP64 path
PAPER_FLOPS = 97   # the paper's count per interaction (82 SP + 15 DP)
NUM_SMS = 152
# DRAM bytes (read + write) of the evaluation kernel per launch, mean over the
# timed launches of one bench configuration, from an ncu capture of exactly
# those launches (dram__bytes_read.sum + dram__bytes_write.sum).  Keyed by
# (N, masses, precision, warm-up steps, timed steps); valid only while that
# kernel is unchanged (None: not captured for the current kernel).
EVAL_TRAFFIC = {
    # the default line with the driver's --steps 20 --warmup 5: 20 launches, 1.962e12 B in 27.4 s of kernel time
    # (72 GB/s); the i-tiles re-read the 436 MB of records from DRAM as they drift apart along them
    (8388608, "salpeter", "mixed", 5, 20): 9.8116e10,
}

# Workload of each mode: (n, imf, seed, eps, t_end); explicit flags override.
MODE_DEFAULTS = {
    "headline": (1 << 23, "salpeter", 5, 1e-4, 0.125),
    "interval": (65536, "equal", 2, 1e-4, 0.125),
    "block-sizes": (65536, "equal", 2, 1e-4, 0.125),
    "accuracy": (1 << 20, "salpeter", 3, 1e-4, 0.125),
    "large": (1 << 23, "salpeter", 5, 1e-4, 0.125),
    "eta-sweep": (16384, "equal", 2, 1e-4, 2.5),
    "jsplit": (16384, "equal", 2, 1e-4, 0.125),
    "step-times": (65536, "equal", 2, 1e-4, 0.125),
    "batch": (0, "equal", 4, 1e-3, 0.125),
}
SUBSET = 4096          # particles of the mixed-vs-FP64 kernel comparison at the headline N
ENERGY_JOB = dict(n=65536, imf="equal", seed=2, eps=1e-4, t_end=0.125)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--imf", choices=["equal", "salpeter"], default=None)
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--interval", type=float, default=1.0 / 16)
    ap.add_argument("--block-steps", type=int, default=0,
                    help="headline: block steps per step (default 1); interval: if > 0, one step = this many "
                         "block steps (no energy) instead of one interval")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--batch", action="store_true",
                    help="independent-clusters workload: batched context vs one context per cluster")
    ap.add_argument("--clusters", type=int, default=512)
    ap.add_argument("--t-end", type=float, default=None, help="block-sizes mode: integrate from 0 to this time")
    ap.add_argument("--bh-mass", type=float, default=0.0,
                    help="block-sizes mode: add a central object of this mass (stars: total mass 1)")
    ap.add_argument("--order", type=int, choices=[4, 6], default=6,
                    help="integration order: 6 (the paper's scheme) or 4 (p = 4 criterion)")
    ap.add_argument("--precisions", default="fp64,mixed", help="block-sizes / eta-sweep modes: which paths")
    ap.add_argument("--mode", choices=list(MODE_DEFAULTS), default="headline",
                    help="headline: the default line (N = 2^23 Salpeter, mixed, block steps); interval: N = 65536 "
                         "Plummer, one 1/16 interval of block steps + energy per step; batch: 512 clusters; "
                         "block-sizes: evaluation time per block-size bucket, FP64 and mixed, N = 65536 to t = 1/8; "
                         "accuracy: N = 2^20 Salpeter, mixed vs FP64 per block step and |dE/E| of both; large: "
                         "N = 2^23 Salpeter, 32 block steps including the start-up evaluation; eta-sweep: energy "
                         "and angular-momentum errors against eta (N = 16384, both paths); jsplit: evaluation "
                         "rate against m at N_j = 16384 with the j-split forced off and on (Sect. 5.5 Bfactor); "
                         "step-times: device time of every block step from t = 0 to --t-end, one graph replay each, "
                         "no section events")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the cost model's launch plans (no hg_tune before the warm-up)")
    a = ap.parse_args()
    if a.batch:
        a.mode = "batch"
    n, imf, seed, eps, t_end = MODE_DEFAULTS[a.mode]
    a.n = n if a.n is None else a.n
    a.imf = imf if a.imf is None else a.imf
    a.seed = seed if a.seed is None else a.seed
    a.eps = eps if a.eps is None else a.eps
    a.t_end = t_end if a.t_end is None else a.t_end
    return a


def workload_name(a):
    if a.mode == "headline":
        step = (f"{a.block_steps or 1} graph-replayed block step(s) (select+predict, evaluate, reduce, correct); "
                f"start-up evaluation before the warm-up")
    elif a.block_steps > 0:
        step = f"{a.block_steps} block steps"
    else:
        step = f"one {a.interval:g} time-unit interval of block steps + energy at its end"
    masses = "Salpeter masses 0.1-100" if a.imf == "salpeter" else "equal masses"
    return (f"Plummer N={a.n} Henon units, {masses} (seed {a.seed}), eps={a.eps:g}, eta=0.45, "
            f"dt_max=1/16, power-of-two block steps, mixed precision; step = {step}")


def sm_max_mhz():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]), "measured"
    except Exception:
        return 2070.0, "fallback"


def fp32_peak_tflops(mhz):
    return NUM_SMS * 128 * 2 * mhz * 1e6 / 1e12


def fp64_peak_tflops(mhz):
    return NUM_SMS * 2 * 2 * mhz * 1e6 / 1e12     # 2 DFMA/clk/SM (GB300 nominal 1.25 TFLOP/s)


class Clocks:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.proc, self.path = device, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_samples(f)
        os.unlink(self.path)
        return out


def parse_clock_samples(lines):
    """Median SM clock, the largest max clock and the throttle reasons seen in
    `nvidia-smi --query-gpu=<Clocks.FIELDS> --format=csv,noheader,nounits` lines
    (reasons: hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown,
    sw_power_cap when reported Active in any sample)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, val in zip(names, f[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload.
# ----------------------------------------------------------------------------
def oracle_sample_step(p, m_sample, eps, h):
    """An oracle block step restricted to m_sample active particles: predict all N
    by h, evaluate the sample against all N, correct the sample.  (interactions, s)."""
    import oracle

    n = p.n
    z = np.zeros((n, 3))
    idx = np.linspace(0, n - 1, m_sample).astype(np.int32)
    t0 = time.perf_counter()
    xp, vp, ap = oracle.predict(p.pos, p.vel, z, z, z, z, np.zeros(n), h)
    acc, jerk, snap = oracle.evaluate(p.mass, xp, vp, ap, eps, idx)
    for q, i in enumerate(idx):
        oracle.correct(h, p.pos[i], p.vel[i], z[i], z[i], z[i], acc[q], jerk[q], snap[q])
    return m_sample * n, time.perf_counter() - t0


def oracle_sample_size(n, target_interactions=6e8):
    return int(max(1, min(n, target_interactions // n)))


def cpu_baseline(p, eps):
    m = oracle_sample_size(p.n)
    inter, sec = oracle_sample_step(p, m, eps, 1.0 / 64)
    return {"value": inter / sec, "unit": "interactions/s", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one oracle block step with {m} of N={p.n} active (predict all N, evaluate {m}xN, "
                      f"correct {m}): {sec:.1f} s of single-threaded C FP64 on 1 of the host's "
                      f"{os.cpu_count()} cores"}


def run_reference(a, rank):
    if rank != 0:
        return
    from paper_1207_2367_gb300 import inputs
    p = inputs.plummer(a.n, a.seed, imf=a.imf)
    m = oracle_sample_size(a.n, 1.2e8)
    for _ in range(a.warmup):
        oracle_sample_step(p, m, a.eps, 1.0 / 64)
    tot_i, tot_s = 0, 0.0
    for _ in range(a.steps):
        i, s = oracle_sample_step(p, m, a.eps, 1.0 / 64)
        tot_i += i
        tot_s += s
    v = tot_i / tot_s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "interactions/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_s / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": a.n,
                   "sample": f"each step: oracle block step, {m} of N active"},
        "cpu_baseline": {"value": v, "unit": "interactions/s", "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"each step: oracle block step with {m} of N={a.n} active (predict all N, "
                                   f"evaluate {m}xN, correct {m}), single-threaded C FP64"},
        "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------
# Our engine.
# ----------------------------------------------------------------------------
def make_ctx(hg, p, a, precision, stream, device, profile=1):
    opts = hg.hg_default_opts(precision=precision, energy_precision=precision, dt_max=1.0 / 16, device=device,
                              profile=profile, stream=stream)
    return hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, opts)


class Runner:
    """Advances a context step by step (interval or fixed block-step count)."""

    def __init__(self, hg, ctx, a):
        self.hg, self.ctx, self.a, self.t = hg, ctx, a, 0.0

    def step(self):
        if self.a.block_steps > 0:
            self.hg.hg_step(self.ctx, self.a.block_steps)
            self.hg.hg_get_stats(self.ctx)          # synchronizes
            return None
        self.t += self.a.interval
        self.hg.hg_advance(self.ctx, self.t)
        return self.hg.hg_energy(self.ctx)


def tune(hg, ctx, a):
    """Autotune the evaluation plans on the context's start-up state (setup,
    before the warm-up; never inside the timed region).  Returns a summary."""
    if a.no_tune:
        return None
    w0 = time.perf_counter()
    rep = hg.hg_tune(ctx)
    return {"seconds": time.perf_counter() - w0, "buckets": len(rep),
            "changed": [{"bucket": e["bucket"], "m": e["m"], "plan": e["chosen"],
                         "model_us": round(e["model_us"], 2), "tuned_us": round(e["best_us"], 2)}
                        for e in rep if e["chosen"] >= 0]}


def roofline(hg, inter, prof, mixed, mhz, kind, traffic=None, measured=None):
    """Roofline of the evaluation kernel: algorithmic flops (pairs x 77) over the
    evaluation section's CUDA-event time, against the FMA-pipe peak derived from
    unit counts and the maximum clock, and (when given) against the peak the
    library's FMA microbenchmark measured on this GPU."""
    eval_s = prof["ms"]["evaluate"] / 1e3
    peak = fp32_peak_tflops(mhz) if mixed else fp64_peak_tflops(mhz)
    flops = FLOPS_F32 if mixed else FLOPS_F64
    ach = inter * flops / eval_s / 1e12 if eval_s > 0 else None
    out = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
           "frac": (ach / peak) if ach else None, "traffic": traffic,
           "kernel": "k_eval<Mixed>" if mixed else "k_eval<F64>",
           "flops_per_interaction": flops,
           "flops_per_interaction_rsqrt_as_4": flops + 4,
           "paper_flops_per_interaction": PAPER_FLOPS,
           "peak_note": ((f"FP32 FMA pipe: {NUM_SMS} SMs x 128 lanes x 2 flops" if mixed else
                          f"FP64 pipe: {NUM_SMS} SMs x 2 DFMA x 2 flops") + f" x {mhz:.0f} MHz ({kind} max clock)"),
           "eval_share_of_step": eval_s / (sum(prof["ms"].values()) / 1e3) if prof["ms"] else None}
    if measured:
        mp = max(measured.get("f32", 0.0), measured.get("f32x2", 0.0)) if mixed else measured.get("f64", 0.0)
        if mp > 0 and ach:
            out["measured_peak"] = mp
            out["frac_of_measured"] = ach / mp
            out["measured_peak_note"] = ("FMA microbenchmark on this GPU (hg_peak_flops: every SM full, 8 "
                                         "independent chains per thread, CUDA events), best of scalar and packed "
                                         "FP32" if mixed else "FMA microbenchmark on this GPU (hg_peak_flops, DFMA)")
    return out


def measure_peaks(hg, device, stream):
    """FMA rates of the CUDA cores measured by the library (TFLOP/s)."""
    out = {}
    for form in ("f32", "f32x2", "f64"):
        try:
            out[form] = hg.hg_peak_flops(form, device, stream)[0]
        except Exception as e:    # reported, never fatal to the line
            out[form + "_error"] = str(e)
    return out


def aggregate(ms, interactions, dist, device):
    """Whole-job figures over ranks: the slowest rank's time and the sum of the
    interactions every rank evaluated (weak scaling)."""
    if dist is None:
        return ms, interactions
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([int(interactions)], dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def run_headline(a, rank, world, dist):
    """The default line: N = 2^23 Salpeter Plummer sphere, mixed precision,
    graph-replayed block steps timed one step at a time."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    hg.load()
    stream = torch.cuda.Stream()
    bs = a.block_steps or 1
    peaks = measure_peaks(hg, local, stream) if rank == 0 else None
    p = inputs.plummer(a.n, a.seed + rank, imf=a.imf)
    # The context times its sections with CUDA events (profile = 1): a few us
    # per block step against ~1 s of evaluation at this N.
    opts = hg.hg_default_opts(precision=hg.HG_MIXED, energy_precision=hg.HG_MIXED, dt_max=1.0 / 16,
                              device=local, profile=1, stream=stream)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, opts)
    startup_s = time.perf_counter() - w0
    try:
        tuning = tune(hg, ctx, a)
        for _ in range(a.warmup):
            hg.hg_step(ctx, bs)
        hg.hg_get_stats(ctx)

        def barrier():
            if dist is not None:
                dist.barrier()

        s0 = hg.hg_get_stats(ctx)
        hg.hg_get_profile(ctx, reset=True)
        clocks = Clocks(local)
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        ms, per_step, m_step, eval_step = 0.0, [], [], []
        prof = {"ms": {k: 0.0 for k in hg.SECTIONS}, "block_steps": 0}
        torch.cuda.nvtx.range_push("timed")      # ncu --nvtx --nvtx-include "timed/" profiles only these launches
        for _ in range(a.steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0 = hg.hg_get_stats(ctx)["interactions"]
            ev0.record(stream)
            hg.hg_step(ctx, bs)
            ev1.record(stream)
            ev1.synchronize()
            per_step.append(ev0.elapsed_time(ev1))
            ms += per_step[-1]
            m_step.append((hg.hg_get_stats(ctx)["interactions"] - q0) // a.n)   # outside the event pair
            pr = hg.hg_get_profile(ctx, reset=True)
            eval_step.append(pr["ms"]["evaluate"])
            for k, v in pr["ms"].items():
                prof["ms"][k] += v
            prof["block_steps"] += pr["block_steps"]
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clk = clocks.stop()
        barrier()
        s1 = hg.hg_get_stats(ctx)
        inter = s1["interactions"] - s0["interactions"]
        launches = s1["kernels"] - s0["kernels"]
        steps_taken = s1["block_steps"] - s0["block_steps"]
        ms_max, inter_tot = aggregate(ms, inter, dist, "cuda")
        value = inter_tot / (ms_max / 1e3)
        mhz, kind = sm_max_mhz()
        roof = roofline(hg, inter, prof, True, mhz, kind, EVAL_TRAFFIC.get((a.n, a.imf, "mixed", a.warmup, a.steps)),
                        peaks)
        roof["eval_ms_per_launch"] = prof["ms"]["evaluate"] / max(1, prof["block_steps"])
        roof["pairs_per_launch"] = inter / max(1, steps_taken)
        e2e = run_e2e_blocks(a, hg, ctx, bs) if (not a.no_e2e and rank == 0) else None
        subset = subset_vs_fp64(hg, ctx, p, a, stream, local) if (not a.no_fp64 and rank == 0) else None
        if subset and peaks and peaks.get("f64"):
            subset["fp64_frac_of_measured_fp64_peak"] = subset["fp64_rate"] * FLOPS_F64 / 1e12 / peaks["f64"]
            subset["mixed_frac_of_measured_fp32_peak"] = subset["mixed_rate"] * FLOPS_F32 / 1e12 / max(
                peaks.get("f32", 0.0), peaks.get("f32x2", 0.0))
    finally:
        hg.hg_free(ctx)
    energy = energy_comparison(hg, stream, local) if (not a.no_fp64 and rank == 0) else None
    cpu = cpu_baseline(p, a.eps) if (not a.no_cpu_baseline and rank == 0) else None
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": a.n, "imf": a.imf, "seed": a.seed, "eps": a.eps,
                   "block_steps_per_step": bs,
                   "precision": "mixed: f32 pair arithmetic (packed f32x2, two pairs per instruction), "
                                "double-single dr, Kahan f32 sums widened to f64, f64 state/predictor/corrector",
                   "l2": "not flushed: the working set (436 MB of j-records streamed by every i-tile, 1.5 GB "
                         "of FP64 state) is larger than L2 (129 MB); inputs resident in HBM",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": int(launches),
        "block_steps": steps_taken,
        "interactions": inter,
        "mean_block_size": inter / max(1, steps_taken) / a.n,
        "ms_per_step_each": per_step,
        "pairs_per_step_over_n": m_step,
        "eval_ms_per_step": eval_step,
        "startup": {"seconds": startup_s, "interactions": a.n * a.n,
                    "rate": a.n * a.n / startup_s,
                    "note": "hg_init wall time: upload, validation, evaluation with all N active, first steps"},
        "gflops_paper_convention": value * PAPER_FLOPS / 1e9,
        "sections_ms": prof["ms"],
        "peaks_measured_tflops": peaks,
        "tuning": tuning,
        "mixed_vs_fp64": {"subset_at_n": subset, "energy_job": energy},
        "process_wall_s": time.perf_counter() - PROCESS_T0,
    }), flush=True)


def run_e2e_blocks(a, hg, ctx, bs):
    """The headline metric through the public C ABI with host buffers: every step
    uploads the whole state from pinned host memory (hg_set_state), takes the
    block step(s) (hg_step) and reads the whole state back (hg_get_state)."""
    import torch
    n = a.n
    host = {f: torch.empty((n,) if f in ("mass", "t", "dt") else (n, 3), dtype=torch.float64).pin_memory()
            for f in hg.STATE_FIELDS}
    t_sys = hg.hg_get_state(ctx, host)
    nbytes = sum(h.numel() * 8 for h in host.values())
    s0 = hg.hg_get_stats(ctx)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(a.steps):
        hg.hg_set_state(ctx, host, t_sys)
        hg.hg_step(ctx, bs)
        t_sys = hg.hg_get_state(ctx, host)
    wall = time.perf_counter() - w0
    inter = hg.hg_get_stats(ctx)["interactions"] - s0["interactions"]
    return {"value": inter / wall, "unit": "interactions/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "wall_s": wall, "steps": a.steps,
            "note": "host wall clock; per step: hg_set_state from pinned host memory, hg_step, hg_get_state"}


def subset_vs_fp64(hg, ctx, p, a, stream, device):
    """The mixed kernel against the FP64 kernel on the same state: a seeded
    subset of SUBSET particles (numpy default_rng(6)) of the mixed context's
    current state, both predicted 2^-20 past its last block time.  Also each
    kernel's device time and rate on that evaluation."""
    import torch
    n = a.n
    rng = np.random.default_rng(6)
    lst = np.sort(rng.choice(n, SUBSET, replace=False)).astype(np.int32)
    lst_d = torch.tensor(lst, device="cuda")
    dst, t_sys = _device_state(hg, ctx, n)
    ref = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45,
                     hg.hg_default_opts(precision=hg.HG_FP64, dt_max=1.0 / 16, stream=stream, device=device,
                                        start_mode=1))
    try:
        hg.hg_set_state(ref, dst, t_sys)
        del dst
        t = t_sys + 2.0 ** -20
        got = [np.empty((SUBSET, 3)) for _ in range(3)]
        want = [np.empty((SUBSET, 3)) for _ in range(3)]
        hg.hg_predict(ctx, t)
        us_mixed = hg.hg_time_evaluate(ctx, lst_d, SUBSET, 3)
        hg.hg_evaluate(ctx, lst, SUBSET, *got)
        scale = hg.hg_condition_scale(ctx, SUBSET)
        hg.hg_predict(ref, t)
        us_f64 = hg.hg_time_evaluate(ref, lst_d, SUBSET, 1)
        hg.hg_evaluate(ref, lst, SUBSET, *want)
    finally:
        hg.hg_free(ref)
    pairs = SUBSET * n
    return {"subset": f"{SUBSET} particles (numpy default_rng(6) choice), predicted 2^-20 past the last block "
                      f"time t = {t_sys!r}",
            "errors_vs_fp64_kernel": {name: _rel_stats(g, w) for name, g, w in
                                      zip(("acc", "jerk", "snap"), got, want)},
            "acc_conditioning": _kappa_stats(got[0], want[0], scale),
            "tolerance_normwise": {"acc": 1e-6, "jerk": 1e-5, "snap": 1e-4},
            "mixed_rate": pairs / (us_mixed * 1e-6), "fp64_rate": pairs / (us_f64 * 1e-6),
            "mixed_over_fp64": us_f64 / us_mixed, "unit": "interactions/s (evaluation + reduction kernels)"}


def energy_comparison(hg, stream, device):
    """Mixed vs FP64 at the same job: both paths integrate the N = 65536 Plummer
    sphere (equal masses, seed 2, eps 1e-4, eta 0.45, dt_max 1/16) from t = 0 to
    1/8 with the cost model's plans; energies of both with FP64 pair arithmetic;
    device time of the block steps (CUDA events) for the rate."""
    import torch
    from paper_1207_2367_gb300 import inputs
    j = ENERGY_JOB
    p = inputs.plummer(j["n"], j["seed"], imf=j["imf"])
    out = {"workload": f"Plummer N={j['n']}, {j['imf']} masses (seed {j['seed']}), eps={j['eps']:g}, eta=0.45, "
                       f"dt_max=1/16, t = 0 -> {j['t_end']:g}; FP64-pair energies for both paths"}
    for name, prec in (("mixed", hg.HG_MIXED), ("fp64", hg.HG_FP64)):
        o = hg.hg_default_opts(precision=prec, energy_precision=hg.HG_FP64, dt_max=1.0 / 16, stream=stream,
                               device=device)
        ctx = hg.hg_init(p.mass, p.pos, p.vel, j["eps"], 0.45, o)
        try:
            E0 = sum(hg.hg_energy(ctx))
            L0 = hg.hg_angular_momentum(ctx)
            s0 = hg.hg_get_stats(ctx)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            hg.hg_advance(ctx, j["t_end"])
            ev1.record(stream)
            ev1.synchronize()
            sec = ev0.elapsed_time(ev1) / 1e3
            s1 = hg.hg_get_stats(ctx)
            E1 = sum(hg.hg_energy(ctx))
            L1 = hg.hg_angular_momentum(ctx)
            inter = s1["interactions"] - s0["interactions"]
            out[name] = {"dE_over_E": abs((E1 - E0) / E0), "E0": E0, "t": s1["t_sys"],
                         "dL": float(np.linalg.norm(L1 - L0)), "block_steps": s1["block_steps"] - s0["block_steps"],
                         "interactions": inter, "seconds": sec, "value": inter / sec, "unit": "interactions/s"}
        finally:
            hg.hg_free(ctx)
    out["rate_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["dE_mixed_over_fp64"] = out["mixed"]["dE_over_E"] / out["fp64"]["dE_over_E"]
    return out


def run_step_times(a):
    """Device time of every block step of the integration from t = 0 to --t-end
    (default 1/8) on the Plummer sphere of --n particles (default 65536), each
    step one graph replay (hg_step(ctx, 1)) between CUDA events on the context's
    stream, without section events, both precisions, cost-model plans.  Per
    power-of-two bucket of m: steps, mean m, median and mean step time; and the
    whole run's device time."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    p = inputs.plummer(a.n, a.seed, imf=a.imf)
    out = {"metric": "device time per block step (graph replay, no section events)", "unit": "us",
           "config": {"workload": f"Plummer N={a.n}, {a.imf} masses (seed {a.seed}), eps={a.eps:g}, eta=0.45, "
                                  f"dt_max=1/16, t = 0 -> {a.t_end:g}, every block step, one graph replay each"}}
    wanted = {"fp64": hg.HG_FP64, "mixed": hg.HG_MIXED}
    for name in [x for x in a.precisions.split(",") if x]:
        o = hg.hg_default_opts(precision=wanted[name], dt_max=1.0 / 16, stream=stream)
        ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, o)
        try:
            hg.hg_step(ctx, 1)                  # graphs captured, first replay
            rows, total = [], 0.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            while True:
                q0 = hg.hg_get_stats(ctx)
                if q0["t_sys"] >= a.t_end:
                    break
                e0.record(stream)
                hg.hg_step(ctx, 1)
                e1.record(stream)
                e1.synchronize()
                us = 1e3 * e0.elapsed_time(e1)
                total += us
                rows.append(((hg.hg_get_stats(ctx)["interactions"] - q0["interactions"]) // a.n, us))
        finally:
            hg.hg_free(ctx)
        buckets = {}
        for m, us in rows:
            buckets.setdefault(max(1, m).bit_length() - 1, []).append((m, us))
        table = []
        for k in sorted(buckets):
            ms = np.array([x[0] for x in buckets[k]])
            ts = np.array([x[1] for x in buckets[k]])
            table.append({"bucket": f"[{1 << k}, {(2 << k) - 1}]", "steps": len(ts), "mean_m": float(ms.mean()),
                          "median_us": float(np.median(ts)), "mean_us": float(ts.mean())})
        out[name] = {"buckets": table, "total_ms": total / 1e3, "block_steps": len(rows)}
    print(json.dumps(out), flush=True)


def run_jsplit(a):
    """Sect. 5.5 Bfactor comparison: evaluation rate against the block size m at
    N_j = --n (default 16384, equal-mass Plummer, seed 2) with the j-split forced
    off (opts.jsplit = 1: one j-chunk per i-tile) against the cost model's plan
    and the autotuned plan, both precisions; evaluation + reduction kernels timed
    with CUDA events (hg_time_evaluate).  m = 1, 2, 4, ..., N_j; each list is
    spread evenly over the particles."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    n = a.n
    p = inputs.plummer(n, a.seed, imf=a.imf)
    ms = []
    m = 1
    while m <= n:
        ms.append(m)
        m *= 2
    out = {"metric": "evaluation rate against block size, j-split off / cost model / tuned", "unit": "interactions/s",
           "config": {"workload": f"Plummer N={n}, {a.imf} masses (seed {a.seed}), eps={a.eps:g}, start-up state, "
                                  "lists spread evenly, evaluation + reduction timed (hg_time_evaluate)"}}
    wanted = {"fp64": hg.HG_FP64, "mixed": hg.HG_MIXED}
    for name in [x for x in a.precisions.split(",") if x]:
        rows = {}
        for arm, jsplit in (("no_jsplit", 1), ("cost_model", 0), ("tuned", 0)):
            o = hg.hg_default_opts(precision=wanted[name], dt_max=1.0 / 16, stream=stream, jsplit=jsplit)
            ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, o)
            try:
                if arm == "tuned":
                    hg.hg_tune(ctx, m_max=n)
                hg.hg_predict(ctx, 0.0)
                for m in ms:
                    lst = np.unique(np.linspace(0, n - 1, m).astype(np.int32))
                    us = hg.hg_time_evaluate(ctx, lst, lst.shape[0], 0)
                    rows.setdefault(m, {})[arm] = {"us": us, "rate": lst.shape[0] * n / (us * 1e-6)}
            finally:
                hg.hg_free(ctx)
        table = []
        for m in ms:
            r = rows[m]
            table.append({"m": m, **{k: r[k] for k in r},
                          "gain_cost_model": r["no_jsplit"]["us"] / r["cost_model"]["us"],
                          "gain_tuned": r["no_jsplit"]["us"] / r["tuned"]["us"]})
        out[name] = table
    print(json.dumps(out), flush=True)


def run_interval(a, rank, world, dist):
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    hg.load()
    stream = torch.cuda.Stream()
    mixed = a.precision == "mixed"
    prec = hg.HG_MIXED if mixed else hg.HG_FP64
    peaks = measure_peaks(hg, local, stream) if rank == 0 else None
    p = inputs.plummer(a.n, a.seed + rank, imf=a.imf)
    ctx = make_ctx(hg, p, a, prec, stream, local, profile=0)
    tuning = tune(hg, ctx, a)
    run = Runner(hg, ctx, a)
    K0, W0 = hg.hg_energy(ctx)
    E0 = K0 + W0
    dE_at = {}
    for w in range(a.warmup):
        e = run.step()
        if e is not None and abs(run.t - 0.125) < 1e-15:
            dE_at["0.125"] = abs((sum(e) - E0) / E0)

    def barrier():
        if dist is not None:
            dist.barrier()

    # L2 (129 MB) is flushed between timed steps by writing a larger buffer,
    # outside the per-step event pairs.
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s0 = hg.hg_get_stats(ctx)
    hg.hg_get_profile(ctx, reset=True)
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ms = 0.0
    e = None
    for _ in range(a.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e = run.step() or e
        ev1.record(stream)
        ev1.synchronize()
        ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    del flush
    s1 = hg.hg_get_stats(ctx)
    inter = s1["interactions"] - s0["interactions"]
    launches = s1["kernels"] - s0["kernels"]
    if e is None:
        e = hg.hg_energy(ctx)
    dE_end = abs((sum(e) - E0) / E0)

    ms_max, inter_tot = aggregate(ms, inter, dist, "cuda")
    value = inter_tot / (ms_max / 1e3)
    mhz, kind = sm_max_mhz()

    e2e = run_e2e(a, hg, ctx, stream, run) if (not a.no_e2e and rank == 0) else None
    table = hg.hg_get_tuning(ctx)
    hg.hg_free(ctx)
    # Section times for the roofline: the same warm-up and timed steps again on a
    # context whose graphs carry CUDA events around each section (those events
    # add ~5 % to a block step, so the timed run above has none).
    pctx = make_ctx(hg, p, a, prec, stream, local, profile=1)
    hg.hg_set_tuning(pctx, table)
    prun = Runner(hg, pctx, a)
    for _ in range(a.warmup):
        prun.step()
    q0 = hg.hg_get_stats(pctx)
    hg.hg_get_profile(pctx, reset=True)
    for _ in range(a.steps):
        prun.step()
    prof = hg.hg_get_profile(pctx)
    prof_inter = hg.hg_get_stats(pctx)["interactions"] - q0["interactions"]
    hg.hg_free(pctx)
    fp64 = energy_comparison(hg, stream, local) if (mixed and not a.no_fp64 and rank == 0) else None
    cpu = cpu_baseline(p, a.eps) if (not a.no_cpu_baseline and rank == 0) else None
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if mixed else "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n": a.n,
                   "precision": ("mixed: f32 pair arithmetic (packed f32x2, two pairs per instruction), "
                                 "double-single dr, Kahan f32 sums widened to f64, f64 state/corrector, "
                                 "f64 x + h v in the predictor" if mixed else "f64 throughout"),
                   "l2": "flushed between timed steps (256 MB write outside the timed events); "
                         "inputs resident in HBM",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline(hg, prof_inter, prof, mixed, mhz, kind,
                             EVAL_TRAFFIC.get((a.n, a.imf, a.precision, a.warmup, a.steps)) if a.block_steps == 0 else None,
                             peaks),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": int(launches),
        "block_steps": s1["block_steps"] - s0["block_steps"],
        "interactions": inter,
        "dE_over_E": {"t_0.125": dE_at.get("0.125"), "end_of_timed_region": dE_end, "t_end": run.t},
        "gflops_paper_convention": value * PAPER_FLOPS / 1e9,
        "sections_ms": prof["ms"],
        "tuning": tuning,
        "mixed_vs_fp64": fp64,
    }
    print(json.dumps(out), flush=True)


def run_e2e(a, hg, ctx, stream, run):
    """The same metric through the public C ABI with host buffers: every step uploads
    the state from pinned host memory, advances, reads the energy and the state back."""
    import torch
    n = a.n
    host = {f: torch.empty((n,) if f in ("mass", "t", "dt") else (n, 3), dtype=torch.float64).pin_memory()
            for f in hg.STATE_FIELDS}
    t_sys = hg.hg_get_state(ctx, host)
    nbytes = sum(h.numel() * 8 for h in host.values())
    s0 = hg.hg_get_stats(ctx)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(a.steps):
        hg.hg_set_state(ctx, host, t_sys)
        run.step()
        t_sys = hg.hg_get_state(ctx, host)
    wall = time.perf_counter() - w0
    inter = hg.hg_get_stats(ctx)["interactions"] - s0["interactions"]
    return {"value": inter / wall, "unit": "interactions/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes + (16 if a.block_steps == 0 else 0), "wall_s": wall}


def run_batch(a):
    """512 independent Plummer clusters (sizes log-uniform in [256, 16384], seed 4,
    cluster c seed 1000 + c), eps = 1e-3, eta = 0.45, mixed precision, advanced to
    t = 1/8: one context with one persistent evaluation per global block step
    (CUDA graphs) against one context per cluster advanced one after another."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    offsets, p = inputs.cluster_batch(a.clusters, 4)
    eps, t_end = 1e-3, 0.125
    opts = hg.hg_default_opts(precision=hg.HG_MIXED, energy_precision=hg.HG_FP64, dt_max=1.0 / 16, stream=stream)

    def timed(fn):
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        w0 = time.perf_counter()
        fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / 1e3, time.perf_counter() - w0

    def batched(tuned):
        ctx = hg.hg_init_batch(offsets, p.mass, p.pos, p.vel, eps, 0.45, opts)
        tuning = tune(hg, ctx, a) if tuned else None
        E0 = sum(hg.hg_energy(ctx))
        s0 = hg.hg_get_stats(ctx)
        dev_s, wall_s = timed(lambda: hg.hg_advance(ctx, t_end))
        s1 = hg.hg_get_stats(ctx)
        dE = abs((sum(hg.hg_energy(ctx)) - E0) / E0)
        hg.hg_free(ctx)
        inter = s1["interactions"] - s0["interactions"]
        return {"seconds": dev_s, "wall_s": wall_s, "block_steps": s1["block_steps"] - s0["block_steps"],
                "interactions": inter, "value": inter / dev_s, "dE_over_E": dE, "tuning": tuning}

    model = batched(False)
    best = batched(True) if not a.no_tune else None
    main_arm = best or model

    inter_s, dev_sep, wall_sep, steps_s = 0, 0.0, 0.0, 0
    for c in range(a.clusters):
        sl = slice(int(offsets[c]), int(offsets[c + 1]))
        cx = hg.hg_init(np.ascontiguousarray(p.mass[sl]), np.ascontiguousarray(p.pos[sl]),
                        np.ascontiguousarray(p.vel[sl]), eps, 0.45, opts)
        q0 = hg.hg_get_stats(cx)
        d, w = timed(lambda: hg.hg_advance(cx, t_end))
        q1 = hg.hg_get_stats(cx)
        inter_s += q1["interactions"] - q0["interactions"]
        steps_s += q1["block_steps"] - q0["block_steps"]
        dev_sep += d
        wall_sep += w
        hg.hg_free(cx)
    print(json.dumps({
        "metric": "batched acc/jerk/snap interactions/s (independent clusters)", "unit": "interactions/s",
        "value": main_arm["value"], "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{a.clusters} Plummer clusters, sizes log-uniform in [256, 16384] (seed 4), "
                               f"N = {int(offsets[-1])}, eps = 1e-3, eta = 0.45, t = 0 -> 1/8, mixed precision"},
        "batched": main_arm,
        "batched_cost_model_plans": model if best else None,
        "one_by_one": {"seconds": dev_sep, "wall_s": wall_sep, "block_steps": steps_s, "interactions": inter_s,
                       "value": inter_s / dev_sep, "plans": "cost model"},
        "speedup": main_arm["value"] / (inter_s / dev_sep),
    }), flush=True)


# ----------------------------------------------------------------------------
# Further configurations (one JSON line each; not the driver's default line).
# ----------------------------------------------------------------------------
def _device_state(hg, ctx, n):
    import torch
    st = hg.new_state(n, like="cuda")
    t = hg.hg_get_state(ctx, st)
    return st, t


def _kappa_stats(got_acc, ref_acc, scale):
    """Acceleration errors against the condition scale sum_j m_j / (r_ij^2 + eps^2)
    (hg_condition_scale): the worst per-particle relative error with that
    particle's condition number kappa = scale / |a|, the largest error relative
    to the scale, and the median kappa."""
    g, r = np.asarray(got_acc).reshape(-1, 3), np.asarray(ref_acc).reshape(-1, 3)
    err = np.linalg.norm(g - r, axis=1)
    rn = np.linalg.norm(r, axis=1)
    per = err / np.where(rn > 0, rn, 1.0)
    kappa = scale / np.where(rn > 0, rn, 1.0)
    w = int(np.argmax(per))
    return {"worst_particle_rel_err": float(per[w]), "worst_particle_kappa": float(kappa[w]),
            "max_err_over_scale": float((err / scale).max()), "median_kappa": float(np.median(kappa)),
            "max_kappa": float(kappa.max())}


def _rel_stats(got, ref):
    """Normwise and per-particle relative errors of an [m][3] result."""
    g, r = np.asarray(got).reshape(-1, 3), np.asarray(ref).reshape(-1, 3)
    den = np.linalg.norm(r, axis=1)
    per = np.linalg.norm(g - r, axis=1) / np.where(den > 0, den, 1.0)
    return {"normwise": float(np.linalg.norm(g - r) / np.linalg.norm(r)), "max": float(per.max()),
            "median": float(np.median(per)), "p99": float(np.quantile(per, 0.99))}


def run_block_sizes(a):
    """Evaluation time of every block size that occurs from t = 0 to --t-end
    (default 1/8) on the Plummer sphere of --n particles (default 65536, eps
    1e-4), for the paths in --precisions, grouped in power-of-two buckets of m;
    CUDA events around each section of every graph-replayed block step.  Also
    the paper's block-group attribution H_G (Sect. 5.5) per section."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    mhz, kind = sm_max_mhz()
    if a.bh_mass > 0:
        p = inputs.plummer_black_hole(a.n, a.seed, a.bh_mass, imf=a.imf)
    else:
        p = inputs.plummer(a.n, a.seed, imf=a.imf)
    bh = f" + central object of mass {a.bh_mass:g} (particle N-1)" if a.bh_mass > 0 else ""
    out = {"metric": "evaluation time per block-size bucket", "unit": "us",
           "config": {"workload": f"Plummer N={a.n}, {a.imf} masses (seed {a.seed}){bh}, eps={a.eps:g}, eta=0.45, "
                                  f"dt_max=1/16, t = 0 -> {a.t_end:g}, every block step"}}
    wanted = {"fp64": hg.HG_FP64, "mixed": hg.HG_MIXED}
    for name in [x for x in a.precisions.split(",") if x]:
        prec = wanted[name]
        ctx = make_ctx(hg, p, a, prec, stream, 0)
        tuning = tune(hg, ctx, a)
        buckets, groups = {}, {}
        total_ms = 0.0
        hg.hg_get_profile(ctx, reset=True)
        while True:
            hg.hg_step(ctx, 1)
            st = hg.hg_get_stats(ctx)
            if st["t_sys"] > a.t_end:
                break
            pr = hg.hg_get_profile(ctx, reset=True)["ms"]
            m = st["last_m"]
            b = buckets.setdefault(m.bit_length() - 1, {"steps": 0, "m_sum": 0, "eval_ms": 0.0, "step_ms": 0.0})
            b["steps"] += 1
            b["m_sum"] += m
            b["eval_ms"] += pr["evaluate"] + pr["reduce"]
            b["step_ms"] += sum(pr.values())
            g = groups.setdefault(paper_group(m), {"steps": 0, "m_sum": 0, **{k: 0.0 for k in pr}})
            g["steps"] += 1
            g["m_sum"] += m
            for k, v in pr.items():
                g[k] += v
            total_ms += sum(pr.values())
        hg.hg_free(ctx)
        peak = fp64_peak_tflops(mhz) if prec == hg.HG_FP64 else fp32_peak_tflops(mhz)
        rows = []
        for k in sorted(buckets):
            b = buckets[k]
            inter = b["m_sum"] * a.n
            rate = inter / (b["eval_ms"] / 1e3)
            rows.append({"bucket": f"[{1 << k}, {(2 << k) - 1}]", "steps": b["steps"],
                         "mean_m": b["m_sum"] / b["steps"], "eval_us": 1e3 * b["eval_ms"] / b["steps"],
                         "step_us": 1e3 * b["step_ms"] / b["steps"], "interactions_per_s": rate,
                         "gflops_77": rate * 77 / 1e9, "gflops_paper_97": rate * PAPER_FLOPS / 1e9,
                         "frac_of_peak": rate * 77 / 1e12 / peak})
        # H_G (Sect. 5.5): share of the total time spent in block steps whose size
        # falls in group G, per section (sections 5-7 and 9 of the paper's Table 1,
        # host copies and MPI, do not exist here; section 1 runs inside the
        # prediction kernel of one system).
        hgroups = []
        for gname in sorted(groups):
            g = groups[gname]
            hgroups.append({"group": gname, "range": PAPER_GROUPS[gname], "steps": g["steps"],
                            "mean_m": g["m_sum"] / g["steps"],
                            "H_G_percent": {k: 100.0 * g[k] / total_ms for k in ("next", "predict", "evaluate",
                                                                              "reduce", "correct")},
                            "H_G_total_percent": 100.0 * sum(g[k] for k in ("next", "predict", "evaluate",
                                                                          "reduce", "correct")) / total_ms})
        out[name] = {"buckets": rows, "groups": hgroups, "total_ms": total_ms, "peak_tflops": peak,
                     "tuning": tuning}
    print(json.dumps(out), flush=True)


# The paper's block-size groups of Sect. 5.5 (bounds overlap in the text at 1k,
# 10k, 100k; read as half-open from below).
PAPER_GROUPS = {"A": [1, 20], "B": [21, 100], "C": [101, 1000], "D": [1001, 10000], "E": [10001, 100000],
                "F": [100001, 1 << 40]}


def paper_group(m):
    for g, (lo, hi) in PAPER_GROUPS.items():
        if lo <= m <= hi:
            return g
    return "F"


def run_eta_sweep(a):
    """Sect. 5.1 accuracy test: |dE/E| and ||L| - |L0|| / |L0| at ten equally
    spaced synchronisation times, averaged (Delta E_k, Delta L_k), against eta,
    for both paths; Plummer N (default 16384), equal masses, eps 1e-4,
    dt_max = 1/16, integrated to --t-end (default 2.5, synchronisation every 0.25)."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    n = a.n
    p = inputs.plummer(n, a.seed, imf=a.imf)
    T = a.t_end
    etas = (0.15, 0.3, 0.45, 0.6, 0.8, 1.0) if a.order == 6 else (0.05, 0.1, 0.15, 0.2, 0.3)
    wanted = {"fp64": hg.HG_FP64, "mixed": hg.HG_MIXED}
    out = {"metric": "energy and angular-momentum errors against eta (Sect. 5.1)", "order": a.order,
           "config": {"workload": f"Plummer N={n}, {a.imf} masses (seed {a.seed}), eps={a.eps:g}, dt_max=1/16, "
                                  f"t = 0 -> {T:g}, errors at t_i = i {T / 10:g}, i = 1..10; FP64 energy sums"}}
    for name in [x for x in a.precisions.split(",") if x]:
        rows = []
        for eta in etas:
            o = hg.hg_default_opts(precision=wanted[name], energy_precision=hg.HG_FP64, dt_max=1.0 / 16,
                                   stream=stream, order=a.order)
            ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, eta, o)
            E0 = sum(hg.hg_energy(ctx))
            L0 = float(np.linalg.norm(hg.hg_angular_momentum(ctx)))
            dE, dL = [], []
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for i in range(1, 11):
                hg.hg_advance(ctx, i * T / 10)
                dE.append(abs((sum(hg.hg_energy(ctx)) - E0) / E0))
                dL.append(abs(float(np.linalg.norm(hg.hg_angular_momentum(ctx))) - L0) / L0)
            wall = time.perf_counter() - w0
            st = hg.hg_get_stats(ctx)
            hg.hg_free(ctx)
            rows.append({"eta": eta, "dE_k": float(np.mean(dE)), "dL_k": float(np.mean(dL)),
                         "dE_max": float(np.max(dE)), "dL_max": float(np.max(dL)), "block_steps": st["block_steps"],
                         "interactions": st["interactions"], "wall_s": wall, "L0": L0, "E0": E0})
        out[name] = rows
    print(json.dumps(out), flush=True)


def run_accuracy(a):
    """N = 2^20 Salpeter (seed 3), eps 1e-4: 64 block steps of the mixed path;
    at each, the mixed evaluation of the block against the FP64 kernel on the same
    state (FP64 context given the mixed context's state, both predicting to the
    block time); then 64 block steps of the FP64 path from its own start-up, and
    |dE/E| of both with FP64 pair energies at their last block times."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    n, steps = a.n, (a.block_steps or 64)
    p = inputs.plummer(n, a.seed, imf=a.imf)

    def opts(prec, start_mode=0):
        return hg.hg_default_opts(precision=prec, energy_precision=hg.HG_FP64, dt_max=1.0 / 16, stream=stream,
                                  start_mode=start_mode)

    mix = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, opts(hg.HG_MIXED))
    ref = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, opts(hg.HG_FP64, start_mode=1))
    E0 = sum(hg.hg_energy(mix))
    per_step, worst = [], {"acc": 0.0, "jerk": 0.0, "snap": 0.0}
    idx = np.empty(n, dtype=np.int32)
    for _ in range(steps):
        st, t_sys = _device_state(hg, mix, n)
        hg.hg_set_state(ref, st, t_sys)
        t, m = hg.hg_next_block(mix, idx)
        lst = np.ascontiguousarray(idx[:m])
        got = [np.empty((m, 3)) for _ in range(3)]
        want = [np.empty((m, 3)) for _ in range(3)]
        hg.hg_predict(mix, t)
        hg.hg_evaluate(mix, None, m, *got)
        scale = hg.hg_condition_scale(mix, m)
        hg.hg_predict(ref, t)
        hg.hg_evaluate(ref, lst, m, *want)
        hg.hg_correct(mix, None, m)
        row = {"t": t, "m": m}
        for name, g, w in zip(("acc", "jerk", "snap"), got, want):
            row[name] = _rel_stats(g, w)
            worst[name] = max(worst[name], row[name]["normwise"])
        row["acc_conditioning"] = _kappa_stats(got[0], want[0], scale)
        per_step.append(row)
        del st
    hg.hg_free(ref)
    t_mix = hg.hg_get_stats(mix)["t_sys"]
    dE_mix = abs((sum(hg.hg_energy(mix)) - E0) / E0)
    hg.hg_free(mix)

    f64 = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, opts(hg.HG_FP64))
    torch.cuda.synchronize()
    hg.hg_step(f64, steps)
    t_f64 = hg.hg_get_stats(f64)["t_sys"]
    dE_f64 = abs((sum(hg.hg_energy(f64)) - E0) / E0)
    hg.hg_free(f64)
    ms = [r["m"] for r in per_step]
    print(json.dumps({
        "metric": "mixed vs FP64 relative error per block step; |dE/E| of both paths",
        "config": {"workload": f"Plummer N={n}, {a.imf} masses (seed {a.seed}), eps={a.eps:g}, eta=0.45, "
                               f"dt_max=1/16, {steps} block steps after the start-up evaluation"},
        "tolerance": {"acc": 1e-6, "jerk": 1e-5, "snap": 1e-4},
        "max_normwise": worst,
        "max_per_particle": {k: max(r[k]["max"] for r in per_step) for k in ("acc", "jerk", "snap")},
        "acc_worst_particle": max((r["acc_conditioning"] for r in per_step),
                                  key=lambda c: c["worst_particle_rel_err"]),
        "acc_max_err_over_scale": max(r["acc_conditioning"]["max_err_over_scale"] for r in per_step),
        "median_per_particle": {k: float(np.median([r[k]["median"] for r in per_step]))
                                for k in ("acc", "jerk", "snap")},
        "block_sizes": {"min": min(ms), "max": max(ms), "mean": float(np.mean(ms))},
        "dE_over_E": {"mixed": dE_mix, "fp64": dE_f64, "t_mixed": t_mix, "t_fp64": t_f64},
        "steps": per_step,
    }), flush=True)


def run_large(a):
    """N = 2^23 Salpeter (seed 5), eps 1e-4, mixed: the start-up evaluation
    (all N active) plus 31 block steps, timed; then a seeded (seed 6) subset of
    4096 particles evaluated by the mixed and the FP64 kernels on the same state."""
    import torch
    from paper_1207_2367_gb300 import binding as hg
    from paper_1207_2367_gb300 import inputs

    torch.cuda.set_device(0)
    hg.load()
    stream = torch.cuda.Stream()
    n, steps = a.n, (a.block_steps or 31)
    p = inputs.plummer(n, a.seed, imf=a.imf)
    mhz, kind = sm_max_mhz()
    o = hg.hg_default_opts(precision=hg.HG_MIXED, energy_precision=hg.HG_MIXED, dt_max=1.0 / 16, stream=stream,
                           profile=1)
    torch.cuda.synchronize()
    ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    ev0.record(stream)
    ctx = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45, o)
    ev1.record(stream)
    hg.hg_step(ctx, steps)
    ev2.record(stream)
    ev2.synchronize()
    init_ms, steps_ms = ev0.elapsed_time(ev1), ev1.elapsed_time(ev2)
    st = hg.hg_get_stats(ctx)
    prof = hg.hg_get_profile(ctx)
    inter = n * n + st["interactions"]
    # accuracy on a seeded subset, same state for both kernels
    rng = np.random.default_rng(6)
    lst = np.sort(rng.choice(n, 4096, replace=False)).astype(np.int32)
    dst, t_sys = _device_state(hg, ctx, n)
    ref = hg.hg_init(p.mass, p.pos, p.vel, a.eps, 0.45,
                     hg.hg_default_opts(precision=hg.HG_FP64, dt_max=1.0 / 16, stream=stream, start_mode=1))
    hg.hg_set_state(ref, dst, t_sys)
    del dst
    t = t_sys + 2.0 ** -20
    got = [np.empty((4096, 3)) for _ in range(3)]
    want = [np.empty((4096, 3)) for _ in range(3)]
    hg.hg_predict(ctx, t)
    hg.hg_evaluate(ctx, lst, 4096, *got)
    hg.hg_predict(ref, t)
    hg.hg_evaluate(ref, lst, 4096, *want)
    hg.hg_free(ref)
    hg.hg_free(ctx)
    total_s = (init_ms + steps_ms) / 1e3
    rate = inter / total_s
    print(json.dumps({
        "metric": "acc/jerk/snap interactions/s and % FP32 peak (N = 2^23)", "unit": "interactions/s",
        "value": rate, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Plummer N={n}, {a.imf} masses (seed {a.seed}), eps={a.eps:g}, eta=0.45, "
                               f"start-up evaluation + {steps} block steps, mixed precision"},
        "startup": {"ms": init_ms, "interactions": n * n, "rate": n * n / (init_ms / 1e3),
                    "note": "hg_init: upload, validation, all-active evaluation, first steps"},
        "block_steps": {"ms": steps_ms, "interactions": st["interactions"], "steps": st["block_steps"],
                        "sections_ms": prof["ms"]},
        "frac_of_fp32_peak": rate * FLOPS_F32 / 1e12 / fp32_peak_tflops(mhz),
        "subset_vs_fp64": {name: _rel_stats(g, w) for name, g, w in zip(("acc", "jerk", "snap"), got, want)},
        "subset": "4096 particles (numpy default_rng(6) choice), predicted 2^-20 past the last block time",
    }), flush=True)


def main():
    a = parse()
    modes = {"batch": run_batch, "block-sizes": run_block_sizes, "accuracy": run_accuracy, "large": run_large,
             "eta-sweep": run_eta_sweep, "jsplit": run_jsplit, "step-times": run_step_times}
    if a.mode in modes and a.impl == "ours":
        modes[a.mode](a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        run_reference(a, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl")
        dist = td
    try:
        (run_interval if a.mode == "interval" else run_headline)(a, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
