#!/usr/bin/env python3
"""Benchmark: semi-implicit ADI Cahn-Hilliard step on one 2048 x 2048 periodic grid.

Workload (the "single large run"): c_t = Lap(c^3 - c - gamma Lap c) on [0, 2 pi)^2,
2048^2 points, gamma = 0.005, dt = 5e-4, c0 ~ U[-0.05, 0.05] (SplitMix64 seed 3),
C^{-1} = C^0.  A bench step is one full ADI time step (stencil right-hand side,
x sweep, y sweep, update) through ``ch_step``.  Metric: grid-point-steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chx|reference]

``--impl reference`` times the CPU oracle (plain FP64 C, one core) on the same
workload.  With torchrun (N > 1) every rank advances its own replica (replicas
only: the path has no exchange step) and rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N = 2048
LX = 2 * np.pi
GAMMA, DT = 0.005, 5e-4
SEED = 3
WORKLOAD = "ch2d_periodic_2048sq_gamma0.005_dt5e-4"
PREWARM_S = 1.5  # untimed steps before the first measurement (see measure())
# DRAM bytes (read + write) of one whole step on this workload, summed over its
# kernels from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum).
# ncu flushes the caches before each kernel it measures, so these are cold-cache
# figures: intermediates that a live step finds in L2 are counted as DRAM reads.
STEP_DRAM_BYTES_F64 = 373.58e6 + 53.25e6
STEP_DRAM_BYTES_F32R = 213.10e6 + 63.37e6  # the three fused kernels
# DRAM bytes (read + write) per launch of the FP64 step's kernels on this
# workload, from one ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum, mean of 3 launches).  The first right-hand-side pass
# (ch_rhs: Cbar and M) writes two fields that partly stay in L2 for the
# kernels that read them next.  None: not captured for the current kernel.
KERNEL_TRAFFIC_BYTES = {"ch_rhs": 67.21e6 + 22.66e6, "ch_rhs_lap": 100.72e6 + 7.47e6}
# Algorithmic FP64 operations and bytes per grid point of each FP64 kernel.
KERNEL_FP64_OPS = {"ch_rhs": 8.0, "ch_rhs_lap": 6.0, "spike_local_x": 5.0, "spike_local_y": 5.0, "ch_xfinish": 4.0,
                   "ch_update": 5.0}
KERNEL_BYTES = {"ch_rhs": 32, "ch_rhs_lap": 32, "spike_local_x": 16, "spike_local_y": 16, "ch_xfinish": 16,
                "ch_update": 24}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, dist, device):
    """Element-wise max of per-rank timings (ms) over all ranks; identity without a process group."""
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def fp32_accuracy(dev, checkpoints=(0, 1, 100, 1000, 5000)):
    """Config-3 accuracy of the FP32+refine step at steps 0, 1, 100, 1000 and 5000:
    the per-step error against the CPU oracle from the state the FP64 path has
    reached (step 0: the first step, from the rough initial state), the FP32
    trajectory's error against the FP64 trajectory, and its mass drift."""
    import torch

    import oracle
    import paper_2101_06550_gb300 as chx

    c0 = torch.from_numpy(synth.field(SEED, N, N, -0.05, 0.05)).to(dev)
    p64 = chx.ChPlan(N, N, LX, LX, GAMMA, DT, chx.PREC_F64)
    p32 = chx.ChPlan(N, N, LX, LX, GAMMA, DT, chx.PREC_F32_REFINE)
    w64, w32 = p64.alloc_work(dev), p32.alloc_work(dev)
    a, b, c, d = c0.clone(), c0.clone(), c0.clone(), c0.clone()
    out, done = [], 0
    for k in checkpoints:
        p64.step(a, b, w64, k - done)
        p32.step(c, d, w32, k - done)
        done = k
        torch.cuda.synchronize()
        traj = float((a - c).abs().max() / a.abs().max())
        drift = float(abs(c.sum() - c0.sum()) / c0.abs().sum())
        an, bn = a.cpu().numpy(), b.cpu().numpy()
        e, f = a.clone(), b.clone()
        p32.step(e, f, w32, 1)
        ref, _ = oracle.ch_step(an, bn, LX, LX, GAMMA, DT)
        step_err = float(np.max(np.abs(e.cpu().numpy() - ref)) / np.max(np.abs(ref)))
        out.append({"step": k, "per_step_rel_err_vs_oracle": step_err, "trajectory_rel_err_vs_fp64_gpu": traj,
                    "mass_drift_rel_to_sum_abs_c": drift})
    p64.sync_status()
    p32.sync_status()
    return {"checkpoints": out,
            "note": "per-step error: one FP32+refine step from the FP64 state against the oracle; the "
                    "trajectory error grows with the spinodal instability (growth rate up to 1/(4 gamma))"}


# Algorithmic bytes per grid point of one FP32 + refinement step: the scope
# table's lower figure (48 B per point-step: the FP64 fields C^n and C^{n-1}
# read, C^{n+1} written, and the FP32 / double-float intermediates of the two
# sweeps).  The fused kernels move 72 B per point as designed (right-hand side
# 16 B in + 16 B out, x solve 8 + 8, y solve 16 in + 8 out), and 88 B when a
# one-step call keeps the roles (the x solve's 16 B copy of C^n into C^{n-1}).
FP32R_BYTES_PER_POINT = 48
FP32R_DESIGN_BYTES_PER_POINT = 88


def fp32_roofline(pts, ms_step, peaks):
    """The FP32+refine step against the measured HBM copy bandwidth, on the
    algorithmic bytes per point (the step is bound by instruction issue of its
    double-float arithmetic; this is the fraction of the memory roofline)."""
    peak = peaks.get("hbm_gbs") or 6800.0
    ach = FP32R_BYTES_PER_POINT * pts / (ms_step * 1e-3) / 1e9
    return {"kernel": "step (ch_rhs + x_solve_ff + y_solve_ff)", "bound": "hbm", "achieved": ach, "peak": peak,
            "unit": "GB/s", "frac": ach / peak, "traffic": None,
            "algorithmic_bytes_per_point": FP32R_BYTES_PER_POINT,
            "design_bytes_per_point": FP32R_DESIGN_BYTES_PER_POINT,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)" if peaks.get("hbm_gbs") else "fallback"}


def hbm_fraction(pts, ms64, ms32, peak_gbs):
    """The step's HBM traffic against the measured copy bandwidth.  The minimum a
    step must move is 24 B per point (Cn and Cn-1 in, Cn+1 out); the ncu figure
    is every kernel's DRAM bytes, cold-cache.  Both fall far below the peak: the
    step is bound by the FP64 pipe (the roofline object), not by HBM."""
    def one(ms, dram):
        d = {"ms_per_step": ms, "algorithmic_bytes_per_step": 24 * pts, "dram_bytes_per_step_ncu_cold": dram,
             "gbs_algorithmic": 24 * pts / (ms * 1e-3) / 1e9,
             "gbs_dram_ncu_cold": dram / (ms * 1e-3) / 1e9 if dram else None}
        if peak_gbs:
            d["frac_algorithmic"] = d["gbs_algorithmic"] / peak_gbs
            d["frac_dram_ncu_cold"] = d["gbs_dram_ncu_cold"] / peak_gbs if dram else None
        return d

    return {"peak_gbs": peak_gbs, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
            "fp64": one(ms64, STEP_DRAM_BYTES_F64), "fp32_refine": one(ms32, STEP_DRAM_BYTES_F32R)}


def cpu_baseline_oracle(steps: int):
    """The CPU oracle, as it stands (plain C, FP64, single thread), on `steps` full steps."""
    import oracle

    c0 = synth.field(SEED, N, N, -0.05, 0.05)
    oracle.ch_run(c0, c0, LX, LX, GAMMA, DT, 1)  # warm-up (page-in, library load)
    t0 = time.perf_counter()
    oracle.ch_run(c0, c0, LX, LX, GAMMA, DT, steps)
    dt = time.perf_counter() - t0
    return N * N * steps / dt, dt


def cpu_baseline_oracle_all_cores(steps: int):
    """The same oracle, unchanged, as independent replicas on every host core: one
    thread per core, each advancing its own 2048^2 field `steps` steps (the
    oracle is reentrant and its ctypes calls release the GIL).  Mirrors the
    paper's all-core CPU comparison with the work split by simulation."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    cores = os.cpu_count() or 1
    fields = [synth.field(SEED + k, N, N, -0.05, 0.05) for k in range(cores)]
    oracle.ch_run(fields[0], fields[0], LX, LX, GAMMA, DT, 1)  # warm-up

    def one(c0):
        oracle.ch_run(c0, c0, LX, LX, GAMMA, DT, steps)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(one, fields))
        dt = time.perf_counter() - t0
    return cores * N * N * steps / dt, dt, cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    # the oracle as it stands, on every host core: one independent 2048^2 field
    # per core (its ctypes calls release the GIL; it keeps no global state).
    # Bounded sample: a full oracle step takes about a second per core, so the
    # warm-up and the timed steps are capped to keep the run within a few minutes.
    cores = os.cpu_count() or 1
    state = [[c, c.copy()] for c in (synth.field(SEED + k, N, N, -0.05, 0.05) for k in range(cores))]

    def advance(k, nsteps):
        cn, cp = state[k]
        for _ in range(nsteps):
            cn, cp = oracle.ch_step(cn, cp, LX, LX, GAMMA, DT)
        state[k] = [cn, cp]

    warm = max(1, min(args.warmup, 3))
    with ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda k: advance(k, warm), range(cores)))
        per_step = (time.perf_counter() - t0) / warm
        steps = max(1, min(args.steps, int(120.0 / max(per_step, 1e-3))))
        t0 = time.perf_counter()
        list(ex.map(lambda k: advance(k, steps), range(cores)))
        el = time.perf_counter() - t0
    v = cores * N * N * steps / el
    line = {"impl": "reference", "metric": "grid-pt-steps/s", "value": v, "unit": "grid-pt-steps/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N, N], "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "grid-pt-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{cores} independent 2048^2 fields (one thread each) x {steps} full ADI "
                                       f"steps ({args.steps} requested, capped at about 120 s) after {warm} "
                                       f"warm-up steps"},
            "e2e": {"value": v, "unit": "grid-pt-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_chx(args, rank, world, local_rank):
    import torch

    import paper_2101_06550_gb300 as chx

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    c0 = torch.from_numpy(synth.field(SEED, N, N, -0.05, 0.05)).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MiB > L2 (129 MB)

    def measure(precision, prewarm_s=0.0):
        plan = chx.ChPlan(N, N, LX, LX, GAMMA, DT, precision)
        cn = c0.clone()
        cp = c0.clone()
        work = plan.alloc_work(dev)
        # a GPU fresh from idle runs the first second or so of work about 4% slow
        # (measured: the first process on a box, at the same reported SM clock),
        # so the first measurement is preceded by that long a run of steps
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < prewarm_s:
            plan.step(cn, cp, work, 8)
            torch.cuda.synchronize()
        for _ in range(args.warmup):
            plan.step(cn, cp, work, 1)
        torch.cuda.synchronize()

        def timed_steps():
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for k in range(args.steps):
                flush.fill_(k & 0xFF)  # L2 flush between timed steps (not timed)
                evs[k][0].record(stream)
                plan.step(cn, cp, work, 1)
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b) for a, b in evs)

        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ms = timed_steps()  # the headline: no per-kernel events inside the steps
        if dist:
            dist.barrier()
        # the same steps again with an event pair around every kernel, for the
        # per-kernel split and the roofline (the events themselves cost time, so
        # this pass is not the headline)
        plan.profile(True)
        plan.profile_read(reset=True)
        ms_profiled = timed_steps()
        prof = plan.profile_read(reset=True)
        plan.profile(False)
        plan.sync_status()
        return ms, ms_profiled, prof, plan, cn, cp, work

    clk = ClockSampler(local_rank).__enter__()
    ms64, ms64_prof, prof64, plan64, cn64, cp64, work64 = measure(chx.PREC_F64, prewarm_s=PREWARM_S)
    ms32, ms32_prof, prof32, plan32, _, _, _ = measure(chx.PREC_F32_REFINE)
    launches_per_step = sum(n for _, n in prof64.values()) / max(1, args.steps)

    # end to end through the C ABI with host buffers (ch_step_host): H2D of both
    # fields from pinned memory, one step, D2H of the new field, every step.  Three
    # plans with their own device fields rotate over three streams, so the copy
    # engines (the host link, not the SMs, bounds this number) stay busy while
    # the kernels of the other lanes run.
    lanes_n = 3
    h_cn = c0.cpu().pin_memory()
    h_cp = h_cn.clone().pin_memory()
    h_out = [torch.empty_like(h_cn).pin_memory() for _ in range(lanes_n)]
    extra_plans = [chx.ChPlan(N, N, LX, LX, GAMMA, DT, chx.PREC_F64) for _ in range(lanes_n - 1)]
    lanes = [(plan64, cn64, cp64, work64)] + [(p, torch.empty_like(cn64), torch.empty_like(cp64), p.alloc_work(dev))
                                              for p in extra_plans]
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(lanes_n)]
    e2e_steps = max(1, args.steps)

    def e2e_run(k_steps):
        for k in range(k_steps):
            plan, dn, dp, wk = lanes[k % lanes_n]
            st = e2e_streams[k % lanes_n]
            plan.step_host(h_cn, h_cp, h_out[k % lanes_n], dn, dp, wk, 1, stream=st)  # H2D, step, D2H in one call

    e2e_run(2 * lanes_n)  # warm: captures each lane's step graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in e2e_streams:
        st.wait_stream(stream)
    e2e_run(e2e_steps)
    for st in e2e_streams:
        stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    for p in extra_plans:
        p.sync_status()

    ms64, ms32, e2e_ms = max_over_ranks([ms64, ms32, e2e_ms], dist, dev)
    if rank != 0:
        clk.__exit__(None, None, None)
        if dist:
            dist.destroy_process_group()
        return

    pts = N * N
    value = world * pts * args.steps / (ms64 * 1e-3)
    peaks = _peaks()
    # dominant kernel of the FP64 step and its roofline (FP64-pipe bound)
    dom, (dom_ms, dom_n) = max(prof64.items(), key=lambda kv: kv[1][0])
    per_launch_ms = dom_ms / max(1, dom_n)
    # the FP64 pipe's rate measured in this process (DFMA throughput kernel, G DP-ops/s)
    fp64_peak_gops = chx.fp64_fma_rate()
    if dom in KERNEL_FP64_OPS:
        ach = KERNEL_FP64_OPS[dom] * pts / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp64_peak_gops, "unit": "G fp64-op/s",
                "frac": ach / fp64_peak_gops, "fp64_ops_per_point": KERNEL_FP64_OPS[dom],
                "traffic": KERNEL_TRAFFIC_BYTES.get(dom), "traffic_unit": "bytes per launch",
                "algorithmic_bytes": KERNEL_BYTES[dom] * pts, "ms_per_launch": per_launch_ms,
                "peak_source": "in-run chx_fp64_fma_rate (DFMA throughput kernel, same process)"}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp64_peak_gops, "unit": "G fp64-op/s",
                "frac": None, "traffic": None, "ms_per_launch": per_launch_ms}
    extras = {}
    if not args.no_extras:
        extras["fp32_refine_accuracy"] = fp32_accuracy(dev)
        torch.cuda.empty_cache()
        extras["solvers"] = bench_solvers(dev)
        torch.cuda.empty_cache()
        extras["ch1d"] = bench_ch1d(dev)
        extras["cn1d"] = bench_cn1d(dev)
        torch.cuda.empty_cache()
        extras["cook"] = bench_cook(dev)
        torch.cuda.empty_cache()
        extras["ensemble"] = bench_ensemble(dev, chx.PREC_F32_REFINE, args.ens_steps, 3)
        torch.cuda.empty_cache()
        extras["coarsening_stats"] = bench_coarsening_stats(dev)
        torch.cuda.empty_cache()
        extras.update(serving_suite(dev, args.serve_requests, args.serve_rate))
    clk.__exit__(None, None, None)
    cb_v, cb_t = cpu_baseline_oracle(max(1, args.cpu_steps))
    cba_v, cba_t, cba_cores = cpu_baseline_oracle_all_cores(max(1, args.cpu_steps // 4))
    line = {
        "metric": "grid-pt-steps/s", "value": value, "unit": "grid-pt-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N, N], "precision": "fp64", "l2": "flushed between timed steps",
                   "replicas": world, "prewarm_s": PREWARM_S},
        "fp32_refine": {"value": world * pts * args.steps / (ms32 * 1e-3), "ms_per_step": ms32 / args.steps,
                        "ms_per_step_profiled": ms32_prof / args.steps, "dtype": "f32+f64-residual",
                        "roofline": fp32_roofline(pts, ms32 / args.steps, peaks)},
        "ms_per_step_profiled": ms64_prof / args.steps,
        "timing": "headline steps carry no per-kernel events; kernels_ms_per_step and the roofline come from a "
                  "second pass of the same steps with an event pair around every kernel (ms_per_step_profiled)",
        "roofline": roof,
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof64.items())},
        "kernels_ms_per_step_fp32_refine": {k: v[0] / args.steps for k, v in sorted(prof32.items())},
        "cpu_baseline": {"value": cb_v, "unit": "grid-pt-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.cpu_steps} full 2048^2 ADI steps, {cb_t:.1f} s"},
        "cpu_baseline_all_cores": {"value": cba_v, "unit": "grid-pt-steps/s", "cores": cba_cores, "kind": "oracle",
                                   "sample": f"{cba_cores} independent 2048^2 fields x {max(1, args.cpu_steps // 4)} "
                                             f"ADI steps, one thread each, {cba_t:.1f} s"},
        "e2e": {"value": world * pts * e2e_steps / (e2e_ms * 1e-3), "unit": "grid-pt-steps/s",
                "h2d_bytes_per_step": 2 * pts * 8, "d2h_bytes_per_step": pts * 8},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk.summary(),
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
        "hbm": hbm_fraction(pts, ms64 / args.steps, ms32 / args.steps, peaks.get("hbm_gbs")),
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def bench_solvers(dev, reps=5):
    """Standalone batched solvers, N = 1024, batch 65536, interleaved (one solve = one call)."""
    import torch

    import paper_2101_06550_gb300 as chx

    n, batch = 1024, 65536
    sig = 0.01 * 1e-3 / (2 * np.pi / n) ** 4  # a = gamma dt / dx^4
    co = [sig, -4 * sig, 1 + 6 * sig, -4 * sig, sig]
    f = synth.uniform_torch(1, n * batch, -1, 1, device=dev)
    x = torch.empty_like(f)
    out = {}

    def timeit(fn, k=reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(k):
            x.copy_(f)  # 512 MiB copy also flushes L2
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        return ms / k

    unknowns = n * batch
    p = chx.PentaPlan(n, co, batch, mode=chx.COEF_UNIFORM)
    ms = timeit(lambda: p.solve(x))
    out["penta_uniform_f64"] = {"ms": ms, "unknowns_per_s": unknowns / (ms * 1e-3),
                                "hbm_gbs_algorithmic": 16 * unknowns / (ms * 1e-3) / 1e9,
                                "fp64_gops": 9 * unknowns / (ms * 1e-3) / 1e9}
    ms = timeit(lambda: p.solve(x, refine=True))
    out["penta_uniform_f32_refine"] = {"ms": ms, "unknowns_per_s": unknowns / (ms * 1e-3)}
    p.close()
    # variable diagonally dominant coefficients, factor + solve each call ("Rewrite")
    # the same streams as synth.diag_dominant_penta(2, n, batch), drawn on the device
    a_, b_, d_, e_ = [synth.uniform_torch(2, unknowns, -1, 1, device=dev, offset=k * unknowns) for k in range(4)]
    u = synth.uniform_torch(2, unknowns, 0, 1, device=dev, offset=4 * unknowns)
    c_ = (1.5 + 0.5 * u) * (a_.abs() + b_.abs() + d_.abs() + e_.abs())
    del u
    pp = chx.PentaPlan(n, [a_, b_, c_, d_, e_], batch, mode=chx.COEF_PER_SYSTEM)
    ms_f = timeit(lambda: pp.refactor([a_, b_, c_, d_, e_]))
    ms_s = timeit(lambda: pp.solve(x))
    out["penta_per_system_f64"] = {"ms_factor": ms_f, "ms_solve": ms_s,
                                   "unknowns_per_s_rewrite": unknowns / ((ms_f + ms_s) * 1e-3)}
    pp.close()
    del a_, b_, c_, d_, e_
    sig_t = 1e-3 / (2 * (2 * np.pi / n) ** 2)
    tp = chx.TriPlan(n, [-sig_t, 1 + 2 * sig_t, -sig_t], batch, mode=chx.COEF_UNIFORM)
    ms = timeit(lambda: tp.solve(x))
    out["tri_uniform_f64"] = {"ms": ms, "unknowns_per_s": unknowns / (ms * 1e-3),
                              "hbm_gbs_algorithmic": 16 * unknowns / (ms * 1e-3) / 1e9}
    tp.close()
    # variable diagonally dominant tri (the streams of synth.diag_dominant_tri(3, n, batch))
    ta, tc = [synth.uniform_torch(3, unknowns, -1, 1, device=dev, offset=k * unknowns) for k in range(2)]
    u = synth.uniform_torch(3, unknowns, 0, 1, device=dev, offset=2 * unknowns)
    tb = (1.5 + 0.5 * u) * (ta.abs() + tc.abs())
    del u
    tq = chx.TriPlan(n, [ta, tb, tc], batch, mode=chx.COEF_PER_SYSTEM)
    ms_f = timeit(lambda: tq.refactor([ta, tb, tc]))
    ms_s = timeit(lambda: tq.solve(x))
    out["tri_per_system_f64"] = {"ms_factor": ms_f, "ms_solve": ms_s,
                                 "unknowns_per_s_rewrite": unknowns / ((ms_f + ms_s) * 1e-3)}
    tq.close()
    return out


def bench_ch1d(dev, steps=20):
    """Batched 1D Cahn-Hilliard (Sec. 6.2.3): 2^20 simulations of N = 256, dt = 0.1 dx, FP64."""
    import torch

    import paper_2101_06550_gb300 as chx

    n, batch, l, gamma = 256, 1 << 20, 2 * np.pi, 0.01
    dt = 0.1 * l / n
    c = synth.uniform_torch(5, n * batch, -0.1, 0.1, device=dev)
    plan = chx.Ch1DPlan(n, batch, l, gamma, dt)
    plan.step(c, 3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plan.step(c, steps)  # 2 GiB of state per step: larger than L2
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    plan.sync_status()
    pts = n * batch
    return {"sims": batch, "n": n, "ms_per_step": ms, "value": pts / (ms * 1e-3), "unit": "grid-pt-steps/s",
            "fp64_gops": 14 * pts / (ms * 1e-3) / 1e9, "hbm_gbs_algorithmic": 16 * pts / (ms * 1e-3) / 1e9}


def bench_cn1d(dev, steps=100, rewrite_steps=20):
    """The paper's batched solver benchmarks (Sec. 4.3, Sec. 5.3): Crank-Nicolson
    hyperdiffusion (pentadiagonal) and diffusion (tridiagonal) on 65536 identical-shape
    systems of 1024 unknowns, L = kappa = 1, in the Constant (factor once) and Rewrite
    (reset + refactorise every system every step) variants, FP64."""
    import torch

    import paper_2101_06550_gb300 as chx

    n, batch = 1024, 1 << 16
    # FP64 operations per unknown and step as implemented (C^{n+1} = 2 A^{-1} C^n - C^n):
    # forward sweep + backward sweep + the final 2u - C
    ops = {4: 5 + 4 + 1, 2: 3 + 2 + 1}
    out = {"n": n, "systems": batch, "unit": "unknown-steps/s"}
    for order, name, dt in ((4, "hyperdiffusion_penta", 1e-8), (2, "diffusion_tri", 1e-5)):
        x = np.arange(n) / n
        c = torch.from_numpy(np.cos(4 * np.pi * x)).to(dev)[:, None].repeat(1, batch).reshape(-1).contiguous()
        res = {"dt": dt}
        for rewrite in (False, True):
            plan = chx.CN1DPlan(order, n, batch, 1.0, 1.0, dt, rewrite)
            k = rewrite_steps if rewrite else steps
            plan.step(c, 3)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.step(c, k)  # 512 MiB of state per step: larger than L2
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / k
            plan.sync_status()
            plan.close()
            pts = n * batch
            r = {"ms_per_step": ms, "value": pts / (ms * 1e-3)}
            if not rewrite:
                r["fp64_gops"] = ops[order] * pts / (ms * 1e-3) / 1e9
            res["rewrite" if rewrite else "constant"] = r
        res["rewrite_over_constant_time"] = res["rewrite"]["ms_per_step"] / res["constant"]["ms_per_step"]
        out[name] = res
        del c
        torch.cuda.empty_cache()
    return out


def bench_cook(dev, steps=50):
    """Cahn-Hilliard-Cook runs (Sec. 7.7) on the 2048^2 workload: C = 0 initially,
    sigma = 1e-14, fresh Philox + Box-Muller deviates every step (drawn inside the FP64
    right-hand-side pass), FP64 step.  deviates_ms_per_step times the standalone
    deviate kernel for comparison."""
    import torch

    import paper_2101_06550_gb300 as chx

    n, l, gamma, dt = 2048, 2 * np.pi, 0.005, 5e-4
    plan = chx.ChPlan(n, n, l, l, gamma, dt)
    cn = torch.zeros(n * n, dtype=torch.float64, device=dev)
    cp = torch.zeros_like(cn)
    work = plan.alloc_work(dev)
    rho = torch.empty(2 * n * n, dtype=torch.float64, device=dev)
    plan.cook_run(cn, cp, work, rho, 3, 1e-14, seed=7)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plan.cook_run(cn, cp, work, rho, steps, 1e-14, seed=7, step0=3)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    a.record()
    for k in range(steps):
        chx.noise_normals(rho, n, n, 7, 0, k)
    b.record()
    torch.cuda.synchronize()
    ms_dev = a.elapsed_time(b) / steps
    plan.sync_status()
    pts = n * n
    return {"n": n, "sigma": 1e-14, "ms_per_step": ms, "value": pts / (ms * 1e-3), "unit": "grid-pt-steps/s",
            "deviates_ms_per_step": ms_dev, "max_abs_c": float(cn.abs().max())}


def ensemble_sims(count=512, seed=11):
    """Uneven ensemble: n uniform in {128, 256, 512, 1024}, gamma in {0.005, 0.01, 0.02}."""
    u = synth.uniform(seed, 2 * count, 0.0, 1.0).reshape(2, count)
    sizes = np.array([128, 256, 512, 1024])[np.minimum((u[0] * 4).astype(int), 3)]
    gammas = np.array([0.005, 0.01, 0.02])[np.minimum((u[1] * 3).astype(int), 2)]
    return [(int(sizes[k]), float(gammas[k]), 1000 + k) for k in range(count)]


def bench_ensemble(dev, precision, steps, warmup, count=512, long_steps=2000):
    """The uneven ensemble (512 simulations, n in {128, ..., 1024}, FP32+refine): one
    ensemble step advances every simulation with the packed phase launches; the
    schedule and the segment counts are autotuned first.  Grid-pt-steps/s over
    `steps` steps, then the run continued to `long_steps` steps with its accuracy
    (per grid size: one FP32+refine step from the FP64 state of two simulations
    against the FP64 step, the ensemble trajectories against FP64 single plans,
    and mass drift), and the plain per-simulation FP64 step as the baseline."""
    import torch

    import paper_2101_06550_gb300 as chx

    dx, dt = 2 * np.pi / 256, 1e-3
    sims = ensemble_sims(count)
    ens = chx.Ensemble(dt, precision)
    by_n = {}
    for n, g, sd in sims:
        by_n.setdefault(n, []).append((g, sd))
    gids = {}
    for n, lst in sorted(by_n.items()):
        gid = ens.group_create(n, n * dx, lst[0][0], len(lst))
        gids[n] = gid
        for slot, (g, sd) in enumerate(lst):
            c0 = synth.uniform_torch(sd, n * n, -0.1, 0.1, device=dev)
            ens.load(gid, slot, c0, None, g)
        ens.set_active(gid, len(lst))
    mass0 = {}
    for n, gid in gids.items():
        for slot in (0, 1):
            x = torch.empty(n * n, dtype=torch.float64, device=dev)
            ens.read(gid, slot, x)
            mass0[(n, slot)] = (float(x.sum()), float(x.abs().sum()))
    tuned = {n: ens.autotune(gid, 2) for n, gid in gids.items()}
    sched = ens.tune_schedule(2) if precision == chx.PREC_F32_REFINE else None
    ens.step(max(2, warmup))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ens.step(steps)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ens.sync_status()
    pts = sum(n * n for n, _, _ in sims)
    res = {"sims": count, "grid_pts": pts, "steps": steps, "ms_per_ensemble_step": ms / steps,
           "value": pts * steps / (ms * 1e-3), "unit": "grid-pt-steps/s", "segments": tuned,
           "hbm_bytes": ens.bytes_used}
    if sched is not None:
        res["schedule"] = dict(ens.schedule_info(), tuned=sched,
                               launches_per_step="3 persistent phase launches (rhs, x, y) over all groups")
    # continue to long_steps steps, then the accuracy at that length
    done = max(2, warmup) + steps
    t0 = time.perf_counter()
    ens.step(max(0, long_steps - done))
    torch.cuda.synchronize()
    res["long_run"] = {"steps": long_steps, "wall_s": time.perf_counter() - t0 + ms * 1e-3}
    acc = {}
    for n, lst in sorted(by_n.items()):
        rows = []
        for slot in (0, 1):
            g, sd = lst[slot]
            x = torch.empty(n * n, dtype=torch.float64, device=dev)
            ens.read(gids[n], slot, x)
            m, sa = mass0[(n, slot)]
            p64 = chx.ChPlan(n, n, n * dx, n * dx, g, dt)
            c = synth.uniform_torch(sd, n * n, -0.1, 0.1, device=dev)
            pc = c.clone()
            w = p64.alloc_work(dev)
            p64.step(c, pc, w, long_steps)
            # one step of each precision from the FP64 state
            p32 = chx.ChPlan(n, n, n * dx, n * dx, g, dt, chx.PREC_F32_REFINE)
            e, f = c.clone(), pc.clone()
            p32.step(e, f, p32.alloc_work(dev), 1)
            p64.step(c, pc, w, 1)
            torch.cuda.synchronize()
            rows.append({"slot": slot, "gamma": g,
                         "per_step_rel_err_vs_fp64": float((e - c).abs().max() / c.abs().max()),
                         "trajectory_rel_err_vs_fp64": float((x - pc).abs().max() / pc.abs().max()),
                         "mass_drift_rel_to_sum_abs_c": abs(float(x.sum()) - m) / sa})
            p64.close()
            p32.close()
        acc[n] = rows
    res["accuracy_at_long_steps"] = acc
    ens.close()
    # the plain per-simulation FP64 step on the same GPU: each simulation advanced
    # by its own ch_step plan, one after another (measured step time per size and gamma)
    t_step = {}
    for n in sorted(by_n):
        for g in sorted({gg for gg, _ in by_n[n]}):
            plan = chx.ChPlan(n, n, n * dx, n * dx, g, dt)
            c = synth.uniform_torch(1, n * n, -0.1, 0.1, device=dev)
            pc = c.clone()
            w = plan.alloc_work(dev)
            plan.step(c, pc, w, 3)
            torch.cuda.synchronize()
            a.record()
            plan.step(c, pc, w, 20)
            b.record()
            torch.cuda.synchronize()
            t_step[(n, g)] = a.elapsed_time(b) / 20
            plan.close()
    serial_ms = sum(t_step[(n, g)] for n, lst in by_n.items() for g, _ in lst)
    res["per_simulation_fp64_baseline"] = {"ms_per_ensemble_step": serial_ms, "value": pts / (serial_ms * 1e-3),
                                           "step_ms_by_n_gamma": {f"{n}/{g}": v for (n, g), v in t_step.items()},
                                           "kind": "one FP64 ch_step plan per simulation, run in turn"}
    res["speedup_vs_per_simulation_fp64"] = serial_ms / (ms / steps)
    return res


def bench_coarsening_stats(dev, sims=1024, samples=20, every=10):
    """The statistics workload of Sec. 7.3.2: a batch of 1024 simulations on the
    2 pi x 2 pi domain (256^2, gamma = 0.01, dt = 0.1 dx, symmetric U[-0.1, 0.1]
    mixtures, FP64), the observables (mass, F, s, k1) of every simulation sampled
    every `every` steps on the device and beta = -(t/F) dF/dt formed per
    simulation at the end."""
    import torch

    import paper_2101_06550_gb300 as chx

    n, l, gamma = 256, 2 * np.pi, 0.01
    dt = 0.1 * l / n
    ens = chx.Ensemble(dt, chx.PREC_F64)
    gid = ens.group_create(n, l, gamma, sims)
    for s in range(sims):
        ens.load(gid, s, synth.uniform_torch(5000 + s, n * n, -0.1, 0.1, device=dev))
    ens.set_active(gid, sims)
    obs = torch.empty(samples, sims, 4, dtype=torch.float64, device=dev)
    ens.step(2)
    ens.observables(gid, obs[0], with_k1=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(samples):
        ens.step(every)
        ens.observables(gid, obs[k], with_k1=True)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ens.sync_status()
    t = (2 + every * (1 + np.arange(samples))) * dt
    F = obs[:, :, 1].cpu().numpy()
    beta = np.stack([chx.coarsening_rate(t, F[:, s]) for s in range(sims)], axis=1)
    steps = samples * every
    pts = sims * n * n
    res = {"sims": sims, "n": n, "steps": steps, "samples": samples, "ms_per_ensemble_step": ms / steps,
           "value": pts * steps / (ms * 1e-3), "unit": "grid-pt-steps/s", "t_end": float(t[-1]),
           "beta_median_last": float(np.median(beta[-1])),
           "s_median_last": float(np.median(obs[-1, :, 2].cpu().numpy())),
           "k1_median_last": float(np.median(obs[-1, :, 3].cpu().numpy())),
           "mass_drift_max": float(np.max(np.abs(
               obs[-1, :, 0].cpu().numpy() - obs[0, :, 0].cpu().numpy())))}
    ens.close()
    return res


def serial_fp64_serving(dev, reqs, dx, dt, time_limit=900.0):
    """The serial per-request FP64 baseline, run for real on the same GPU: requests
    in arrival order, each starting at its arrival or when the previous one is
    done, advanced alone by its own FP64 ch_step plan; latency from arrival to its
    result on the host (host clock)."""
    import torch

    import paper_2101_06550_gb300 as chx

    t0 = time.perf_counter()
    lat, work, done = [], 0, 0
    for r in sorted(reqs, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now > time_limit:
            break
        if now < r.arrival:
            time.sleep(r.arrival - now)
        plan = chx.ChPlan(r.n, r.n, r.n * dx, r.n * dx, r.gamma, dt)
        c = synth.uniform_torch(r.seed, r.n * r.n, -0.1, 0.1, device=dev)
        pc = c.clone()
        plan.step(c, pc, plan.alloc_work(dev), r.steps)
        c.cpu()
        lat.append(time.perf_counter() - t0 - r.arrival)
        work += r.n * r.n * r.steps
        done += 1
        plan.close()
    makespan = time.perf_counter() - t0
    lat = np.array(lat)
    return {"completed": done, "submitted": len(reqs), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "makespan_s": makespan,
            "grid_pt_steps_per_s": work / makespan,
            "kind": "measured: one FP64 ch_step plan per request, FIFO over the same arrivals, host-clock latency"}


SERVE_FILL_POINTS = 2 * 2048 * 2048  # admitted grid points that fill the GPU
SERVE_TICK_MS = 20.0


def bench_serving(dev, count, rate, precision, serial=True):
    """Poisson arrivals of the request mix (n log-uniform in [128, 2048], 500-5000
    steps, gamma in [0.005, 0.02]) served by continuous batching; latency
    percentiles, throughput, and the serial FP64 baseline on the same arrivals."""
    import paper_2101_06550_gb300 as chx
    from paper_2101_06550_gb300 import serving

    dx, dt = 2 * np.pi / 256, 1e-3
    reqs = serving.poisson_requests(count, rate, seed=7)
    srv = serving.Server(dt, dx, precision=precision, hbm_budget=96 << 30, capacity=16, chunk=100,
                         keep_results=False, fill_points=SERVE_FILL_POINTS, tick_ms=SERVE_TICK_MS)
    stats = serving.serve(reqs, srv, time_limit=900)
    offered = sum(r.n * r.n * r.steps for r in reqs) / max(reqs[-1].arrival, 1e-9)
    stats["offered_grid_pt_steps_per_s"] = offered
    stats["arrival_rate_per_s"] = rate
    stats["precision"] = "f32+f64-residual" if precision == chx.PREC_F32_REFINE else "f64"
    stats["admission"] = {"fill_points": SERVE_FILL_POINTS, "tick_ms": SERVE_TICK_MS, "capacity_per_size": 16}
    srv.ens.close()
    if serial:
        stats["serial_fp64_baseline"] = serial_fp64_serving(dev, reqs, dx, dt)
    return stats


def serving_suite(dev, count, rate):
    """The burst at the given arrival rate, then the same mix at a sustainable rate
    (60% of the throughput the burst achieved), each beside the serial baseline."""
    import paper_2101_06550_gb300 as chx
    from paper_2101_06550_gb300 import serving

    import torch

    out = {"serving": bench_serving(dev, count, rate, chx.PREC_F32_REFINE)}
    torch.cuda.empty_cache()
    mix = serving.poisson_requests(count, 1.0, seed=7)
    work = np.mean([r.n * r.n * r.steps for r in mix])
    steady = 0.6 * out["serving"]["grid_pt_steps_per_s"] / work
    out["serving_steady"] = bench_serving(dev, count, steady, chx.PREC_F32_REFINE)
    torch.cuda.empty_cache()
    return out


def kernel_case(args, local_rank):
    """The headline workload's step at one precision, W + K one-step calls and
    nothing else: the program ncu captures of single kernels run."""
    import torch

    import paper_2101_06550_gb300 as chx

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if args.kernel_case == "ens":
        dx, dt = 2 * np.pi / 256, 1e-3
        ens = chx.Ensemble(dt, chx.PREC_F32_REFINE)
        by_n = {}
        for n, g, sd in ensemble_sims(512):
            by_n.setdefault(n, []).append((g, sd))
        for n, lst in sorted(by_n.items()):
            gid = ens.group_create(n, n * dx, lst[0][0], len(lst))
            for slot, (g, sd) in enumerate(lst):
                ens.load(gid, slot, synth.uniform_torch(sd, n * n, -0.1, 0.1, device=dev), None, g)
            ens.set_active(gid, len(lst))
        ens.step(args.warmup + args.steps)
        torch.cuda.synchronize()
        ens.sync_status()
        print(json.dumps({"kernel_case": "ens", "steps": args.warmup + args.steps, "info": ens.schedule_info()}))
        ens.close()
        return
    prec = chx.PREC_F64 if args.kernel_case == "fp64" else chx.PREC_F32_REFINE
    plan = chx.ChPlan(N, N, LX, LX, GAMMA, DT, prec)
    cn = torch.from_numpy(synth.field(SEED, N, N, -0.05, 0.05)).to(dev)
    cp = cn.clone()
    work = plan.alloc_work(dev)
    for _ in range(args.warmup + args.steps):
        plan.step(cn, cp, work, 1)
    torch.cuda.synchronize()
    plan.sync_status()
    print(json.dumps({"kernel_case": args.kernel_case, "steps": args.warmup + args.steps,
                      "max_abs_c": float(cn.abs().max())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chx", choices=["chx", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--no-extras", action="store_true", help="skip the solver / ensemble / serving sub-benchmarks")
    ap.add_argument("--ens-steps", type=int, default=20)
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving benchmarks (burst and sustainable rate) and print their JSON")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--kernel-case", choices=["fp64", "fp32", "ens"],
                    help="untimed: run --warmup + --steps single steps of the headline workload at that precision "
                         "(ens: ensemble steps of the 512-simulation FP32+refine ensemble, untuned) and exit; "
                         "the programs ncu captures are taken on")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.kernel_case:
        kernel_case(args, local_rank)
    elif args.serve_only:
        import torch

        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        out = serving_suite(dev, args.serve_requests, args.serve_rate)
        if rank == 0:
            print(json.dumps({"serving_only": True, "requests": args.serve_requests, **out}))
    else:
        run_chx(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
