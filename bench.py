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


def cpu_baseline_oracle(steps: int):
    """The CPU oracle, as it stands (plain C, FP64, single thread), on `steps` full steps."""
    import oracle

    c0 = synth.field(SEED, N, N, -0.05, 0.05)
    oracle.ch_run(c0, c0, LX, LX, GAMMA, DT, 1)  # warm-up (page-in, library load)
    t0 = time.perf_counter()
    oracle.ch_run(c0, c0, LX, LX, GAMMA, DT, steps)
    dt = time.perf_counter() - t0
    return N * N * steps / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = max(1, args.steps)
    import oracle

    c0 = synth.field(SEED, N, N, -0.05, 0.05)
    cn, cp = c0.copy(), c0.copy()
    for _ in range(args.warmup):
        cn, cp = oracle.ch_step(cn, cp, LX, LX, GAMMA, DT)
    t0 = time.perf_counter()
    for _ in range(steps):
        cn, cp = oracle.ch_step(cn, cp, LX, LX, GAMMA, DT)
    el = time.perf_counter() - t0
    v = N * N * steps / el
    line = {"impl": "reference", "metric": "grid-pt-steps/s", "value": v, "unit": "grid-pt-steps/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N, N], "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "grid-pt-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{steps} full 2048^2 ADI steps after {args.warmup} warm-up steps"},
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

    def measure(precision):
        plan = chx.ChPlan(N, N, LX, LX, GAMMA, DT, precision)
        cn = c0.clone()
        cp = c0.clone()
        work = plan.alloc_work(dev)
        for _ in range(args.warmup):
            plan.step(cn, cp, work, 1)
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_read(reset=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # L2 flush between timed steps (not timed)
            evs[k][0].record(stream)
            plan.step(cn, cp, work, 1)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = plan.profile_read(reset=True)
        plan.profile(False)
        plan.sync_status()
        return ms, prof, plan, cn, cp, work

    with ClockSampler(local_rank) as clk:
        ms64, prof64, plan64, cn64, cp64, work64 = measure(chx.PREC_F64)
    ms32, prof32, plan32, _, _, _ = measure(chx.PREC_F32_REFINE)
    launches_per_step = sum(n for _, n in prof64.values()) / max(1, args.steps)

    # end to end through the public API with host buffers: H2D of both fields
    # from pinned memory, one step, D2H of the new field, every step.
    h_cn = c0.cpu().pin_memory()
    h_cp = h_cn.clone().pin_memory()
    h_out = torch.empty_like(h_cn).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        cn64.copy_(h_cn, non_blocking=True)
        cp64.copy_(h_cp, non_blocking=True)
        plan64.step(cn64, cp64, work64, 1)
        h_out.copy_(cn64, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    t = torch.tensor([ms64, ms32, e2e_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms64, ms32, e2e_ms = t.tolist()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pts = N * N
    value = world * pts * args.steps / (ms64 * 1e-3)
    peaks = _peaks()
    # dominant kernel of the FP64 step and its roofline (FP64-pipe bound)
    dom, (dom_ms, dom_n) = max(prof64.items(), key=lambda kv: kv[1][0])
    dp_ops = {"ch_rhs": 15.0, "spike_local_x": 5.0, "spike_local_y": 5.0, "ch_xfinish": 4.0, "ch_update": 6.0}
    per_launch_ms = dom_ms / max(1, dom_n)
    fp64_peak_gops = 1.90 * 152 * 2.070  # measured DFMA issue rate x SMs x max clock (G DP-ops/s)
    if dom in dp_ops:
        ach = dp_ops[dom] * pts / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp64_peak_gops, "unit": "G fp64-op/s",
                "frac": ach / fp64_peak_gops, "traffic": None, "ms_per_launch": per_launch_ms,
                "peak_source": "measured DFMA microbenchmark 1.90/clk/SM x 152 SMs x 2070 MHz"}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp64_peak_gops, "unit": "G fp64-op/s",
                "frac": None, "traffic": None, "ms_per_launch": per_launch_ms}
    cb_v, cb_t = cpu_baseline_oracle(max(1, args.cpu_steps))
    line = {
        "metric": "grid-pt-steps/s", "value": value, "unit": "grid-pt-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N, N], "precision": "fp64", "l2": "flushed between timed steps",
                   "replicas": world},
        "fp32_refine": {"value": world * pts * args.steps / (ms32 * 1e-3), "ms_per_step": ms32 / args.steps,
                        "dtype": "f32+f64-residual"},
        "roofline": roof,
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof64.items())},
        "kernels_ms_per_step_fp32_refine": {k: v[0] / args.steps for k, v in sorted(prof32.items())},
        "cpu_baseline": {"value": cb_v, "unit": "grid-pt-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.cpu_steps} full 2048^2 ADI steps, {cb_t:.1f} s"},
        "e2e": {"value": world * pts * e2e_steps / (e2e_ms * 1e-3), "unit": "grid-pt-steps/s",
                "h2d_bytes_per_step": 2 * pts * 8, "d2h_bytes_per_step": pts * 8},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk.summary(),
        "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chx", choices=["chx", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=12)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_chx(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
