"""Continuous-batching server for whole Cahn-Hilliard simulations.

Requests (grid n, step count, gamma, seed) arrive over time.  Each is admitted
into a slot of the ensemble group for its grid size as soon as a slot and HBM
budget are free; all admitted simulations advance together (one graph-captured
``ens_step`` per tick: the packed phase launches of an FP32 + refinement
ensemble, or one graph branch per group in FP64), so requests that arrive while
others run join the running batch instead of waiting for it to drain.

Two limits keep the tail short.  Admission stops while the admitted grid
points already fill the GPU (``fill_points``; a request is always admitted when
nothing runs), so a large request keeps most of the GPU instead of being
shared among everything that arrived -- requests that would not speed up the
batch wait in FIFO order.  A tick advances every active simulation by the
smallest remaining step count, capped so that a tick lasts about
``tick_ms`` by the measured per-point step time, so arrivals are admitted and
finished results harvested promptly.  The thesis motivates the workload
(batches of 2D simulations for growth-rate statistics, Sec. 7.3.2); it has no
serving layer.

This module is host-side scheduling only: all arithmetic runs in ``libchx.so``.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from ._chx import ChxError, Ensemble, PREC_F64


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    steps: int
    gamma: float
    seed: int
    arrival: float  # seconds after the server starts
    admitted: Optional[float] = None
    done: Optional[float] = None
    remaining: int = 0
    result: Optional[object] = None  # host tensor with C^{steps}

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class Server:
    """Admission by HBM budget, per-size groups with per-slot gamma, continuous batching."""

    def __init__(self, dt: float, dx: float, precision: int = PREC_F64, hbm_budget: int = 0, capacity: int = 16,
                 chunk: int = 100, keep_results: bool = True, device: str = "cuda",
                 make_ic: Optional[Callable[[Request], object]] = None, autotune: bool = False,
                 fill_points: int = 0, tick_ms: float = 0.0):
        import torch

        self.torch = torch
        self.dt, self.dx = dt, dx
        self.capacity, self.chunk = capacity, chunk
        self.fill_points = fill_points  # 0: no limit on admitted grid points
        self.tick_ms = tick_ms          # 0: ticks of up to `chunk` steps
        self.ns_per_point = None        # measured step time per grid point (tick_ms)
        self.keep_results = keep_results
        self.device = device
        self.autotune = autotune
        self.ens = Ensemble(dt, precision, hbm_budget)
        self.group_of: Dict[int, int] = {}  # n -> group id
        self.active: Dict[int, List[Request]] = collections.defaultdict(list)
        self.make_ic = make_ic or self._default_ic
        self.stream = torch.cuda.current_stream()
        self.ticks = 0
        self.pt_steps = 0

    def _default_ic(self, req: Request):
        import synth

        return synth.uniform_torch(req.seed, req.n * req.n, -0.1, 0.1, device=self.device)

    def _group(self, n: int) -> Optional[int]:
        gid = self.group_of.get(n)
        if gid is not None:
            return gid
        try:
            gid = self.ens.group_create(n, n * self.dx, 0.01, self.capacity)
        except ChxError as e:
            if e.status != -4:  # CHX_ENOMEM: over the HBM budget; anything else is a real error
                raise
            if not self._evict_idle():
                return None
            try:
                gid = self.ens.group_create(n, n * self.dx, 0.01, self.capacity)
            except ChxError as e2:
                if e2.status != -4:
                    raise
                return None
        self.group_of[n] = gid
        return gid

    def _evict_idle(self) -> bool:
        idle = [n for n, g in self.group_of.items() if not self.active[g]]
        for n in idle:
            g = self.group_of.pop(n)
            self.ens.group_destroy(g)
            self.active.pop(g, None)
        return bool(idle)

    def active_points(self) -> int:
        return sum(r.n * r.n for reqs in self.active.values() for r in reqs)

    def try_admit(self, req: Request, now: float) -> bool:
        if self.fill_points and self.busy() and self.active_points() + req.n * req.n > self.fill_points:
            return False
        gid = self._group(req.n)
        if gid is None or len(self.active[gid]) >= self.capacity:
            return False
        slot = len(self.active[gid])
        c0 = self.make_ic(req)
        self.ens.load(gid, slot, c0, None, req.gamma, stream=self.stream)
        req.remaining = req.steps
        req.admitted = now
        self.active[gid].append(req)
        self.ens.set_active(gid, len(self.active[gid]))
        if self.autotune and slot == 0:
            self.ens.autotune(gid, 2, stream=self.stream)
        return True

    def busy(self) -> bool:
        return any(self.active.values())

    def tick(self, clock: Callable[[], float]) -> List[Request]:
        """Advance every active simulation; returns the requests that finished."""
        live = [r for reqs in self.active.values() for r in reqs]
        if not live:
            return []
        k = min(min(r.remaining for r in live), self.chunk)
        if self.tick_ms and self.ns_per_point:
            per_step_ms = self.ns_per_point * sum(r.n * r.n for r in live) * 1e-6
            k = max(1, min(k, int(self.tick_ms / max(per_step_ms, 1e-6))))
            if k > 1 and k % 2:
                k -= 1  # whole captured step pairs
        t_tick = time.perf_counter()
        self.ens.step(k, stream=self.stream)
        self.ticks += 1
        if self.tick_ms:
            self.stream.synchronize()
            pts = sum(r.n * r.n for r in live) * k
            est = (time.perf_counter() - t_tick) * 1e9 / max(pts, 1)
            self.ns_per_point = est if self.ns_per_point is None else 0.7 * self.ns_per_point + 0.3 * est
        finished = []
        for gid, reqs in self.active.items():
            for r in reqs:
                r.remaining -= k
                self.pt_steps += k * r.n * r.n
            done_slots = [s for s, r in enumerate(reqs) if r.remaining == 0]
            for s in sorted(done_slots, reverse=True):
                r = reqs[s]
                if self.keep_results:
                    out = self.torch.empty(r.n * r.n, dtype=self.torch.float64).pin_memory()
                    self.ens.read(gid, s, out, None, stream=self.stream)
                    r.result = out
                last = len(reqs) - 1
                if s != last:
                    self.ens.move(gid, last, s, stream=self.stream)
                    reqs[s] = reqs[last]
                reqs.pop()
                finished.append(r)
            if done_slots:
                self.ens.set_active(gid, len(reqs))
        if finished:
            self.stream.synchronize()
            now = clock()
            for r in finished:
                r.done = now
        return finished


def serve(requests: List[Request], server: Server, time_limit: float = 600.0) -> Dict[str, float]:
    """Runs the arrival process in real time; returns latency percentiles and throughput."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting: collections.deque = collections.deque()
    t0 = time.perf_counter()

    def clock():
        return time.perf_counter() - t0

    while pending or waiting or server.busy():
        now = clock()
        if now > time_limit:
            break
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        progressed = True
        while waiting and progressed:
            progressed = server.try_admit(waiting[0], now)
            if progressed:
                waiting.popleft()
        if not server.busy():
            if pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - clock())))
            elif waiting:
                raise RuntimeError("a waiting request can never be admitted (HBM budget too small for it)")
            continue
        server.tick(clock)
    server.stream.synchronize()
    makespan = clock()
    lat = np.array([r.latency for r in requests if r.latency is not None])
    work = sum(r.n * r.n * r.steps for r in requests if r.done is not None)
    return {
        "completed": int(len(lat)),
        "submitted": len(requests),
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_s": float(lat.mean()) if len(lat) else None,
        "makespan_s": makespan,
        "grid_pt_steps_per_s": work / makespan if makespan > 0 else None,
        "ticks": server.ticks,
    }


def poisson_requests(count: int, rate: float, seed: int, n_min: int = 128, n_max: int = 2048,
                     steps_lo: int = 500, steps_hi: int = 5000, g_lo: float = 0.005, g_hi: float = 0.02) -> List[Request]:
    """Seeded request stream: exponential inter-arrivals (mean 1/rate); n log-uniform
    in [n_min, n_max] rounded to a multiple of 32; steps uniform integers; gamma uniform."""
    import synth

    u = synth.uniform(seed, 4 * count, 0.0, 1.0).reshape(4, count)
    inter = -np.log1p(-u[0]) / rate
    arrivals = np.cumsum(inter)
    n = np.exp(np.log(n_min) + u[1] * (np.log(n_max) - np.log(n_min)))
    n = np.clip((np.round(n / 32) * 32).astype(int), n_min, n_max)
    steps = (steps_lo + np.floor(u[2] * (steps_hi - steps_lo + 1))).astype(int)
    gamma = g_lo + u[3] * (g_hi - g_lo)
    return [Request(rid=k, n=int(n[k]), steps=int(steps[k]), gamma=float(gamma[k]), seed=1000 + k,
                    arrival=float(arrivals[k])) for k in range(count)]
