"""Continuous-batching server for many solves on one GPU.

Requests (grid, eps, Ma, number of steps, initial velocity/pressure) arrive
over time.  The server keeps every admitted solve resident in HBM inside one
batch handle; each round it

  1. admits arrived requests in arrival order while a slot is free and the
     resident workspaces stay within the HBM budget,
  2. advances every resident solve by up to `chunk` IMEX steps, each by no
     more than it still needs (ap_dvm_step_slots: a solve that is done sits
     out the round's remaining steps), all solves in each kernel launch,
     replayed from a CUDA graph,
  3. retires the solves that are done: their state is copied to pinned host
     memory asynchronously, the slot and the workspace are released.

A request's latency runs from its arrival to the moment its result is on the
host.  `run_alone` serves the same stream with the plain per-solve path
(one Solver at a time, first come first served) for comparison.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api


@dataclass
class Job:
    rid: int
    arrival: float                 # seconds after the start of the stream
    params: api.Params
    steps: int
    fields: tuple                  # (u1, u2, p): pinned CPU float64 tensors (ny, nx)
    admitted: float = math.nan
    done: float = math.nan
    result: torch.Tensor | None = None   # (6, ny, nx) float64 moments on the host

    @property
    def cells(self) -> int:
        return self.params.nx * self.params.ny

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    makespan: float
    cell_steps: int
    latencies: list = field(default_factory=list)
    max_resident: int = 0
    max_bytes: int = 0

    @property
    def mcells_per_s(self) -> float:
        return self.cell_steps / self.makespan / 1e6

    def pct(self, q: float) -> float:
        return float(np.percentile(np.array(self.latencies) * 1e3, q)) if self.latencies else math.nan

    def summary(self) -> dict:
        return {"requests": len(self.latencies), "p50_ms": round(self.pct(50), 2), "p99_ms": round(self.pct(99), 2),
                "value": round(self.mcells_per_s, 2), "unit": "Mcell-updates/s", "makespan_s": round(self.makespan, 3),
                "max_resident": self.max_resident, "max_hbm_bytes": self.max_bytes}


class Server:
    """Continuous batching over one ap_dvm batch handle."""

    def __init__(self, template: api.Params, capacity: int, hbm_budget: float, chunk: int = 10, tile: int | None = None):
        self.batch = api.Batch(template, capacity)
        self.batch.set_graph_steps(1)
        if tile is not None:
            self.batch.set_tile(tile)
        self.capacity = capacity
        self.budget = float(hbm_budget)
        self.chunk = chunk
        self.free = list(range(capacity))[::-1]
        self.resident = {}             # slot -> [job, remaining steps, workspace bytes]
        self.base = self.batch.workspace.numel()
        self.bytes = self.base
        self.inflight = []             # (job, host tensor, event)

    def _admit(self, job: Job, now: float) -> bool:
        need = api.Batch.instance_bytes(job.params)
        if not self.free or self.bytes + need > self.budget:
            return False
        slot = self.free.pop()
        self.batch.attach(slot, job.params)
        dev = [t.to("cuda", non_blocking=True) for t in job.fields]
        self.batch.set_equilibrium(*dev, slot=slot)
        self.resident[slot] = [job, job.steps, need]
        self.bytes += need
        job.admitted = now
        return True

    def _retire(self, slot: int):
        job, _, need = self.resident.pop(slot)
        out = self.batch.get_state(slot)
        host = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
        host.copy_(out, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream())
        self.batch.detach(slot)
        self.free.append(slot)
        self.bytes -= need
        self.inflight.append((job, host, ev))

    def _poll(self, now: float, wait: bool = False):
        keep = []
        for job, host, ev in self.inflight:
            if wait:
                ev.synchronize()
            if ev.query():
                job.result = host
                job.done = now() if callable(now) else now
            else:
                keep.append((job, host, ev))
        self.inflight = keep

    def run(self, jobs: list[Job]) -> ServeStats:
        # admission is in arrival order: a request that cannot fit even alone would hold
        # up every later one forever
        for j in jobs:
            if self.base + api.Batch.instance_bytes(j.params) > self.budget:
                raise ValueError(f"request {j.rid}: its workspace does not fit the HBM budget "
                                 f"of {self.budget:.0f} bytes even alone")
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        queue = collections.deque()
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        stats = ServeStats(0.0, sum(j.cells * j.steps for j in jobs))
        while pending or queue or self.resident or self.inflight:
            now = clock()
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while queue and self._admit(queue[0], now):
                queue.popleft()
            stats.max_resident = max(stats.max_resident, len(self.resident))
            stats.max_bytes = max(stats.max_bytes, int(self.bytes))
            if self.resident:
                c = min(self.chunk, max(r[1] for r in self.resident.values()))
                counts = {slot: min(c, r[1]) for slot, r in self.resident.items()}
                self.batch.step_slots(c, counts)
                for slot in list(self.resident):
                    self.resident[slot][1] -= counts[slot]
                    if self.resident[slot][1] == 0:
                        self._retire(slot)
            elif not self.inflight and pending:
                time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)))
            self._poll(clock, wait=not self.resident and not pending and not queue)
        torch.cuda.synchronize()
        stats.makespan = clock()
        stats.latencies = [j.latency for j in jobs]
        return stats


def run_alone(jobs: list[Job], tile: int | None = None) -> ServeStats:
    """The same request stream served one solve at a time with the plain
    per-solve path (ap_dvm_create + ap_dvm_step), first come first served."""
    t0 = time.perf_counter()
    clock = lambda: time.perf_counter() - t0
    stats = ServeStats(0.0, sum(j.cells * j.steps for j in jobs))
    for job in sorted(jobs, key=lambda j: j.arrival):
        while clock() < job.arrival:
            time.sleep(min(job.arrival - clock(), 0.01))
        job.admitted = clock()
        s = api.Solver(job.params)
        if tile is not None:
            s.set_tile(tile)
        s.set_graph_steps(1)
        s.set_equilibrium(*[t.to("cuda", non_blocking=True) for t in job.fields])
        s.step(job.steps)
        out = s.get_state()
        job.result = out.cpu()
        job.done = clock()
        stats.max_resident = 1
        stats.max_bytes = max(stats.max_bytes, s.workspace.numel())
        del s
    stats.makespan = clock()
    stats.latencies = [j.latency for j in jobs]
    return stats


def make_jobs(requests, template: api.Params, field_fn) -> list[Job]:
    """Jobs from workload requests (arrival, n, eps, steps, seed); field_fn(n, seed)
    returns the initial (u1, u2, p) as numpy arrays, dt is set per request by
    the caller's rule through field_fn's returned dt."""
    jobs = []
    for k, r in enumerate(requests):
        u1, u2, p, dt = field_fn(r.n, r.seed)
        prm = template.copy()
        prm.nx = prm.ny = r.n
        prm.eps = r.eps
        prm.dt = dt
        fields = tuple(torch.from_numpy(a).pin_memory() for a in (u1, u2, p))
        jobs.append(Job(k, r.arrival, prm, r.steps, fields))
    return jobs
