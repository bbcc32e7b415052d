"""Serving loop: continuous batching of Swendsen-Wang simulation requests.

A request (job) is one lattice -- model, dimension, L, q, T, seed -- and a
number of measured sweeps; its result is the moments of sw_measure.  The
engine admits queued jobs, oldest first, while their device footprint
(sw_device_bytes) fits the HBM budget.  Admitted Ising/Potts jobs join the
ragged batch of their dimension, so one launch per phase advances all of
them.  XY jobs run on their own handle and stream and overlap with the
batches.  Every engine iteration advances each active job by
min(chunk, its remaining sweeps) -- one batch call of chunk sweeps per
dimension, each member stopping at its own sweep target (the job's sweep
count, sw_set_sweep_target) -- then retires finished jobs, which frees
budget for the queue.  Results do not depend on the mix: the
random numbers are keyed by seed, sweep, site and purpose only.

`run_serial` is the one-job-at-a-time plain path used as the comparison:
create, sweep, measure, destroy, in arrival order.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable

from . import sw


@dataclasses.dataclass
class Job:
    id: int
    model: int
    dim: int
    L: int
    q: int
    T: float
    seed: int
    sweeps: int
    arrival: float = 0.0          # seconds after the start of the run
    # filled in by the engine
    start: float | None = None
    finish: float | None = None
    result: dict | None = None

    @property
    def sites(self) -> int:
        return self.L ** self.dim

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class _Active:
    __slots__ = ("job", "handle", "done", "bytes")

    def __init__(self, job, handle, nbytes):
        self.job, self.handle, self.done, self.bytes = job, handle, 0, nbytes

    @property
    def remaining(self):
        return self.job.sweeps - self.done


class Server:
    """Continuous-batching engine over the C ABI (one GPU, current device)."""

    def __init__(self, budget_bytes: int, chunk: int = 64, max_active: int = 1024):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.max_active = int(max_active)
        self.used = 0
        self.queue: list[Job] = []
        self.active: list[_Active] = []
        self.batches = {2: sw.sw_batch_create(2), 3: sw.sw_batch_create(3)}
        self.completed: list[Job] = []

    def close(self):
        for a in self.active:
            sw.sw_destroy(a.handle)
        self.active.clear()
        for b in self.batches.values():
            sw.sw_batch_destroy(b)
        self.batches = {}

    # ------------------------------------------------------------------
    def submit(self, job: Job):
        self.queue.append(job)

    def _admit(self, now: float):
        while self.queue and len(self.active) < self.max_active:
            job = self.queue[0]
            nbytes = sw.sw_device_bytes(job.model, job.dim, job.L, job.q)
            if nbytes == 0:
                raise sw.SwError(sw.SW_ERR_BAD_ARG, f"job {job.id}: invalid lattice")
            if self.used + nbytes > self.budget and self.active:
                return                     # wait for memory to free up
            self.queue.pop(0)
            h = sw.sw_create(job.model, job.dim, job.L, job.q, job.T, job.seed)
            if job.model != sw.SW_XY:
                sw.sw_set_sweep_target(h, job.sweeps)
                sw.sw_batch_add(self.batches[job.dim], h)
            self.used += nbytes
            job.start = now
            self.active.append(_Active(job, h, nbytes))

    def _advance(self):
        groups: dict[int, list[_Active]] = {2: [], 3: []}
        xy = []
        for a in self.active:
            (xy if a.job.model == sw.SW_XY else groups[a.job.dim]).append(a)
        for dim, members in groups.items():
            if members:
                # every member stops at its own target
                sw.sw_batch_sweep(self.batches[dim], self.chunk)
                for a in members:
                    a.done += min(self.chunk, a.remaining)
        for a in xy:
            n = min(self.chunk, a.remaining)
            sw.sw_sweep(a.handle, n)
            a.done += n

    def _retire(self, now_fn: Callable[[], float]):
        keep = []
        for a in self.active:
            if a.remaining > 0:
                keep.append(a)
                continue
            a.job.result = sw.sw_measure(a.handle)   # waits for the job's work
            a.job.finish = now_fn()
            sw.sw_destroy(a.handle)                  # leaves its batch first
            self.used -= a.bytes
            self.completed.append(a.job)
        self.active = keep

    def _sync(self):
        # one member per batch (its stream waits for the batch) and every XY job
        seen = set()
        for a in self.active:
            key = a.job.dim if a.job.model != sw.SW_XY else ("xy", a.job.id)
            if key not in seen:
                seen.add(key)
                sw.sw_sync(a.handle)

    def step(self, now_fn: Callable[[], float]):
        """One engine iteration: admit, advance every active job, wait for
        the device, retire finished jobs."""
        self._admit(now_fn())
        if not self.active:
            return
        self._advance()
        self._sync()
        self._retire(now_fn)

    def run(self, jobs: list[Job], realtime: bool = True) -> list[Job]:
        """Serve `jobs` (their `arrival` times, seconds from now when
        realtime, else all queued at once) until every one has finished."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        t0 = time.perf_counter()
        now = (lambda: time.perf_counter() - t0)
        k = 0
        while k < len(pending) or self.queue or self.active:
            t = now()
            while k < len(pending) and (not realtime or pending[k].arrival <= t):
                self.submit(pending[k])
                k += 1
            if not self.queue and not self.active:
                time.sleep(max(0.0, pending[k].arrival - now()))   # idle until the next arrival
                continue
            self.step(now)
        return self.completed


def run_serial(jobs: list[Job], realtime: bool = True) -> list[Job]:
    """The plain path: one job at a time in arrival order."""
    t0 = time.perf_counter()
    now = (lambda: time.perf_counter() - t0)
    done = []
    for job in sorted(jobs, key=lambda j: j.arrival):
        if realtime:
            time.sleep(max(0.0, job.arrival - now()))
        job.start = now()
        h = sw.sw_create(job.model, job.dim, job.L, job.q, job.T, job.seed)
        try:
            sw.sw_sweep(h, job.sweeps)
            job.result = sw.sw_measure(h)
        finally:
            sw.sw_destroy(h)
        job.finish = now()
        done.append(job)
    return done


def summary(jobs: list[Job], wall: float) -> dict:
    lat = sorted(j.latency for j in jobs)

    def pct(p):
        if not lat:
            return None
        return lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
    su = sum(j.sites * j.sweeps for j in jobs)
    return {"jobs": len(jobs), "wall_s": wall, "jobs_per_s": len(jobs) / wall if wall > 0 else None,
            "site_updates_per_ns": su / (wall * 1e9) if wall > 0 else None,
            "p50_s": pct(0.50), "p99_s": pct(0.99)}
