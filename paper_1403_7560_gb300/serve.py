"""Serving loop: continuous batching of Swendsen-Wang simulation requests.

A request (job) is one lattice -- model, dimension, L, q, T, seed -- and a
number of measured sweeps; its result is the moments of sw_measure.

The engine keeps a set of independently advancing groups on the GPU: the
ragged batch of each dimension (its Ising/Potts jobs, one launch per phase
over all their tiles, sw_batch_*) and every job that runs alone on its own
handle and stream -- the XY jobs, and lattices of at least `solo_sites`
sites, which fill the GPU by themselves and run faster on the single-lattice
path than inside a batch.  A group gets a chunk of sweeps, and the host
polls it without blocking (sw_batch_query / sw_query).  As soon as a group's chunk is done
the engine retires its finished jobs (sw_measure, destroy), lets queued jobs
join it, and enqueues its next chunk -- so a group never waits for another
group, and requests that arrive while others run are admitted as memory
frees up.  Admission is oldest first by device footprint (sw_device_bytes)
against the HBM budget; the lattice buffers come from the library's
stream-ordered pool, so creating or destroying a job does not stall the
groups that are running.  A job whose footprint alone exceeds the budget is
rejected with an error instead of being admitted.

Each batch member stops at its own sweep count (sw_set_sweep_target), so
the batch is always advanced by a full chunk.  Results do not depend on the
mix: the random numbers are keyed by seed, sweep, site and purpose only.

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
    error: str | None = None      # set when the job was rejected

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


class _Group:
    """What the engine advances as one unit: the batch of one dimension or
    one job running alone.  `busy` is set while a chunk is enqueued."""
    __slots__ = ("key", "batch", "members", "joining", "busy")

    def __init__(self, key, batch=None):
        self.key, self.batch = key, batch
        self.members: list[_Active] = []
        self.joining: list[_Active] = []
        self.busy = False


class Server:
    """Continuous-batching engine over the C ABI (one GPU, current device)."""

    def __init__(self, budget_bytes: int, chunk: int = 64, max_active: int = 1024,
                 poll_s: float = 2e-4, solo_sites: int = 1 << 22):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.solo_sites = int(solo_sites)
        self.max_active = int(max_active)
        self.poll_s = float(poll_s)
        self.used = 0
        self.queue: list[Job] = []
        self.groups: dict = {d: _Group(d, sw.sw_batch_create(d)) for d in (2, 3)}
        self.completed: list[Job] = []
        self.rejected: list[Job] = []

    @property
    def active(self) -> list[_Active]:
        return [a for g in self.groups.values() for a in g.members + g.joining]

    def close(self):
        for g in self.groups.values():
            for a in g.members + g.joining:
                sw.sw_destroy(a.handle)
            if g.batch is not None:
                sw.sw_batch_destroy(g.batch)
        self.groups = {}

    # ------------------------------------------------------------------
    def submit(self, job: Job):
        self.queue.append(job)

    def _admit(self, now: float):
        n_active = len(self.active)
        while self.queue and n_active < self.max_active:
            job = self.queue[0]
            nbytes = sw.sw_device_bytes(job.model, job.dim, job.L, job.q)
            if nbytes == 0 or nbytes > self.budget:
                self.queue.pop(0)
                job.error = ("invalid lattice" if nbytes == 0 else
                             f"needs {nbytes} bytes of device memory, more than the whole budget "
                             f"of {self.budget}")
                job.finish = now
                self.rejected.append(job)
                continue
            if self.used + nbytes > self.budget:
                return                     # wait for memory to free up
            self.queue.pop(0)
            h = sw.sw_create(job.model, job.dim, job.L, job.q, job.T, job.seed)
            self.used += nbytes
            job.start = now
            a = _Active(job, h, nbytes)
            if job.model == sw.SW_XY or job.sites >= self.solo_sites:
                g = _Group(("solo", job.id))
                self.groups[g.key] = g
            else:
                sw.sw_set_sweep_target(h, job.sweeps)
                g = self.groups[job.dim]
            g.joining.append(a)
            n_active += 1

    def _idle(self, g: _Group) -> bool:
        if not g.busy:
            return True
        done = sw.sw_batch_query(g.batch) if g.batch is not None else sw.sw_query(g.members[0].handle)
        if done:
            g.busy = False
        return done

    def _retire(self, g: _Group, now_fn: Callable[[], float]):
        keep = []
        for a in g.members:
            if a.remaining > 0:
                keep.append(a)
                continue
            a.job.result = sw.sw_measure(a.handle)   # the group is idle: no wait
            a.job.finish = now_fn()
            sw.sw_destroy(a.handle)                  # leaves its batch first
            self.used -= a.bytes
            self.completed.append(a.job)
        g.members = keep

    def _launch(self, g: _Group):
        for a in g.joining:
            if g.batch is not None:
                sw.sw_batch_add(g.batch, a.handle)
            g.members.append(a)
        g.joining = []
        if not g.members:
            return
        if g.batch is not None:
            sw.sw_batch_sweep(g.batch, self.chunk)   # every member stops at its own target
            for a in g.members:
                a.done += min(self.chunk, a.remaining)
        else:
            a = g.members[0]
            n = min(self.chunk, a.remaining)
            sw.sw_sweep(a.handle, n)
            a.done += n
        g.busy = True

    def step(self, now_fn: Callable[[], float]) -> bool:
        """One pass of the engine: admit, then for every group whose chunk
        has completed retire its finished jobs, add the new ones and enqueue
        its next chunk.  Returns whether any group was advanced."""
        self._admit(now_fn())
        advanced = False
        for key in list(self.groups):
            g = self.groups[key]
            if not self._idle(g):
                continue
            self._retire(g, now_fn)
            if g.members or g.joining:
                self._launch(g)
                advanced = True
            elif g.batch is None:
                del self.groups[key]               # a finished solo job's group
        return advanced

    def run(self, jobs: list[Job], realtime: bool = True) -> list[Job]:
        """Serve `jobs` (their `arrival` times, seconds from now when
        realtime, else all queued at once) until every one has finished or
        been rejected; returns the finished ones."""
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
            if not self.step(now):
                time.sleep(self.poll_s)            # every group is still running its chunk
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
