"""The serving loop's host logic on CPU, against a fake of the C ABI that
counts sweeps the way the library does (a batch call advances each member by
min(n, target - counter)): every job gets exactly its sweeps, XY jobs and
large lattices run alone, admission follows arrival order and never exceeds
the HBM budget, and a job larger than the whole budget is rejected with an
error."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class FakeSw:
    SW_ISING, SW_POTTS, SW_XY = 0, 1, 2
    SW_ERR_BAD_ARG = -1

    class SwError(Exception):
        def __init__(self, code, msg):
            super().__init__(msg)
            self.code = code

    class Handle:
        def __init__(self, model, dim, L):
            self.model, self.dim, self.L = model, dim, L
            self.counter, self.target, self.batch, self.alive = 0, 0, None, True

    class Batch:
        def __init__(self, dim):
            self.dim, self.members, self.calls = dim, [], []

    def __init__(self, budget):
        self.budget, self.live_bytes, self.peak_bytes, self.created = budget, 0, 0, []

    def sw_device_bytes(self, model, dim, L, q):
        return 10 * L ** dim

    def sw_create(self, model, dim, L, q, T, seed):
        h = self.Handle(model, dim, L)
        self.live_bytes += self.sw_device_bytes(model, dim, L, q)
        self.peak_bytes = max(self.peak_bytes, self.live_bytes)
        self.created.append(seed)
        return h

    def sw_destroy(self, h):
        if h.batch is not None:
            h.batch.members.remove(h)
        h.alive = False
        self.live_bytes -= self.sw_device_bytes(h.model, h.dim, h.L, 2)

    def sw_set_sweep_target(self, h, t):
        h.target = t

    def sw_batch_create(self, dim):
        return self.Batch(dim)

    def sw_batch_destroy(self, b):
        pass

    def sw_batch_add(self, b, h):
        assert h.model != self.SW_XY and h.dim == b.dim and h.batch is None
        h.batch = b
        b.members.append(h)

    def sw_batch_sweep(self, b, n):
        b.calls.append(n)
        for h in b.members:
            c = n if not h.target else max(0, min(n, h.target - h.counter))
            h.counter += c

    def sw_sweep(self, h, n):
        assert h.batch is None
        h.counter += n

    def sw_sync(self, h):
        pass

    def sw_query(self, h):
        return True                      # the fake's work completes at once

    def sw_batch_query(self, b):
        return True

    def sw_measure(self, h):
        return {"n_sweeps": h.counter}


def jobs(serve, specs):
    return [serve.Job(id=k, model=m, dim=d, L=L, q=2, T=1.0, seed=1000 + k, sweeps=n, arrival=0.0)
            for k, (m, d, L, n) in enumerate(specs)]


@pytest.fixture
def serve(monkeypatch):
    from paper_1403_7560_gb300 import serve as srv
    return srv


def test_every_job_gets_its_sweeps_within_the_budget(serve, monkeypatch):
    specs = [(0, 2, 64, 300), (1, 2, 100, 77), (2, 3, 16, 150), (0, 3, 20, 1000), (1, 2, 48, 64),
             (0, 2, 30, 5), (2, 3, 12, 65), (1, 3, 10, 129), (0, 2, 90, 200)]
    budget = 10 * 64 ** 2 * 3
    fake = FakeSw(budget)
    monkeypatch.setattr(serve, "sw", fake)
    s = serve.Server(budget, chunk=64)
    batches = {d: s.groups[d].batch for d in (2, 3)}
    done = s.run(jobs(serve, specs), realtime=False)
    s.close()
    assert sorted(j.id for j in done) == list(range(len(specs)))
    for j in done:
        assert j.result["n_sweeps"] == j.sweeps, j.id
        assert j.start is not None and j.finish >= j.start
    assert fake.peak_bytes <= budget
    assert fake.created == sorted(fake.created)        # admitted oldest first
    # each batch call advances by the full chunk; members stop at their targets
    assert all(b.calls and all(n == 64 for n in b.calls) for b in batches.values())


def test_a_job_larger_than_the_budget_is_rejected(serve, monkeypatch):
    fake = FakeSw(100)
    monkeypatch.setattr(serve, "sw", fake)
    s = serve.Server(10 * 8 ** 2 * 2, chunk=16)
    done = s.run(jobs(serve, [(0, 2, 64, 40), (1, 2, 8, 3), (2, 3, 4, 5)]), realtime=False)
    s.close()
    assert [j.id for j in done] == [1, 2]
    assert [j.result["n_sweeps"] for j in done] == [3, 5]
    assert [j.id for j in s.rejected] == [0] and "budget" in s.rejected[0].error
    assert fake.peak_bytes <= 10 * 8 ** 2 * 2                # never above the budget


def test_groups_advance_independently(serve, monkeypatch):
    """A group whose chunk is still running is skipped, not waited for: the
    other groups keep getting chunks meanwhile."""
    fake = FakeSw(1 << 30)
    monkeypatch.setattr(serve, "sw", fake)
    slow = {"busy_polls": 0}

    def batch_query(b):
        if b.dim == 3 and slow["busy_polls"] < 5:       # the 3D batch lags behind
            slow["busy_polls"] += 1
            return False
        return True
    fake.sw_batch_query = batch_query
    s = serve.Server(1 << 30, chunk=8, poll_s=0.0)
    b2, b3 = s.groups[2].batch, s.groups[3].batch
    done = s.run(jobs(serve, [(0, 2, 16, 64), (0, 3, 8, 16)]), realtime=False)
    s.close()
    assert sorted(j.result["n_sweeps"] for j in done) == [16, 64]
    # the 2D batch got chunks while the 3D batch's first chunk was still running
    assert len(b2.calls) == 8 and len(b3.calls) == 2


def test_large_lattices_and_xy_run_alone(serve, monkeypatch):
    """Lattices of at least solo_sites sites and XY jobs get a group of their
    own (sw_sweep on their handle); the others join their dimension's batch."""
    fake = FakeSw(1 << 30)
    monkeypatch.setattr(serve, "sw", fake)
    alone, batched = set(), set()
    sweep, add = fake.sw_sweep, fake.sw_batch_add

    def sw_sweep(h, n):
        alone.add((h.model, h.dim, h.L))
        sweep(h, n)

    def sw_batch_add(b, h):
        batched.add((h.model, h.dim, h.L))
        add(b, h)
    fake.sw_sweep, fake.sw_batch_add = sw_sweep, sw_batch_add
    s = serve.Server(1 << 30, chunk=16, solo_sites=1000)
    specs = [(0, 2, 40, 50), (0, 2, 20, 50), (1, 3, 12, 30), (1, 3, 9, 40), (2, 3, 8, 20)]
    done = s.run(jobs(serve, specs), realtime=False)
    s.close()
    assert alone == {(0, 2, 40), (1, 3, 12), (2, 3, 8)}      # 1600 and 1728 sites, and XY
    assert batched == {(0, 2, 20), (1, 3, 9)}                 # 400 and 729 sites
    assert sorted((j.id, j.result["n_sweeps"]) for j in done) == [(k, n) for k, (_, _, _, n) in enumerate(specs)]


def test_summary_percentiles(serve):
    js = jobs(serve, [(0, 2, 10, 1)] * 4)
    for k, j in enumerate(js):
        j.arrival, j.finish = 0.0, float(k + 1)
    r = serve.summary(js, 4.0)
    assert r["jobs"] == 4 and r["jobs_per_s"] == 1.0
    assert r["p50_s"] == 2.0 and r["p99_s"] == 4.0
