"""Serving loop (continuous batching) on the GPU: every job's result is the
same alone and in the mix; admission respects the HBM budget."""
from __future__ import annotations

import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_7560_gb300 import build, serve as srv
    build.build()
    return srv


def jobs(serve, n, seed, rate=None):
    return [serve.Job(**d) for d in inputs.served_stream(n, seed, rate=rate, max_L2=96, max_L3=20,
                                                          sweeps=(10, 70))]


def test_results_same_alone_and_in_the_mix(serve):
    mixed = jobs(serve, 18, 4242)
    assert len({(j.model, j.dim) for j in mixed}) >= 4
    from paper_1403_7560_gb300 import sw
    budget = 3 * max(sw.sw_device_bytes(j.model, j.dim, j.L, j.q) for j in mixed)
    srv = serve.Server(budget, chunk=16)
    try:
        done = srv.run(mixed, realtime=False)
    finally:
        srv.close()
    assert len(done) == len(mixed)
    alone = {j.id: j for j in serve.run_serial(jobs(serve, 18, 4242), realtime=False)}
    for j in done:
        assert j.result == alone[j.id].result, (j.id, j.model, j.dim, j.L)


def test_admission_respects_budget(serve):
    from paper_1403_7560_gb300 import sw
    js = jobs(serve, 10, 99)
    sizes = [sw.sw_device_bytes(j.model, j.dim, j.L, j.q) for j in js]
    budget = max(sizes) + min(sizes)
    srv = serve.Server(budget, chunk=8)
    peak = 0
    orig = srv._launch

    def watched(g):
        nonlocal peak
        peak = max(peak, srv.used)
        orig(g)
    srv._launch = watched
    try:
        done = srv.run(js, realtime=False)
    finally:
        srv.close()
    assert len(done) == len(js) and peak <= budget and srv.used == 0


def test_realtime_arrivals(serve):
    js = jobs(serve, 8, 5, rate=40.0)
    srv = serve.Server(1 << 32, chunk=16)
    try:
        done = srv.run(js, realtime=True)
    finally:
        srv.close()
    s = serve.summary(done, max(j.finish for j in done))
    assert s["jobs"] == 8 and all(j.latency >= 0 for j in done) and s["p99_s"] >= s["p50_s"]


def test_served_results_equal_the_oracle(serve):
    """Jobs served together in one mix (2D/3D batches, small members in
    shared memory, XY jobs on their own streams): every Ising/Potts job's
    accumulators equal the CPU oracle's run of the same job bit for bit, and
    the XY jobs' mean energy and M^2 (12 independent jobs, each one bin)
    agree with 12 oracle runs within 3 combined standard errors."""
    import math
    import numpy as np
    import oracle
    from paper_1403_7560_gb300 import sw
    exact = [(sw.SW_ISING, 2, 40, 2, 2.269185, 150), (sw.SW_ISING, 2, 100, 2, 2.3, 60),
             (sw.SW_ISING, 3, 12, 2, 4.5115, 90), (sw.SW_POTTS, 2, 50, 3, 0.994973, 120),
             (sw.SW_POTTS, 2, 72, 4, 0.910239, 80), (sw.SW_POTTS, 2, 30, 8, 0.744899, 100),
             (sw.SW_POTTS, 3, 14, 3, 1.8, 70)]
    js = [serve.Job(id=k, model=m, dim=d, L=L, q=q, T=T, seed=7000 + k, sweeps=n)
          for k, (m, d, L, q, T, n) in enumerate(exact)]
    n_xy, xy_sweeps, T_xy = 12, 400, 2.2
    js += [serve.Job(id=100 + k, model=sw.SW_XY, dim=3, L=8, q=2, T=T_xy, seed=8000 + k, sweeps=xy_sweeps)
           for k in range(n_xy)]
    srv = serve.Server(1 << 32, chunk=32)
    try:
        done = {j.id: j for j in srv.run(js, realtime=False)}
    finally:
        srv.close()
    assert len(done) == len(js)
    for k, (m, d, L, q, T, n) in enumerate(exact):
        o = oracle.Oracle(m, d, L, q, T, 7000 + k)
        try:
            o.sweep(n)
            ref = o.take_acc()
        finally:
            o.close()
        got = done[k].result
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert got[f] == ref[f], (k, f, got[f], ref[f])

    def per_job(acc):
        return [acc["sum_E"] / acc["n_sweeps"], acc["sum_M2"] / acc["n_sweeps"]]
    g = np.array([per_job(done[100 + k].result) for k in range(n_xy)])
    c = []
    for k in range(n_xy):
        o = oracle.Oracle(sw.SW_XY, 3, 8, 2, T_xy, 9000 + k)
        try:
            o.sweep(xy_sweeps)
            c.append(per_job(o.take_acc()))
        finally:
            o.close()
    c = np.array(c)
    for j in range(2):
        se = math.hypot(g[:, j].std(ddof=1), c[:, j].std(ddof=1)) / math.sqrt(n_xy)
        assert abs(g[:, j].mean() - c[:, j].mean()) < 3 * se, (j, g[:, j].mean(), c[:, j].mean(), se)
