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
    orig = srv._advance

    def watched():
        nonlocal peak
        peak = max(peak, srv.used)
        orig()
    srv._advance = watched
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
