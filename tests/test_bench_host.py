"""Host-side logic of bench.py on CPU: the multi-rank timing aggregation
(world size 2 over gloo, the N > 1 replica path), the clock parser, the
launch counts and the host-core oracle baseline of the batch and serve legs."""
from __future__ import annotations

import datetime
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    slowest = bench.allreduce_max(w, 1.0 + rank)          # rank 1 is the slowest
    out[rank] = (slowest, bench.aggregate(w, 1000, 10, slowest))
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    # both ranks see the max time; value counts every rank's sites
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 2.0
    assert value == pytest.approx(2 * 1000 * 10 / (2.0 * 1e9))


def test_clock_parser_keeps_only_the_timed_window():
    import bench
    t0 = datetime.datetime(2026, 12, 3, 14, 5, 11).timestamp()
    lines = [
        "2026/12/03 14:05:10.000, 300, 2070, 90, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 14:05:11.100, 1965, 2070, 800, Not Active, Not Active, Not Active, Active",
        "2026/12/03 14:05:11.120, 2070, 2070, 810, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 14:05:13.000, 300, 2070, 90, Active, Not Active, Not Active, Not Active",
    ]
    c = bench.Clocks.parse("\n".join(lines), t0, t0 + 1.0)
    assert c["samples"] == 2 and c["sm_mhz"] == pytest.approx(2017.5)
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.Clocks.parse("", t0, t0 + 1)["samples"] == 0


def test_batch_launch_count():
    """The gpu_launches claim of the batch lines: labels (one per model under
    label layout 0, one under layout 1), merge, compression, apply, one small
    kernel per model with one-CTA members, the step counter."""
    import bench
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import inputs
    ising, potts = inputs.ISING, inputs.POTTS
    big = [(ising, 2, 1024, 2, 2.0, 1), (potts, 2, 512, 3, 1.0, 2)]
    small = [(ising, 2, 32, 2, 2.0, 3), (potts, 2, 90, 4, 0.9, 4), (ising, 2, 100, 2, 2.0, 5)]
    assert bench.batch_launches(big, 0) == 2 + 3 + 1
    assert bench.batch_launches(big, 1) == 1 + 3 + 1
    # the grid form (bit 1) launches the same kernels; the merge split by
    # axis (bit 2) launches one merge per axis
    assert bench.batch_launches(big, 2) == 2 + 3 + 1
    assert bench.batch_launches(big, 3) == 1 + 3 + 1
    assert bench.batch_launches(big, 4) == 2 + 4 + 1
    assert bench.batch_launches([(ising, 3, 64, 2, 4.5, 7)], 5) == 1 + 5 + 1
    # Ising L = 100 (10000 sites) is tiled, Potts L = 90 (8100) and Ising L = 32 are one-CTA
    assert bench.batch_launches(small, 0) == 1 + 3 + 2 + 1
    assert bench.batch_launches([(ising, 3, 16, 2, 4.5, 6)], 0) == 0 + 0 + 1 + 1
    assert bench.batch_launches([(ising, 3, 17, 2, 4.5, 6)], 0) == 1 + 3 + 0 + 1


def test_workload_recipes():
    """The seeded batch recipes stay within their stated ranges."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import inputs
    for specs, lo, hi in ((inputs.ragged_batch(256, 1003), 32, 1024), (inputs.small_batch(256, 1005), 16, 90)):
        assert len(specs) == 256
        for model, dim, L, q, T, seed in specs:
            assert dim == 2 and lo <= L <= hi and q in (2, 3, 4) and seed > 0
            tc = inputs.TC_2D_ISING if model == inputs.ISING else inputs.tc_2d_potts(q)
            assert 0.8 * tc <= T <= 1.2 * tc
    assert inputs.small_batch(8, 7) == inputs.small_batch(8, 7)


def test_host_core_oracle_baseline():
    """The batch/serve legs' oracle baseline: independent jobs on a spawn
    pool over the host cores, their site updates summed over its wall time."""
    import bench
    specs = [(0, 2, 32, 2, 2.269185, 11 + k, 2) for k in range(3)] + [(1, 2, 24, 3, 0.994973, 5, 2)]
    out = bench.cpu_baseline_jobs(specs, "four small jobs")
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    assert "M site updates" in out["sample"] and out["unit"] == bench.UNIT
