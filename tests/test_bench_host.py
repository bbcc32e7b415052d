"""Host-side logic of bench.py on CPU: the multi-rank timing aggregation
(world size 2 over gloo, the N > 1 replica path) and the clock parser."""
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
