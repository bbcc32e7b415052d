"""Benchmark of the Swendsen-Wang sweep on GB300.

Workload: 3D Ising, simple cubic L=256 periodic (16,777,216 sites), J=1,
K=0.2216546 (T=1/K), random start from seed 1001, 100 discarded sweeps
before timing.  One step = one measured SW sweep (Philox bonds + tile
labels, boundary merge, flip, moment reduction).  Metric: site-updates per
nanosecond = sites x steps / device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Timing: CUDA events on the library's stream around every step, the L2
flushed (a 512 MiB write) between timed steps, untimed; K steps bracketed by
a barrier and torch.cuda.synchronize(); the max over ranks.  N > 1 runs N
independent replicas (one lattice per GPU, seed 1001 + rank): the sweep of
one lattice does not shard.  The reference arm times the CPU oracle (single
thread) on the same workload, over a bounded number of sweeps.

On one GPU the same line also carries the two serving workloads: `batch`
(256 ragged 2D lattices advanced together, 500 sweeps) and `serve` (a mixed
request stream with the full size ranges -- 2D L up to 4096, 3D L up to
256, 100 to 5000 sweeps -- 48 jobs, served by continuous batching against
one job at a time, with jobs/s and p50/p99 latency).  --headline-only skips
them; --workload batch|serve runs one alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "SW site-updates/ns (3D Ising L=256) vs HBM roofline; served mix jobs/s, p50/p99"
UNIT = "site-updates/ns"
MODEL, DIM, L, Q = 0, 3, 256, 2
K_COUPLING = 0.2216546
T = 1.0 / K_COUPLING
SEED = 1001
DISCARD = 100
N_SITES = L ** DIM
WORKLOAD = {"workload": "3D Ising SW sweep, simple cubic L=256 periodic, K=0.2216546, "
                        "int8 spins, random start (seed 1001), 100 discarded sweeps, "
                        "measured sweeps (bonds+labels+flip+moments)",
            "model": "ising", "dim": 3, "L": L, "sites": N_SITES, "T": T,
            "l2": "flushed between timed steps (512 MiB write)"}

# Bytes per site per sweep of each phase (3D Ising) in the reference bytes
# model: bond (read the spin, 1 B; write the bond bits, 3/8 B) plus tile
# label (read the bond bits, 3/8 B; write the label, 4 B) for the fused
# bond+label kernel; flip (read the label, 4 B; write the spin, 1 B);
# measurement (read the spin, 1 B).  The merge touches tile faces only.
KERNEL_BYTES_PER_SITE = {"bond_label": 1 + 3 / 8 + 3 / 8 + 4, "merge": None, "flip": 4 + 1, "measure": 1}
PHASES = ["bond_label", "merge", "flip", "measure"]
# The committed ncu summary of the dominant kernel carries its DRAM bytes
# per launch, its limiter and a hash of the sources it was built from; the
# figures are reported only while the sources still hash the same.
KERNEL_PROFILE = os.path.join(ROOT, "profiles", "k_label_ising3d_L256.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1403_7560_gb300", "csrc", f)
                  for f in ("sw_label.cu", "sw_device.cuh", "sw_internal.h")]
# kernels one measured sweep launches: k_label (bonds + tile labels + the
# previous sweep's measurement), k_merge, k_compress, k_apply
KERNELS_PER_SWEEP = 4
# Reference bytes model: 10.75 B/site/sweep for 3D Ising (bond 1.375,
# tile label 4.375, flip 5), independent of the schedule.
B_REF = 10.75


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_kernel():
    """(DRAM bytes per launch, limiter, note) from the committed ncu summary
    of the labeling kernel; None figures when the summary is missing or was
    taken on other sources."""
    fields = {}
    try:
        with open(KERNEL_PROFILE) as f:
            for line in f:
                line = line.strip().lstrip("-").strip()
                for key in ("source_sha", "dram_bytes_per_launch", "limiter"):
                    if line.startswith(key + ":"):
                        fields[key] = line.split(":", 1)[1].strip().strip("`")
    except OSError:
        return None, None, "no committed ncu summary of the kernel"
    if fields.get("source_sha") != kernel_source_hash():
        return None, None, "the kernel's sources changed since the committed ncu capture"
    return float(fields["dram_bytes_per_launch"]), fields.get("limiter"), None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons; only samples
    taken between mark_start() and mark_stop() are kept."""

    FIELDS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.proc = None
        self.t0 = self.t1 = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)   # let the sampler start before the timed region
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        return self.parse(out, self.t0, self.t1)

    @classmethod
    def parse(cls, out: str, t0, t1):
        import datetime
        sm, mx, reasons, n_all = [], [], set(), 0
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            n_all += 1
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, cmax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if t0 is not None and t1 is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                continue
            sm.append(clk)
            mx.append(cmax)
            for name, v in zip(cls.FIELDS, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": [],
                    "note": f"no sample inside the timed region ({n_all} outside)"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, sites_per_rank: int, steps: int, max_seconds: float) -> float:
    """Whole-job site-updates/ns: every rank's sites x steps over the
    slowest rank's time."""
    return world * sites_per_rank * steps / (max_seconds * 1e9)


def cpu_baseline(sweeps: int = 4, warm: int = 1):
    """The oracle, single-threaded, on the same lattice: `sweeps` measured
    sweeps after `warm` untimed ones from creation (a bounded sample of the
    workload)."""
    import oracle
    o = oracle.Oracle(MODEL, DIM, L, Q, T, SEED)
    o.sweep(warm)
    t0 = time.perf_counter()
    o.sweep(sweeps)
    dt = time.perf_counter() - t0
    o.close()
    return {"value": N_SITES * sweeps / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sweeps} measured sweeps of the full L=256 lattice after {warm} untimed sweep(s) "
                      f"from the seeded start; {dt:.1f} s on one host core"}


def cpu_baseline_xy(sweeps: int = 2, warm: int = 1):
    """The oracle on the 3D XY L=256 workload (seed 1002), single-threaded:
    `sweeps` measured sweeps after `warm` untimed ones."""
    import oracle
    name, model, dim, L_, q, T_, seed, _, _ = OTHER_WORKLOADS[0]
    o = oracle.Oracle(model, dim, L_, q, T_, seed)
    o.sweep(warm)
    t0 = time.perf_counter()
    o.sweep(sweeps)
    dt = time.perf_counter() - t0
    o.close()
    n = L_ ** dim
    return {"value": n * sweeps / (dt * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sweeps} measured sweeps of the full {name} lattice after {warm} untimed sweep(s); "
                      f"{dt:.1f} s on one host core"}


def _oracle_ready(_):
    import oracle  # noqa: F401  (the worker loads the oracle library once)
    return 0


def _oracle_job(spec):
    """One job of the host-core baseline: create the oracle lattice and run
    `sweeps` sweeps; returns (site updates, seconds)."""
    import oracle
    model, dim, L_, q, T_, seed, sweeps = spec
    t0 = time.perf_counter()
    o = oracle.Oracle(model, dim, L_, q, T_, seed)
    o.sweep(sweeps)
    o.close()
    return L_ ** dim * sweeps, time.perf_counter() - t0


def cpu_baseline_jobs(specs, what):
    """The oracle on independent jobs (model, dim, L, q, T, seed, sweeps)
    across every host core: a spawn-context pool (the process has CUDA
    initialised, so no fork), started and warmed before the clock; the
    largest jobs first.  Aggregate site-updates/ns over the pool's wall
    time, lattice creation included."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    order = sorted(specs, key=lambda s: -(s[2] ** s[1]) * s[6])
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_ready, range(cores), chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, order, chunksize=1)
        wall = time.perf_counter() - t0
    su = sum(r[0] for r in res)
    return {"value": su / (wall * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}; {su / 1e6:.1f} M site updates in {wall:.1f} s on {cores} host cores"}


def batch_specs():
    import inputs
    return inputs.ragged_batch(256, 1003)


def serve_specs(args, max_l2, max_l3, max_sweeps):
    import inputs
    return inputs.served_stream(args.jobs, 1004, max_L2=max_l2, max_L3=max_l3, sweeps=(100, max_sweeps))


def leg_baselines(args, line, sweeps=3):
    """Host-core oracle baselines of the batch and serve legs in `line`."""
    if "batch" in line:
        specs = [s + (sweeps,) for s in batch_specs()]
        line["batch"]["cpu_baseline"] = cpu_baseline_jobs(
            specs, f"the 256 lattices of the ragged batch, {sweeps} sweeps each from creation")
    for key, lims in (("serve", (args.max_l2, args.max_l3, args.max_sweeps)), ("serve_small_jobs", (1024, 128, 1000))):
        if key in line:
            jobs = serve_specs(args, *lims)
            specs = [(j["model"], j["dim"], j["L"], j["q"], j["T"], j["seed"], min(sweeps, j["sweeps"])) for j in jobs]
            line[key]["cpu_baseline"] = cpu_baseline_jobs(
                specs, f"the {len(jobs)} jobs of the stream, {sweeps} sweeps each from creation (not their "
                       f"full sweep counts)")


def run_reference(args):
    # the oracle runs once, on rank 0; other ranks have nothing to do
    if int(os.environ.get("RANK", "0")) != 0:
        return
    # bounded sample: the requested warm-up sweeps (at least 3) untimed, then
    # at most ~90 s of timed oracle sweeps
    t0 = time.perf_counter()
    warm = max(args.warmup, 3)
    probe = cpu_baseline(1, warm=0)
    per = N_SITES / (probe["value"] * 1e9)
    steps = max(1, min(args.steps, int(90.0 / max(per, 1e-9))))
    base = cpu_baseline(steps, warm=warm)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": 1e3 * N_SITES / (base["value"] * 1e9),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


# The other single-lattice workloads of the measurement plan, timed briefly
# beside the headline (CUDA events per measured sweep, L2 flushed between
# sweeps): 3D XY L=256 at K=0.4541652 (seed 1002), the paper's discretised
# XY (the q=512 clock model) at the same temperature, the 2D Ising L=4096
# lattice at T=2.269185, and the small 2D Ising L=64 lattice at the same T
# (seed 1000), which is latency bound.
OTHER_WORKLOADS = [
    ("xy3d_L256", 2, 3, 256, 2, 1.0 / 0.4541652, 1002, 20, 50),
    ("clock3d_q512_L256", 3, 3, 256, 512, 1.0 / 0.4541652, 1002, 20, 50),
    ("ising2d_L4096", 0, 2, 4096, 2, 2.269185, 1000, 20, 50),
]
# reference bytes per site per sweep of the other workloads (3D XY: angle
# in + mask out, mask in + label out, label in + angle in + angle out;
# 2D Ising: spin in + 2/8 mask out, mask in + label out, label in + spin out)
B_REF_OTHER = {"xy3d_L256": 20.75, "ising2d_L4096": 10.5}
# the 2D Ising L=64 configuration as specified: 200 discarded, then 1000
# measured sweeps in one sw_sweep call (events around the call)
SMALL_WORKLOAD = ("ising2d_L64", 0, 2, 64, 2, 2.269185, 1000, 200, 1000)


def other_workloads(sw, stream, flush, rank):
    import torch
    out = {}
    for name, model, dim, L_, q, T_, seed, discard, steps in OTHER_WORKLOADS:
        h = sw.sw_create(model, dim, L_, q, T_, seed + rank)
        sw.sw_set_stream(h, stream.cuda_stream)
        sw.sw_discard(h, discard)
        sw.sw_sweep(h, 3)
        sw.sw_measure(h)
        torch.cuda.synchronize()
        ts = []
        for k in range(steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sw.sw_sweep(h, 1)
            b.record(stream)
            flush.fill_(k & 0xff)
            ts.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in ts)
        mom = sw.sw_measure(h)
        n = L_ ** dim
        out[name] = {"value": n / (ms * 1e6), "unit": UNIT, "ms_per_step": ms, "ns_per_site": ms * 1e6 / n,
                     "steps": steps, "sites": n, "T": T_, "e_per_spin": mom["e_per_spin"]}
        if name in B_REF_OTHER:
            # the reference bytes model of this workload against the measured copy bandwidth
            gbps = out[name]["value"] * B_REF_OTHER[name]
            out[name]["b_ref"] = {"bytes_per_site": B_REF_OTHER[name], "GBps": gbps, "frac": gbps / peaks()[0]}
        sw.sw_destroy(h)
    name, model, dim, L_, q, T_, seed, discard, steps = SMALL_WORKLOAD
    h = sw.sw_create(model, dim, L_, q, T_, seed + rank)
    sw.sw_set_stream(h, stream.cuda_stream)
    sw.sw_discard(h, discard)
    sw.sw_measure(h)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sw.sw_sweep(h, steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    mom = sw.sw_measure(h)
    n = L_ ** dim
    out[name] = {"value": n / (ms * 1e6), "unit": UNIT, "ms_per_step": ms, "ns_per_site": ms * 1e6 / n,
                 "steps": steps, "discarded": discard, "sites": n, "T": T_, "e_per_spin": mom["e_per_spin"],
                 "mode": "one sw_sweep call of 1000 measured sweeps (whole lattice in one CTA's shared memory)"}
    sw.sw_destroy(h)
    return out


def run_gpu(args):
    import torch
    from paper_1403_7560_gb300 import build, sw
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    h = sw.sw_create(MODEL, DIM, L, Q, T, SEED + rank)
    sw.sw_set_stream(h, stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    sw.sw_discard(h, DISCARD)
    for _ in range(max(args.warmup, 3)):
        sw.sw_sweep(h, 1)
        flush.fill_(1)
    sw.sw_measure(h)
    torch.cuda.synchronize()

    # timed region: K measured sweeps, events around each, L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark_start()
    for k in range(args.steps):
        starts[k].record(stream)
        sw.sw_sweep(h, 1)
        ends[k].record(stream)
        flush.fill_(k & 0xff)
    torch.cuda.synchronize()
    clocks.mark_stop()
    barrier(world)
    clk = clocks.stop()
    sw.sw_sync(h)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = allreduce_max(world, sum(step_ms) / 1e3)
    value = aggregate(world, N_SITES, args.steps, total_s)
    moments = sw.sw_measure(h)

    # per-kernel durations: the same steps through the event-instrumented call
    phase = np.zeros(4)
    for k in range(args.steps):
        phase += np.array(sw.sw_sweep_timed(h))
        flush.fill_(k & 0xff)
    torch.cuda.synchronize()
    phase_ms = phase / args.steps
    upd = []
    for k in range(min(args.steps, 50)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sw.sw_discard(h, 1)
        b.record(stream)
        flush.fill_(1)
        torch.cuda.synchronize()
        upd.append(a.elapsed_time(b))
    update_only = N_SITES / (statistics.mean(upd) * 1e6)

    # the paper's labeler (label equivalence) against the tile union-find on
    # the bond planes of the same sweeps, each producing canonical labels
    lab_uf, lab_le, lab_it = [], [], []
    for k in range(5):
        sw.sw_sweep(h, 1)
        flush.fill_(1)
        lab_uf.append(sw.sw_relabel(h, sw.SW_LABEL_TILE_UF, False)[1])
        flush.fill_(2)
        _, ms, it = sw.sw_relabel(h, sw.SW_LABEL_EQUIVALENCE, False)
        lab_le.append(ms)
        lab_it.append(it)
    labeling = {"planes": "bonds of 5 measured sweeps after the timed ones",
                "tile_uf_ms": statistics.mean(lab_uf),
                "label_equivalence_ms": statistics.mean(lab_le),
                "label_equivalence_iterations": statistics.mean(lab_it),
                "speedup": statistics.mean(lab_le) / statistics.mean(lab_uf)}

    secondary = other_workloads(sw, stream, flush, rank)

    # End to end through the C ABI with pinned host buffers: every step
    # uploads its input state, sweeps, and downloads the new state and the
    # step's record.  The timed loop uses the asynchronous calls (transfers
    # on the handle's copy streams, overlapping the sweeps; every step is
    # enqueued, then one wait); the synchronous calls are timed beside it.
    import ctypes
    host_in = torch.empty(N_SITES, dtype=torch.int8, pin_memory=True).numpy()
    host_out = [torch.empty(N_SITES, dtype=torch.int8, pin_memory=True).numpy() for _ in range(2)]
    sw.sw_get_spins(h, host_in)
    e2e_steps = min(args.steps, 50)
    recs = sw.record_buffer(e2e_steps)
    sw.sw_sync(h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        sw.sw_set_spins_async(h, host_in)               # H2D of the step's input state
        sw.sw_sweep(h, 1)
        sw.sw_get_spins_async(h, host_out[k & 1])       # D2H of the new state
        sw.sw_get_record_async(h, sw.sw_sweep_counter(h), recs[k])  # D2H of the step's record
    sw.sw_wait_io(h)
    e2e_s = allreduce_max(world, time.perf_counter() - t0)
    rec_bytes = ctypes.sizeof(sw.sw_record)
    e2e = {"value": aggregate(world, N_SITES, e2e_steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": N_SITES, "d2h_bytes_per_step": N_SITES + rec_bytes,
           "steps": e2e_steps,
           "mode": "sw_set_spins_async + sw_sweep + sw_get_spins_async + sw_get_record_async per step, "
                   "one sw_wait_io"}
    sync_steps = min(args.steps, 20)
    t0 = time.perf_counter()
    for _ in range(sync_steps):
        sw.sw_set_spins(h, host_in)
        sw.sw_sweep(h, 1)
        sw.sw_get_spins(h, host_out[0])
        sw.sw_get_series(h, sw.sw_sweep_counter(h), 1)
    sync_s = allreduce_max(world, time.perf_counter() - t0)
    e2e["synchronous"] = {"value": aggregate(world, N_SITES, sync_steps, sync_s), "steps": sync_steps,
                          "mode": "sw_set_spins + sw_sweep + sw_get_spins + sw_get_series per step"}

    legs = {}
    if world == 1 and not args.headline_only:
        # the ragged batch and the served stream of the same build, one GPU
        legs["batch"] = batch_leg(args, torch.cuda.Stream())   # graph capture needs a non-default stream
        legs["serve"] = serve_leg(args)
        # the same recipe with smaller jobs (2D L <= 1024, 3D L <= 128, <= 1000
        # sweeps), where most of the work is latency-bound small lattices
        legs["serve_small_jobs"] = serve_leg(args, 1024, 128, 1000)

    if rank == 0:
        peak, peak_kind = peaks()
        dom = int(np.argmax(phase_ms))
        traffic, limiter, traffic_note = profiled_kernel() if PHASES[dom] == "bond_label" else (None, None, None)
        bps = KERNEL_BYTES_PER_SITE[PHASES[dom]] or 0.0
        achieved = bps * N_SITES / (phase_ms[dom] * 1e-3) / 1e9
        ms_per_step = 1e3 * total_s / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"replicas{world}"),
            "roofline": {"bound": "hbm", "kernel": PHASES[dom], "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "traffic_note": traffic_note,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "limiter": limiter, "bytes_per_site": bps},
            "phase_ms": dict(zip(PHASES, [float(v) for v in phase_ms])),
            "update_only": {"value": update_only, "unit": UNIT},
            "labeling": labeling,
            "other_workloads": secondary,
            "b_ref": {"bytes_per_site": B_REF, "GBps": value * B_REF, "frac": value * B_REF / peak},
            "gpu_launches": KERNELS_PER_SWEEP * args.steps,
            "clocks": clk,
            "e2e": e2e,
            "moments": {"U": moments["U"], "e_per_spin": moments["e_per_spin"],
                        "mean_cluster_size": moments["mean_cluster_size"]},
        }
        line.update(legs)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_sweeps)
            line["other_workloads"]["xy3d_L256"]["cpu_baseline"] = cpu_baseline_xy()
            leg_baselines(args, line)
        print(json.dumps(line), flush=True)
    sw.sw_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _job_list(specs):
    from paper_1403_7560_gb300.serve import Job
    return [Job(**d) for d in specs]


def batch_launches(specs, schedule):
    """Kernels one batch sweep launches: the tiled members' labels (one
    launch per model under label layout 0, one in all under layout 1 -- bit 0
    of the schedule), merge (one launch, or one per axis under bit 2),
    compression and apply; one launch per model of the small members (2D up
    to 8192 sites, 3D up to 4096); the step counter."""
    def is_small(m, d, L):
        return L ** d <= (8192 if d == 2 else 4096)
    tiled = {m for (m, d, L, _, _, _) in specs if not is_small(m, d, L)}
    small = {m for (m, d, L, _, _, _) in specs if is_small(m, d, L)}
    labels = (len(tiled) if (schedule & 1) == 0 else 1) if tiled else 0
    dim = specs[0][1] if specs else 2
    merges = (dim if schedule & 4 else 1) if tiled else 0
    return labels + (merges + 2 if tiled else 0) + len(small) + 1


def small_batch(sw, inputs, st, sweeps=50):
    """256 small 2D lattices (seed 1005, L 16..90): one batch, every member
    whole in one CTA's shared memory, against the same lattices one after
    another (each a one-CTA launch of all its sweeps)."""
    import torch
    specs = inputs.small_batch(256, 1005)
    sites = sum(L ** d for (_, d, L, _, _, _) in specs)
    hs = [sw.sw_create(m, d, L, q, T, seed) for (m, d, L, q, T, seed) in specs]
    b = sw.sw_batch_create(2)
    sw.sw_batch_set_stream(b, st.cuda_stream)
    for h in hs:
        sw.sw_set_stream(h, st.cuda_stream)
        sw.sw_batch_add(b, h)
    sw.sw_batch_sweep(b, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sw.sw_batch_sweep(b, sweeps)
    e1.record(st)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    sw.sw_batch_destroy(b)
    e0.record(st)
    for h in hs:
        sw.sw_sweep(h, sweeps)
    e1.record(st)
    torch.cuda.synchronize()
    t_serial = e0.elapsed_time(e1) / 1e3
    for h in hs:
        sw.sw_destroy(h)
    return {"workload": "256 2D lattices, model uniform over Ising / Potts q=3 / Potts q=4, L uniform in "
                        "[16,90], T in [0.8,1.2] Tc, seed 1005, 50 measured sweeps",
            "sites": sites, "value": sites * sweeps / (t_batch * 1e9), "unit": UNIT,
            "ms_per_step": 1e3 * t_batch / sweeps,
            "serial": {"value": sites * sweeps / (t_serial * 1e9), "unit": UNIT},
            "speedup_vs_serial": t_serial / t_batch,
            "gpu_launches": batch_launches(specs, 0) * sweeps}


def batch_leg(args, st):
    """Ragged batch of 256 2D Ising/Potts lattices (seed 1003), advanced
    together (one launch per phase, graph-replayed sweeps, autotuned tile
    shape, label layout and grid form) vs the same lattices swept one at a
    time.
    Inputs total ~1 GB (larger than L2)."""
    import torch
    import inputs
    from paper_1403_7560_gb300 import sw
    specs = inputs.ragged_batch(256, 1003)
    sites = sum(L ** d for (_, d, L, _, _, _) in specs)
    hs = [sw.sw_create(m, d, L, q, T, seed) for (m, d, L, q, T, seed) in specs]
    b = sw.sw_batch_create(2)
    sw.sw_batch_set_stream(b, st.cuda_stream)
    for h in hs:
        sw.sw_set_stream(h, st.cuda_stream)
        sw.sw_batch_add(b, h)
    sw.sw_batch_sweep(b, max(args.warmup, 3))
    # untimed: every tile shape, label layout and grid form on real sweeps of the batch
    tune_ms = sw.sw_batch_autotune(b, 5)
    cfg = sw.sw_batch_get_config(b)
    sw.sw_batch_sweep(b, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    clocks.mark_start()
    e0.record(st)
    sw.sw_batch_sweep(b, args.batch_sweeps)
    e1.record(st)
    torch.cuda.synchronize()
    clocks.mark_stop()
    clk = clocks.stop()
    t_batch = e0.elapsed_time(e1) / 1e3
    sw.sw_batch_destroy(b)
    # the plain path: each lattice alone, one after another
    k_serial = min(args.batch_sweeps, 50)
    e0.record(st)
    for h in hs:
        sw.sw_sweep(h, k_serial)
    e1.record(st)
    torch.cuda.synchronize()
    t_serial = e0.elapsed_time(e1) / 1e3
    for h in hs:
        sw.sw_measure(h)
        sw.sw_destroy(h)
    v_batch = sites * args.batch_sweeps / (t_batch * 1e9)
    v_serial = sites * k_serial / (t_serial * 1e9)
    small = small_batch(sw, inputs, st)
    return {"metric": "ragged batch site-updates/ns (256 2D Ising/Potts lattices, L 32..1024)",
            "value": v_batch, "unit": UNIT, "steps": args.batch_sweeps,
            "ms_per_step": 1e3 * t_batch / args.batch_sweeps,
            "config": {"workload": "ragged batch: 256 2D lattices, model uniform over Ising / Potts q=3 "
                                   "/ Potts q=4, L uniform over {32,48,...,1024}, T in [0.8,1.2] Tc, "
                                   f"seed 1003, {args.batch_sweeps} measured sweeps in one "
                                   "sw_batch_sweep call, CUDA-graph replay, autotuned tile shape and "
                                   "schedule (label layout, grid form)", "sites": sites,
                       "l2": "inputs larger than L2"},
            "serial": {"value": v_serial, "unit": UNIT, "steps": k_serial,
                       "note": "each lattice alone with sw_sweep, one after another"},
            "speedup_vs_serial": v_batch / v_serial,
            "autotune": {"chosen": cfg, "ms_per_sweep": {f"shape{sh}_schedule{sc}": round(float(tune_ms[sh, sc]), 4)
                                                         for sh in range(tune_ms.shape[0])
                                                         for sc in range(tune_ms.shape[1]) if tune_ms[sh, sc] > 0},
                         "note": "5 timed sweeps per configuration, before the timed region"},
            "small_lattices": small,
            "gpu_launches": batch_launches(specs, cfg["schedule"]) * args.batch_sweeps, "clocks": clk}


def run_batch(args):
    import torch
    from paper_1403_7560_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    leg = batch_leg(args, torch.cuda.Stream())
    line = dict(leg, n_gpus=1, warmup=max(args.warmup, 3), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="int8", data="synthetic")
    if not args.no_cpu_baseline:
        legs = {"batch": line}
        leg_baselines(args, legs)
    print(json.dumps(line), flush=True)


def serve_leg(args, max_l2=None, max_l3=None, max_sweeps=None):
    """Served request stream (seed 1004): continuous batching vs the
    one-at-a-time plain path, at saturation (all queued at t = 0) and at
    0.7 of the serial capacity (Poisson arrivals)."""
    import inputs
    from paper_1403_7560_gb300 import serve
    max_l2 = max_l2 or args.max_l2
    max_l3 = max_l3 or args.max_l3
    max_sweeps = max_sweeps or args.max_sweeps
    kw = dict(max_L2=max_l2, max_L3=max_l3, sweeps=(100, max_sweeps))
    budget = int(args.budget_gb * (1 << 30))

    def served(jobs, realtime):
        srv = serve.Server(budget, chunk=args.chunk)
        t0 = time.perf_counter()
        done = srv.run(jobs, realtime=realtime)
        wall = time.perf_counter() - t0
        srv.close()
        out = serve.summary(done, wall)
        out["rejected"] = len(srv.rejected)
        return out

    def serial(jobs, realtime):
        t0 = time.perf_counter()
        done = serve.run_serial(jobs, realtime=realtime)
        return serve.summary(done, time.perf_counter() - t0)

    # warm-up: the kernels' first launches
    served(_job_list(inputs.served_stream(6, 7, max_L2=256, max_L3=32, sweeps=(100, 200))), False)
    sat_srv = served(_job_list(inputs.served_stream(args.jobs, 1004, **kw)), False)
    sat_ser = serial(_job_list(inputs.served_stream(args.jobs, 1004, **kw)), False)
    rate = 0.7 * sat_ser["jobs_per_s"]
    lat_srv = served(_job_list(inputs.served_stream(args.jobs, 1004, rate=rate, **kw)), True)
    lat_ser = serial(_job_list(inputs.served_stream(args.jobs, 1004, rate=rate, **kw)), True)
    return {"metric": "served mix jobs/s, p50/p99", "value": sat_srv["jobs_per_s"], "unit": "jobs/s",
            "steps": args.jobs,
            "config": {"workload": f"served stream, seed 1004, {args.jobs} jobs, class uniform over "
                                   "2D Ising / 3D Ising / 2D Potts q=3,4,8 / 3D XY, L log-uniform in "
                                   f"[16,{max_l2}] (2D) or [16,{max_l3}] (3D), T = Tc(1+U(-0.02,0.02)), "
                                   f"sweeps log-uniform in [100,{max_sweeps}]",
                       "budget_gb": args.budget_gb, "chunk": args.chunk},
            "saturation": {"served": sat_srv, "serial": sat_ser,
                           "speedup": sat_srv["jobs_per_s"] / sat_ser["jobs_per_s"]},
            "latency_at_0.7_serial_capacity": {"rate_jobs_per_s": rate, "served": lat_srv,
                                               "serial": lat_ser}}


def run_serve(args):
    import torch
    from paper_1403_7560_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    line = dict(serve_leg(args), n_gpus=1, warmup=1, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="int8/uint8/f32", data="synthetic")
    if not args.no_cpu_baseline:
        legs = {"serve": line}
        leg_baselines(args, legs)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sweeps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="ising3d_L256", choices=["ising3d_L256", "batch", "serve"],
                    help="the headline 3D Ising L=256 sweep (default), the ragged batch, or the "
                         "served stream (one GPU)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the ragged-batch and served-stream legs of the default run")
    ap.add_argument("--batch-sweeps", type=int, default=500, help="batch: measured sweeps")
    ap.add_argument("--jobs", type=int, default=48, help="serve: jobs in the stream")
    ap.add_argument("--max-l2", type=int, default=4096, help="serve: largest 2D L")
    ap.add_argument("--max-l3", type=int, default=256, help="serve: largest 3D L")
    ap.add_argument("--max-sweeps", type=int, default=5000, help="serve: most sweeps of a job")
    ap.add_argument("--budget-gb", type=float, default=32.0, help="serve: HBM budget")
    ap.add_argument("--chunk", type=int, default=64, help="serve: sweeps per engine iteration")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
