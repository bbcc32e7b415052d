"""Ragged batches through the C ABI (needs a GB300).

A lattice advanced inside a batch (one launch per phase over every member's
tiles, the sweep replayed from a CUDA graph) must be bit-identical to the
same lattice advanced alone: spins, labels, per-sweep records and FP64
accumulators, also across members leaving and joining.  One member is also
checked against the CPU oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ISING, POTTS, XY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_7560_gb300 import build, sw as swmod
    build.build()
    return swmod


def same_state(sw, a, b, first, count):
    assert np.array_equal(sw.sw_get_spins(a), sw.sw_get_spins(b))
    assert np.array_equal(sw.sw_get_labels(a), sw.sw_get_labels(b))
    ra, rb = sw.sw_get_series(a, first, count), sw.sw_get_series(b, first, count)
    for x, y in zip(ra, rb):
        assert x == y
    ma, mb = sw.sw_measure(a), sw.sw_measure(b)
    for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
        assert ma[f] == mb[f], f


def make(sw, spec, seed):
    model, dim, L, q, T = spec
    return sw.sw_create(model, dim, L, q, T, seed)


SPECS_2D = [(ISING, 2, 32, 2, 2.269185), (POTTS, 2, 48, 3, 0.994973), (POTTS, 2, 100, 4, 0.91),
            (ISING, 2, 64, 2, 2.0), (ISING, 2, 17, 2, 2.5), (POTTS, 2, 33, 8, 0.75),
            (ISING, 2, 300, 2, 2.269185)]
SPECS_3D = [(ISING, 3, 16, 2, 4.5115), (POTTS, 3, 20, 3, 1.8), (ISING, 3, 40, 2, 4.4),
            (ISING, 3, 7, 2, 4.0)]


@pytest.mark.parametrize("specs", [SPECS_2D, SPECS_3D], ids=["2d", "3d"])
def test_batch_equals_alone(sw, specs):
    dim = specs[0][1]
    b = sw.sw_batch_create(dim)
    inb = [make(sw, s, 500 + k) for k, s in enumerate(specs)]
    alone = [make(sw, s, 500 + k) for k, s in enumerate(specs)]
    extra_spec = (POTTS, dim, 24, 5, 0.8 if dim == 2 else 1.5)
    extra_in, extra_alone = make(sw, extra_spec, 999), make(sw, extra_spec, 999)
    try:
        for h in inb:
            sw.sw_batch_add(b, h)
        assert sw.sw_batch_size(b) == len(specs)
        sw.sw_batch_sweep(b, 6)
        for h in alone:
            sw.sw_sweep(h, 6)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, 1, 6)
        # one member leaves (continues alone), a new one joins mid-run
        sw.sw_batch_remove(b, inb[1])
        sw.sw_batch_add(b, extra_in)
        sw.sw_batch_sweep(b, 4)
        sw.sw_sweep(inb[1], 4)
        for h in alone:
            sw.sw_sweep(h, 4)
        sw.sw_sweep(extra_alone, 4)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, 7, 4)
        same_state(sw, extra_in, extra_alone, 1, 4)
        # a batch sweep after discarded single sweeps keeps counters consistent
        sw.sw_discard(inb[0], 2)
        sw.sw_discard(alone[0], 2)
        sw.sw_batch_sweep(b, 2)
        sw.sw_sweep(alone[0], 2)
        same_state(sw, inb[0], alone[0], 13, 2)
    finally:
        sw.sw_batch_destroy(b)
        for h in inb + alone + [extra_in, extra_alone]:
            sw.sw_destroy(h)


def test_batch_member_matches_oracle(sw):
    spec = (POTTS, 2, 48, 3, 0.994973)
    b = sw.sw_batch_create(2)
    h = make(sw, spec, 77)
    other = make(sw, (ISING, 2, 64, 2, 2.2), 78)
    o = oracle.Oracle(POTTS, 2, 48, 3, 0.994973, 77)
    try:
        sw.sw_batch_add(b, other)
        sw.sw_batch_add(b, h)
        sw.sw_batch_sweep(b, 10)
        o.sweep(10)
        assert np.array_equal(sw.sw_get_spins(h), o.spins)
        assert np.array_equal(sw.sw_get_labels(h), o.labels)
        a, r = sw.sw_measure(h), o.take_acc()
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert a[f] == r[f], f
    finally:
        sw.sw_batch_destroy(b)
        sw.sw_destroy(h)
        sw.sw_destroy(other)


def test_batch_rules(sw):
    b = sw.sw_batch_create(2)
    xy = sw.sw_create(XY, 2, 16, 2, 1.0, 1)
    d3 = sw.sw_create(ISING, 3, 8, 2, 4.5, 1)
    ok = sw.sw_create(ISING, 2, 16, 2, 2.0, 1)
    b2 = sw.sw_batch_create(2)
    try:
        with pytest.raises(sw.SwError):
            sw.sw_batch_add(b, xy)
        with pytest.raises(sw.SwError):
            sw.sw_batch_add(b, d3)
        sw.sw_batch_add(b, ok)
        with pytest.raises(sw.SwError):
            sw.sw_batch_add(b2, ok)          # already in a batch
        sw.sw_batch_sweep(b, 0)
        sw.sw_destroy(ok)                    # leaves the batch first
        ok = None
        assert sw.sw_batch_size(b) == 0
        sw.sw_batch_sweep(b, 3)              # empty batch: nothing to do
        assert sw.sw_device_bytes(ISING, 3, 256, 2) > 256 ** 3 * 5
    finally:
        sw.sw_batch_destroy(b)
        sw.sw_batch_destroy(b2)
        for h in (xy, d3, ok):
            if h is not None:
                sw.sw_destroy(h)


@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("schedule", list(range(8)))
@pytest.mark.parametrize("specs", [SPECS_2D, SPECS_3D], ids=["2d", "3d"])
def test_every_launch_configuration_equals_alone(sw, specs, shape, schedule):
    """Tile shapes, label layouts, grid forms (one CTA per tile or a
    persistent grid striding over the tile map) and merge schedules (one
    launch, or one per axis) change no result: every member is
    bit-identical to the same lattice advanced alone."""
    dim = specs[0][1]
    b = sw.sw_batch_create(dim)
    inb = [make(sw, s, 700 + k) for k, s in enumerate(specs)]
    alone = [make(sw, s, 700 + k) for k, s in enumerate(specs)]
    try:
        for h in inb:
            sw.sw_batch_add(b, h)
        sw.sw_batch_set_config(b, shape, schedule)
        cfg = sw.sw_batch_get_config(b)
        assert (cfg["shape"], cfg["schedule"]) == (shape, schedule)
        assert cfg["tile_y"] == ([256, 128, 64] if dim == 2 else [16, 16, 8])[shape]
        assert cfg["tile_z"] == (1 if dim == 2 else [16, 8, 8][shape])
        sw.sw_batch_sweep(b, 5)
        for h in alone:
            sw.sw_sweep(h, 5)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, 1, 5)
    finally:
        sw.sw_batch_destroy(b)
        for h in inb + alone:
            sw.sw_destroy(h)


def test_autotune_keeps_the_fastest_and_changes_no_result(sw):
    specs = SPECS_2D
    b = sw.sw_batch_create(2)
    inb = [make(sw, s, 800 + k) for k, s in enumerate(specs)]
    alone = [make(sw, s, 800 + k) for k, s in enumerate(specs)]
    try:
        for h in inb:
            sw.sw_batch_add(b, h)
        sw.sw_batch_sweep(b, 2)
        ms = sw.sw_batch_autotune(b, 2)
        # Ising and Potts members: every shape with both label layouts, both
        # grid forms and both merge schedules
        assert ms.shape == (sw.SW_BATCH_TILE_SHAPES, sw.SW_BATCH_SCHEDULES)
        assert np.all(ms > 0)
        cfg = sw.sw_batch_get_config(b)
        assert ms[cfg["shape"], cfg["schedule"]] == ms.min()
        tuned = 2 + ms.size * (2 + 1)       # each configuration: one untimed + two timed sweeps
        for h in inb:
            assert sw.sw_sweep_counter(h) == tuned
        sw.sw_batch_sweep(b, 3)
        # a configuration switch between calls, then more sweeps
        sw.sw_batch_set_config(b, (cfg["shape"] + 1) % 3, 7 - cfg["schedule"])
        sw.sw_batch_sweep(b, 2)
        for h in alone:
            sw.sw_sweep(h, tuned + 5)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, tuned + 1, 4)
    finally:
        sw.sw_batch_destroy(b)
        for h in inb + alone:
            sw.sw_destroy(h)


def test_autotune_of_one_model_tries_one_schedule(sw):
    b = sw.sw_batch_create(3)
    hs = [make(sw, (ISING, 3, L, 2, 4.5115), 900 + L) for L in (16, 24)]
    try:
        for h in hs:
            sw.sw_batch_add(b, h)
        ms = sw.sw_batch_autotune(b, 1)
        # one model: the label layouts coincide; both grid forms and both
        # merge schedules are timed
        assert np.all(ms[:, [0, 2, 4, 6]] > 0) and np.all(ms[:, [1, 3, 5, 7]] == -1)
        assert sw.sw_batch_get_config(b)["schedule"] in (0, 2, 4, 6)
        for h in hs:
            assert sw.sw_sweep_counter(h) == 3 * 4 * 2
        with pytest.raises(sw.SwError):
            sw.sw_batch_set_config(b, 3, 0)
        with pytest.raises(sw.SwError):
            sw.sw_batch_set_config(b, 0, 8)
        with pytest.raises(sw.SwError):
            sw.sw_batch_autotune(b, 0)
    finally:
        sw.sw_batch_destroy(b)
        for h in hs:
            sw.sw_destroy(h)


def test_small_members_run_whole_in_shared_memory(sw):
    """Members of at most 8192 sites (2D) take the one-CTA
    branch of the batch graph; a batch of many of them, Ising and Potts,
    with a large member beside them, stays bit-identical to every lattice
    advanced alone, across a member leaving."""
    rng = np.random.default_rng(11)
    specs = []
    for k in range(40):
        L = int(rng.integers(8, 91))
        if k % 3 == 0:
            specs.append((ISING, 2, L, 2, 2.269185 * float(rng.uniform(0.9, 1.1))))
        else:
            q = int(rng.choice([3, 4, 8]))
            specs.append((POTTS, 2, L, q, 1.0 / np.log(1 + np.sqrt(q)) * float(rng.uniform(0.9, 1.1))))
    specs.append((ISING, 2, 200, 2, 2.269185))
    b = sw.sw_batch_create(2)
    inb = [make(sw, s, 1200 + k) for k, s in enumerate(specs)]
    alone = [make(sw, s, 1200 + k) for k, s in enumerate(specs)]
    try:
        for h in inb:
            sw.sw_batch_add(b, h)
        sw.sw_batch_sweep(b, 7)
        for h in alone:
            sw.sw_sweep(h, 7)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, 1, 7)
        sw.sw_batch_remove(b, inb[0])
        sw.sw_batch_sweep(b, 3)
        sw.sw_sweep(inb[0], 3)
        for h in alone:
            sw.sw_sweep(h, 3)
        for x, y in zip(inb, alone):
            same_state(sw, x, y, 8, 3)
    finally:
        sw.sw_batch_destroy(b)
        for h in inb + alone:
            sw.sw_destroy(h)


def test_sweep_targets_and_first_step_measurement(sw):
    """Members stop at their own sweep targets within one batch call; a
    member arriving with a pending record (sweeps run alone) has it measured
    by the batch's first step.  Every lattice stays bit-identical to the same
    lattice advanced alone by the same number of sweeps."""
    specs = SPECS_2D + [(ISING, 2, 160, 2, 2.3), (POTTS, 2, 130, 3, 1.0)]
    targets = [5, 12, 0, 9, 3, 17, 11, 14, 8]
    b = sw.sw_batch_create(2)
    inb = [make(sw, s, 1500 + k) for k, s in enumerate(specs)]
    alone = [make(sw, s, 1500 + k) for k, s in enumerate(specs)]
    try:
        sw.sw_sweep(inb[6], 2)             # tiled (L = 300): its sweep-2 record is pending
        sw.sw_sweep(inb[7], 1)
        for h, t in zip(inb, targets):
            sw.sw_set_sweep_target(h, t)
            sw.sw_batch_add(b, h)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_sweep(b, 10)
        for k, (h, t) in enumerate(zip(inb, targets)):
            expect = t if t else 18
            assert sw.sw_sweep_counter(h) == expect, k
            sw.sw_sweep(alone[k], expect)
        for x, y, t in zip(inb, alone, targets):
            n = sw.sw_sweep_counter(y)
            same_state(sw, x, y, 1, n)
        # a reached target stops the member; clearing it resumes
        sw.sw_batch_sweep(b, 3)
        assert sw.sw_sweep_counter(inb[0]) == 5
        sw.sw_set_sweep_target(inb[0], 0)
        sw.sw_batch_sweep(b, 2)
        assert sw.sw_sweep_counter(inb[0]) == 7
        with pytest.raises(sw.SwError):
            sw.sw_batch_autotune(b, 1)     # targets inside the tuning sweeps
    finally:
        sw.sw_batch_destroy(b)
        for h in inb + alone:
            sw.sw_destroy(h)
