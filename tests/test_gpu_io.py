"""Asynchronous host I/O: uploads and downloads on the handle's copy streams
give the same trajectories, states and records as the synchronous calls
(needs a GB300)."""
from __future__ import annotations

import numpy as np
import pytest

import inputs
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


def pinned(n, dtype):
    import torch
    tdt = {np.int8: torch.int8, np.uint8: torch.uint8, np.float32: torch.float32,
           np.uint16: torch.int16}[dtype]
    return torch.empty(n, dtype=tdt, pin_memory=True).numpy().view(dtype)


def test_round_trip(sw):
    h = sw.sw_create(POTTS, 3, 24, 5, 1.5, 11)
    N = 24 ** 3
    try:
        src = pinned(N, np.uint8)
        src[:] = inputs.random_spins(POTTS, N, 5, seed=3)
        dst = pinned(N, np.uint8)
        sw.sw_set_spins_async(h, src)
        sw.sw_get_spins_async(h, dst)
        sw.sw_wait_io(h)
        assert np.array_equal(dst, src)
        assert np.array_equal(sw.sw_get_spins(h), src)
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("model,dim,L,q,T", [
    (ISING, 3, 40, 2, 1 / 0.2216546),
    (POTTS, 2, 70, 3, inputs.tc_2d_potts(3)),
    (XY, 3, 24, 2, 2.2),
])
def test_pipelined_steps_match_synchronous(sw, model, dim, L, q, T):
    """Every step uploads a fresh state, sweeps, downloads the state and the
    record; all enqueued at once on one handle, step by step on another."""
    steps, N = 6, L ** dim
    dt = inputs.spin_dtype(model)
    ins = [inputs.random_spins(model, N, q, seed=100 + k) for k in range(steps)]
    a = sw.sw_create(model, dim, L, q, T, 77)
    b = sw.sw_create(model, dim, L, q, T, 77)
    try:
        ref_out, ref_rec = [], []
        for k in range(steps):
            sw.sw_set_spins(a, ins[k])
            sw.sw_sweep(a, 1)
            ref_out.append(sw.sw_get_spins(a))
            ref_rec.append(sw.sw_get_series(a, k + 1, 1)[0])
        pin_in = [pinned(N, dt) for _ in range(steps)]
        pin_out = [pinned(N, dt) for _ in range(steps)]
        recs = sw.record_buffer(steps)
        for k in range(steps):
            pin_in[k][:] = ins[k]
        for k in range(steps):
            sw.sw_set_spins_async(b, pin_in[k])
            sw.sw_sweep(b, 1)
            sw.sw_get_spins_async(b, pin_out[k])
            sw.sw_get_record_async(b, k + 1, recs[k])
        sw.sw_wait_io(b)
        for k in range(steps):
            assert np.array_equal(pin_out[k], ref_out[k]), k
            assert sw.record_dict(recs[k]) == ref_rec[k], k
        assert sw.sw_measure(a) == sw.sw_measure(b)
    finally:
        sw.sw_destroy(a)
        sw.sw_destroy(b)


def test_downloads_overlap_later_sweeps(sw):
    """A download enqueued before further sweeps holds the state at its
    enqueue point."""
    L, N = 32, 32 ** 3
    h = sw.sw_create(ISING, 3, L, 2, 4.0, 5)
    try:
        sw.sw_sweep(h, 2)
        want = sw.sw_get_spins(h)
        out = pinned(N, np.int8)
        sw.sw_get_spins_async(h, out)
        sw.sw_sweep(h, 5)
        sw.sw_wait_io(h)
        assert np.array_equal(out, want)
        assert not np.array_equal(sw.sw_get_spins(h), want)
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L", [(3, 32), (2, 32)], ids=["tiled", "one_cta"])
def test_download_snapshots_with_uploads_in_between(sw, dim, L):
    """Downloads interleaved with uploads that swap the two state buffers:
    each download holds the state at its enqueue point, and an upload into a
    buffer still being downloaded waits for that download."""
    N = L ** dim
    rng = np.random.default_rng(77)
    states = [pinned(N, np.int8) for _ in range(3)]
    for st in states:
        st[:] = rng.choice(np.array([-1, 1], dtype=np.int8), N)
    outs = [pinned(N, np.int8) for _ in range(3)]
    h = sw.sw_create(ISING, dim, L, 2, 2.3 if dim == 2 else 4.4, 9)
    ref = sw.sw_create(ISING, dim, L, 2, 2.3 if dim == 2 else 4.4, 9)
    try:
        sw.sw_sweep(h, 1)
        want0 = sw.sw_get_spins(h)
        sw.sw_get_spins_async(h, outs[0])     # buffer A
        sw.sw_set_spins_async(h, states[0])   # into B, swapped in
        sw.sw_get_spins_async(h, outs[1])     # buffer B
        sw.sw_set_spins_async(h, states[1])   # into A, after download 0
        sw.sw_sweep(h, 1)                     # writes A
        sw.sw_get_spins_async(h, outs[2])     # buffer A after the sweep
        sw.sw_set_spins_async(h, states[2])   # into B, after download 1
        sw.sw_wait_io(h)
        sw.sw_sweep(ref, 1)
        sw.sw_set_spins(ref, states[1])
        sw.sw_sweep(ref, 1)
        assert np.array_equal(outs[0], want0)
        assert np.array_equal(outs[1], states[0])
        assert np.array_equal(outs[2], sw.sw_get_spins(ref))
        assert np.array_equal(sw.sw_get_spins(h), states[2])
    finally:
        sw.sw_destroy(h)
        sw.sw_destroy(ref)


def test_errors(sw):
    h = sw.sw_create(ISING, 2, 32, 2, 2.0, 1)
    b = sw.sw_batch_create(2)
    try:
        buf = pinned(32 * 32, np.int8)
        with pytest.raises(sw.SwError) as e:
            sw.sw_set_spins_async(h, pinned(10, np.int8))
        assert e.value.code == sw.SW_ERR_BAD_ARG
        rec = sw.record_buffer(1)
        with pytest.raises(sw.SwError) as e:
            sw.sw_get_record_async(h, 1, rec[0])
        assert e.value.code == sw.SW_ERR_RANGE
        sw.sw_batch_add(b, h)
        with pytest.raises(sw.SwError) as e:
            sw.sw_get_spins_async(h, buf)
        assert e.value.code == sw.SW_ERR_BAD_ARG
        sw.sw_batch_remove(b, h)
        sw.sw_get_spins_async(h, buf)
        sw.sw_wait_io(h)
    finally:
        sw.sw_batch_destroy(b)
        sw.sw_destroy(h)
