"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Ising and Potts: initial state, bond planes, labels, spins, per-sweep records
and FP64 accumulators must be bit-identical to the oracle sweep by sweep.
XY: bonds may differ only where the float bond test is within rounding of
its threshold; labels are bit-identical given the GPU's mask; angles agree
within 1e-5 rad; per-sweep moments within the float summation bound.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import inputs
import oracle
from oracle import CLOCK, ISING, POTTS, XY

pytestmark = pytest.mark.gpu

ANGLE_TOL = 1e-5


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_7560_gb300 import build, sw as swmod
    build.build()
    return swmod


def record_key(model):
    if model == CLOCK:
        return ("mx", "my", "e_xy", "nclusters")
    return ("M", "E", "nclusters") if model == ISING else ("E", "S2", "nclusters")


def run_exact_parity(sw, model, dim, L, q, T, seed, sweeps, check_labels=True):
    h = sw.sw_create(model, dim, L, q, T, seed)
    o = oracle.Oracle(model, dim, L, q, T, seed)
    try:
        assert np.array_equal(sw.sw_get_spins(h), o.spins), "initial state"
        for k in range(1, sweeps + 1):
            sw.sw_sweep(h, 1)
            o.sweep(1)
            assert np.array_equal(sw.sw_get_bonds(h), o.planes), f"bonds, sweep {k}"
            if check_labels:
                assert np.array_equal(sw.sw_get_labels(h), o.labels), f"labels, sweep {k}"
            assert np.array_equal(sw.sw_get_spins(h), o.spins), f"spins, sweep {k}"
            rec = sw.sw_get_series(h, k, 1)[0]
            ref = o.last_record()
            for f in record_key(model) + ("M2", "Ed"):
                assert rec[f] == ref[f], (f, k, rec[f], ref[f])
        got, ref = sw.sw_measure(h), o.take_acc()
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert got[f] == ref[f], (f, got[f], ref[f])
    finally:
        sw.sw_destroy(h)
        o.close()


@pytest.mark.parametrize("model,dim,L,q", [
    (ISING, 2, 4, 2), (ISING, 2, 48, 2), (ISING, 3, 5, 2), (ISING, 3, 40, 2),
    (POTTS, 2, 33, 3), (POTTS, 3, 17, 4), (POTTS, 2, 16, 256), (XY, 2, 20, 2), (XY, 3, 9, 2),
    (CLOCK, 2, 20, 512), (CLOCK, 3, 9, 7)])
def test_initial_state(sw, model, dim, L, q):
    h = sw.sw_create(model, dim, L, q, 1.0, 77)
    try:
        assert np.array_equal(sw.sw_get_spins(h), oracle.init_spins(model, dim, L, q, 77))
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L,T", [
    (2, 4, 2.269185), (2, 16, 2.269185), (2, 31, 2.0), (2, 48, 2.269185), (2, 64, 2.269185),
    (2, 100, 2.4), (2, 130, 1.8), (3, 4, 4.5), (3, 8, 4.5115), (3, 9, 4.0), (3, 33, 4.5115),
    (3, 40, 5.0), (3, 64, 4.5115), (3, 11, 4.5115), (3, 19, 4.5115)])
def test_ising_sweeps_bit_exact(sw, dim, L, T):
    run_exact_parity(sw, ISING, dim, L, 2, T, seed=1000 + L, sweeps=12)


@pytest.mark.parametrize("dim,L,q,T", [
    (2, 64, 3, 0.994973), (2, 48, 4, 0.910239), (2, 37, 8, 0.74), (2, 32, 256, 0.3),
    (3, 16, 3, 1.8), (3, 24, 8, 1.3), (3, 15, 3, 1.8), (3, 19, 3, 1.8)])
def test_potts_sweeps_bit_exact(sw, dim, L, q, T):
    run_exact_parity(sw, POTTS, dim, L, q, T, seed=2000 + L, sweeps=12)


@pytest.mark.parametrize("model,L,q,T,sweeps", [
    (ISING, 60, 2, 4.5115, 10), (ISING, 64, 2, 3.9, 10), (ISING, 64, 2, 6.0, 6),
    (ISING, 128, 2, 4.5115, 4), (POTTS, 62, 3, 1.8, 8), (POTTS, 64, 5, 1.2, 6),
    (CLOCK, 64, 16, 2.0, 6)])
def test_larger_3d_lattices_bit_exact(sw, model, L, q, T, sweeps):
    """3D lattices of several tiles per axis, ragged (L = 60, 62) and not,
    below, at and above the Ising critical temperature."""
    run_exact_parity(sw, model, 3, L, q, T, seed=5000 + L, sweeps=sweeps)


@pytest.mark.parametrize("dim,L,q,T", [
    (2, 32, 512, 0.9), (2, 48, 8, 1.0), (2, 37, 3, 0.7), (3, 16, 512, 2.2), (3, 20, 6, 2.0),
    (3, 9, 1024, 2.1), (2, 40, 16, 0.15), (3, 24, 512, 0.3), (2, 40, 64, 50.0), (2, 300, 8, 0.9),
    (3, 15, 16, 2.0)])
def test_clock_sweeps_bit_exact(sw, dim, L, q, T):
    """The q-state clock model (the paper's discretised XY): trajectories and
    float moments are reproducible bit for bit, from far below to far above
    the transition (2/T from 0.04 to 13: the kernel's float estimate of the
    bond threshold and its margin scale with 2/T)."""
    run_exact_parity(sw, CLOCK, dim, L, q, T, seed=4000 + L, sweeps=10)


def test_clock_states_out_of_range_are_read_mod_q(sw):
    """States set outside [0, q) index no table out of range: the sweep runs
    as on the states mod q (bit-exact), unflipped sites keep their raw value."""
    dim, L, q, T, seed = 3, 24, 12, 2.0, 31
    rng = np.random.default_rng(5)
    raw = rng.integers(0, 65536, size=L ** dim).astype(np.uint16)
    h = sw.sw_create(CLOCK, dim, L, q, T, seed)
    o = oracle.Oracle(CLOCK, dim, L, q, T, seed)
    try:
        sw.sw_set_spins(h, raw)
        o.spins = (raw % q).astype(np.uint16)
        for k in range(1, 5):
            sw.sw_sweep(h, 1)
            o.sweep(1)
            assert np.array_equal(sw.sw_get_bonds(h), o.planes), k
            assert np.array_equal(sw.sw_get_spins(h) % q, o.spins), k
            rec, ref = sw.sw_get_series(h, k, 1)[0], o.last_record()
            assert (rec["mx"], rec["my"], rec["e_xy"]) == (ref["mx"], ref["my"], ref["e_xy"]), k
    finally:
        sw.sw_destroy(h)
        o.close()


def test_clock_config_3d_L64_q512(sw):
    """3D clock q=512 (Sec. 3's XY runs) near its critical temperature."""
    run_exact_parity(sw, CLOCK, 3, 64, 512, 2.20184, seed=1002, sweeps=3)


@pytest.mark.parametrize("model,dim,L,q,T", [
    (ISING, 3, 48, 2, 4.5115), (ISING, 2, 100, 2, 2.269185), (POTTS, 2, 64, 3, 0.994973),
    (POTTS, 3, 20, 8, 1.3), (POTTS, 2, 40, 40, 0.5), (ISING, 3, 7, 2, 4.0)])
def test_back_to_back_sweep_records(sw, model, dim, L, q, T):
    """Records of consecutive measured sweeps (each one measured by the next
    sweep's labeling kernel, the last by the stand-alone kernel), also
    across a measured -> discarded -> measured sequence."""
    h = sw.sw_create(model, dim, L, q, T, 77)
    o = oracle.Oracle(model, dim, L, q, T, 77)
    try:
        sw.sw_sweep(h, 9)
        sw.sw_discard(h, 2)
        sw.sw_sweep(h, 4)
        recs = []
        for n, meas in [(9, True), (2, False), (4, True)]:
            for _ in range(n):
                o.sweep(1, measure=meas)
                if meas:
                    recs.append(o.last_record())
        got = sw.sw_get_series(h, 1, 9) + sw.sw_get_series(h, 12, 4)
        for g, r in zip(got, recs):
            for f in record_key(model) + ("M2", "Ed"):
                assert g[f] == r[f], (f, g["sweep"], g[f], r[f])
        a, b = sw.sw_measure(h), o.take_acc()
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert a[f] == b[f], f
        assert np.array_equal(sw.sw_get_spins(h), o.spins)
    finally:
        sw.sw_destroy(h)
        o.close()


def test_low_and_high_temperature_limits(sw):
    # T -> 0: one cluster per equal-spin domain; T -> infinity: no bonds
    run_exact_parity(sw, ISING, 2, 40, 2, 1e-3, seed=5, sweeps=4)
    run_exact_parity(sw, ISING, 3, 12, 2, 1e-3, seed=6, sweeps=4)
    run_exact_parity(sw, POTTS, 2, 40, 5, 1e6, seed=7, sweeps=3)


def test_config_2d_ising_L64_full_run(sw):
    """2D Ising L=64 at T=2.269185, 200 discarded + 1000 measured sweeps:
    every measured record and the accumulators equal the oracle's."""
    model, dim, L, q, T, seed, ndisc, nmeas = inputs.WORKLOADS["ising2d_L64"]
    h = sw.sw_create(model, dim, L, q, T, seed)
    o = oracle.Oracle(model, dim, L, q, T, seed)
    try:
        sw.sw_discard(h, ndisc)
        o.sweep(ndisc, measure=False)
        sw.sw_measure(h)
        o.take_acc()
        recs = []
        for _ in range(nmeas):
            o.sweep(1)
            recs.append(o.last_record())
        sw.sw_sweep(h, nmeas)
        got = sw.sw_get_series(h, ndisc + 1, nmeas)
        for k, (g, r) in enumerate(zip(got, recs)):
            assert (g["M"], g["E"], g["nclusters"]) == (r["M"], r["E"], r["nclusters"]), k
        a, b = sw.sw_measure(h), o.take_acc()
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert a[f] == b[f], f
        assert np.array_equal(sw.sw_get_spins(h), o.spins)
        assert np.array_equal(sw.sw_get_labels(h), o.labels)
    finally:
        sw.sw_destroy(h)
        o.close()


def test_config_3d_ising_L256_first_sweeps(sw):
    """3D Ising L=256 at K=0.2216546 in the benchmark's launch configuration:
    the first sweeps are bit-identical to the oracle (spins, labels, bonds,
    records)."""
    model, dim, L, q, T, seed, _, _ = inputs.WORKLOADS["ising3d_L256"]
    run_exact_parity(sw, model, dim, L, q, T, seed, sweeps=2)


def test_config_3d_ising_L256_thermalised(sw):
    """The benchmark's lattice in the regime it is timed in: 100 discarded
    sweeps on the GPU from the seeded start (K = 0.2216546, clusters
    spanning the lattice), then the oracle takes over the GPU's state and
    sweep counter and both run 3 measured sweeps.  Bonds, labels, spins,
    records and accumulators are bit-identical."""
    model, dim, L, q, T, seed, ndisc, _ = inputs.WORKLOADS["ising3d_L256"]
    h = sw.sw_create(model, dim, L, q, T, seed)
    o = oracle.Oracle(model, dim, L, q, T, seed)
    try:
        sw.sw_discard(h, ndisc)
        sw.sw_measure(h)
        o.spins = sw.sw_get_spins(h)
        o.sweep_counter = int(sw.sw_sweep_counter(h))
        assert o.sweep_counter == ndisc
        for k in range(ndisc + 1, ndisc + 4):
            sw.sw_sweep(h, 1)
            o.sweep(1)
            assert np.array_equal(sw.sw_get_bonds(h), o.planes), f"bonds, sweep {k}"
            lab = sw.sw_get_labels(h)
            assert np.array_equal(lab, o.labels), f"labels, sweep {k}"
            assert np.array_equal(sw.sw_get_spins(h), o.spins), f"spins, sweep {k}"
            rec, ref = sw.sw_get_series(h, k, 1)[0], o.last_record()
            for f in ("M", "E", "nclusters", "M2", "Ed"):
                assert rec[f] == ref[f], (f, k, rec[f], ref[f])
            # the regime of the benchmark: one cluster holds a sizeable share
            assert np.bincount(lab).max() > 0.01 * lab.size, k
        got, ref = sw.sw_measure(h), o.take_acc()
        for f in ("n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters"):
            assert got[f] == ref[f], (f, got[f], ref[f])
    finally:
        sw.sw_destroy(h)
        o.close()


@pytest.mark.parametrize("model,dim,L,q,T", [
    (ISING, 2, 48, 2, 2.269185), (ISING, 3, 40, 2, 4.5115), (POTTS, 3, 20, 3, 1.8),
    (POTTS, 2, 70, 4, 0.910239), (CLOCK, 3, 12, 512, 2.2)])
def test_derived_moments_follow_their_definitions(sw, model, dim, L, q, T):
    """sw_measure's derived values are the definitions applied to the
    accumulators, which equal the oracle's bit for bit: U = <M^4>/<M^2>^2
    (Sec. 3), e = <E>/N, C/N = (<E^2> - <E>^2)/(N T^2), mean cluster size
    = N/<clusters>; each compared exactly (the same double operations)."""
    h = sw.sw_create(model, dim, L, q, T, 515)
    o = oracle.Oracle(model, dim, L, q, T, 515)
    try:
        sw.sw_discard(h, 20)
        o.sweep(20, measure=False)
        sw.sw_measure(h)
        o.take_acc()
        sw.sw_sweep(h, 60)
        o.sweep(60)
        got, acc = sw.sw_measure(h), o.take_acc()
        for f in acc:
            assert got[f] == acc[f], f
        n, N = acc["n_sweeps"], float(L ** dim)
        m2, m4 = acc["sum_M2"] / n, acc["sum_M4"] / n
        e1, e2 = acc["sum_E"] / n, acc["sum_E2"] / n
        assert got["U"] == m4 / (m2 * m2)
        assert got["e_per_spin"] == e1 / N
        assert got["c_per_spin"] == (e2 - e1 * e1) / (N * T * T)
        assert got["mean_cluster_size"] == N / (acc["sum_nclusters"] / n)
        assert 1.0 <= got["U"] and 1.0 <= got["mean_cluster_size"] <= N and got["c_per_spin"] >= 0.0
    finally:
        sw.sw_destroy(h)
        o.close()


def test_derived_moments_xy_and_limits(sw):
    """XY: the same definitions on the GPU's own accumulators; no bonds at
    T -> infinity give a mean cluster size of exactly 1."""
    h = sw.sw_create(XY, 3, 16, 2, 2.2, 9)
    try:
        sw.sw_sweep(h, 40)
        got = sw.sw_measure(h)
        n, N, T = got["n_sweeps"], 16.0 ** 3, 2.2
        m2, m4 = got["sum_M2"] / n, got["sum_M4"] / n
        e1, e2 = got["sum_E"] / n, got["sum_E2"] / n
        assert got["U"] == m4 / (m2 * m2)
        assert got["e_per_spin"] == e1 / N
        assert got["c_per_spin"] == (e2 - e1 * e1) / (N * T * T)
        assert got["mean_cluster_size"] == N / (got["sum_nclusters"] / n)
    finally:
        sw.sw_destroy(h)
    h = sw.sw_create(ISING, 2, 64, 2, 1e9, 9)
    try:
        sw.sw_sweep(h, 5)
        assert sw.sw_measure(h)["mean_cluster_size"] == 1.0
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L,T", [(3, 1024, 1 / 0.2216546), (2, 32768, 2.269185)])
def test_maximum_ising_lattice(sw, dim, L, T):
    """The largest Ising lattice sw_create accepts (N = 2^30 sites, the forest
    word's limit): one sweep, then properties that hold at any size, checked
    on every site or on a large sample (the oracle cannot run this size)."""
    N = L ** dim
    assert N == 1 << 30
    h = sw.sw_create(ISING, dim, L, 2, T, 7)
    try:
        s0 = sw.sw_get_spins(h)
        sw.sw_sweep(h, 1)
        planes = sw.sw_get_bonds(h)
        s1 = sw.sw_get_spins(h)
        lab = sw.sw_get_labels(h)
        rec = sw.sw_get_series(h, 1, 1)[0]
        assert rec["M"] == int(s1.sum(dtype=np.int64))
        roots = np.flatnonzero(lab == np.arange(N, dtype=np.int32))
        assert rec["nclusters"] == roots.size
        rng = np.random.default_rng(11)
        i = rng.integers(0, N, size=200_000)
        assert np.all(lab[i] <= i) and np.all(lab[lab[i]] == lab[i])   # canonical roots
        W, R = (L + 31) // 32, N // L
        x, row = i % L, i // L
        y, z = row % L, row // L
        for d in range(dim):
            bit = (planes[d * R * W + row * W + (x >> 5)] >> (x & 31).astype(np.uint32)) & 1
            j = [np.where(x + 1 == L, i - x, i + 1),
                 np.where(y + 1 == L, i - y * L, i + L),
                 np.where(z + 1 == L, i - z * L * L, i + L * L)][d]
            on = bit.astype(bool)
            assert on.any()
            assert np.all(s0[i[on]] == s0[j[on]])        # bonds join equal spins
            assert np.all(lab[i[on]] == lab[j[on]])      # bonded sites share a cluster
            assert np.all(s1[i[on]] == s1[j[on]])        # and the cluster's new spin
    finally:
        sw.sw_destroy(h)


def test_maximum_potts_q256_lattice(sw):
    """Potts q=256 needs 8 draw bits, so the forest word limits N to 2^23:
    3D L=203 (8,365,427 sites) is the largest cube, bit-exact for 2 sweeps."""
    with pytest.raises(sw.SwError):
        sw.sw_create(POTTS, 3, 204, 256, 0.5, 1)
    run_exact_parity(sw, POTTS, 3, 203, 256, 0.5, seed=6203, sweeps=2)


# ---------------------------------------------------------------- labels
@pytest.mark.parametrize("dim,L", [(2, 4), (2, 31), (2, 64), (2, 97), (2, 200), (3, 4), (3, 8),
                                   (3, 13), (3, 32), (3, 41)])
@pytest.mark.parametrize("density", [0.3, 0.5, 0.7, 0.95])
def test_labels_random_masks(sw, dim, L, density):
    h = sw.sw_create(ISING, dim, L, 2, 2.0, 1)
    try:
        m = inputs.random_mask(dim, L, density, seed=L * 7 + int(100 * density))
        assert np.array_equal(sw.sw_label_from_bonds(h, m), oracle.labels(dim, L, m))
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L", [(2, 4), (2, 48), (2, 96), (3, 5), (3, 24), (3, 33)])
def test_labels_structured_masks(sw, dim, L):
    h = sw.sw_create(ISING, dim, L, 2, 2.0, 1)
    N = L ** dim
    try:
        on = inputs.pack_planes(np.ones((dim, N), bool), dim, L)
        assert (sw.sw_label_from_bonds(h, on) == 0).all()
        off = inputs.pack_planes(np.zeros((dim, N), bool), dim, L)
        assert np.array_equal(sw.sw_label_from_bonds(h, off), np.arange(N))
        for axis in range(dim):
            m = inputs.stripe_mask(dim, L, axis)
            assert np.array_equal(sw.sw_label_from_bonds(h, m), oracle.labels(dim, L, m))
        if dim == 2:
            m = inputs.spiral_mask(L)
            assert (sw.sw_label_from_bonds(h, m) == 0).all()
    finally:
        sw.sw_destroy(h)


# ---------------------------------------------------------------- XY
def ang_diff(a, b):
    d = np.abs(a.astype(np.float64) - b.astype(np.float64)) % (2 * np.pi)
    return np.minimum(d, 2 * np.pi - d)


def xy_borderline(model_T, dim, L, seed, k, theta, gpu_mask, ora_mask):
    """Every bond where GPU and oracle disagree must have its uniform draw
    within float rounding of the bond probability."""
    diff = inputs.unpack_planes(gpu_mask ^ ora_mask, dim, L)
    if not diff.any():
        return 0
    phi = float(oracle.xy_phi(seed, k))
    th = theta.astype(np.float64)
    x = np.cos(th - phi)
    n = 0
    for d in range(dim):
        idx = np.nonzero(diff[d])[0]
        if idx.size == 0:
            continue
        from exact import neighbours
        j = neighbours(dim, L, d)[idx]
        prod = x[idx] * x[j]
        p = np.where(prod > 0, -np.expm1(-2.0 / model_T * prod), 0.0)
        w = np.array([oracle.philox([int(i), k, 1, 0], [seed & 0xffffffff, seed >> 32])[d] for i in idx])
        u = (w >> 8).astype(np.float64) * 2.0 ** -24
        near = (np.abs(u - p) < 1e-5) | (np.abs(prod) < 1e-5)
        assert np.all(near), (u[~near], p[~near], prod[~near])
        n += idx.size
    return n


@pytest.mark.parametrize("dim,L,T,sweeps", [(2, 64, 0.89, 8), (3, 32, 2.2, 6), (3, 48, 2.0, 4),
                                            (2, 37, 1.1, 6), (3, 64, 2.2, 3), (2, 512, 0.89, 3),
                                            (3, 11, 2.2, 6)])
def test_xy_sweeps(sw, dim, L, T, sweeps):
    seed = 3000 + L
    h = sw.sw_create(XY, dim, L, 2, T, seed)
    N = L ** dim
    try:
        theta = sw.sw_get_spins(h)
        assert np.array_equal(theta, oracle.init_spins(XY, dim, L, 2, seed))
        mismatches = 0
        for k in range(1, sweeps + 1):
            sw.sw_sweep(h, 1)
            gmask = sw.sw_get_bonds(h)
            glab = sw.sw_get_labels(h)
            gnew = sw.sw_get_spins(h)
            omask = oracle.bonds(XY, dim, L, 2, T, seed, k, theta)
            mismatches += xy_borderline(T, dim, L, seed, k, theta, gmask, omask)
            assert np.array_equal(glab, oracle.labels(dim, L, gmask)), k
            onew, ncl = oracle.flip(XY, dim, L, 2, seed, k, glab, theta)
            assert ang_diff(gnew, onew).max() < ANGLE_TOL, k
            rec = sw.sw_get_series(h, k, 1)[0]
            ref = oracle.moments(XY, dim, L, 2, gnew)
            tol = 2e-6 * N * (dim + 1) + 1e-3
            assert abs(rec["mx"] - ref["mx"]) < tol and abs(rec["my"] - ref["my"]) < tol
            assert abs(rec["e_xy"] - ref["e_xy"]) < tol
            assert rec["nclusters"] == ncl
            theta = gnew
        assert mismatches <= max(2, N * dim * sweeps // 100000)
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("ndisc", [0, 30])
def test_xy_config_3d_L256(sw, ndisc):
    """3D XY L=256 at K = 0.4541652, from the seeded start and after 30
    discarded sweeps: every bond that differs from the oracle's lies at the
    rounding edge of its probability (checked bit by bit), labels equal the
    oracle's on the GPU's mask, angles agree within 1e-5 rad, and the
    record's moments within the float summation bound."""
    model, dim, L, q, T, seed, _, _ = inputs.WORKLOADS["xy3d_L256"]
    N = L ** dim
    h = sw.sw_create(model, dim, L, q, T, seed)
    try:
        sw.sw_discard(h, ndisc)
        theta = sw.sw_get_spins(h)
        for k in range(ndisc + 1, ndisc + 3):
            sw.sw_sweep(h, 1)
            gmask = sw.sw_get_bonds(h)
            glab = sw.sw_get_labels(h)
            gnew = sw.sw_get_spins(h)
            omask = oracle.bonds(XY, dim, L, 2, T, seed, k, theta)
            xy_borderline(T, dim, L, seed, k, theta, gmask, omask)
            assert np.array_equal(glab, oracle.labels(dim, L, gmask)), k
            onew, ncl = oracle.flip(XY, dim, L, 2, seed, k, glab, theta)
            assert ang_diff(gnew, onew).max() < ANGLE_TOL, k
            rec = sw.sw_get_series(h, k, 1)[0]
            ref = oracle.moments(XY, dim, L, 2, gnew)
            tol = 2e-6 * N * (dim + 1) + 1e-3
            assert abs(rec["mx"] - ref["mx"]) < tol and abs(rec["my"] - ref["my"]) < tol, k
            assert abs(rec["e_xy"] - ref["e_xy"]) < tol and rec["nclusters"] == ncl, k
            theta = gnew
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L,T,bins,per", [(2, 16, 0.9, 20, 2000), (3, 8, 2.2, 20, 2000)])
def test_xy_ensemble_moments_within_3_sigma(sw, dim, L, T, bins, per):
    """Independent GPU and oracle XY runs (different seeds): binned means of
    E and M^2 agree within 3 combined standard errors.  Each bin averages
    2000 sweeps, far longer than the SW autocorrelation time at these sizes,
    so the bins are independent and their spread gives the error."""

    def binned(step_measure):
        rows = []
        for _ in range(bins):
            a = step_measure()
            rows.append([a["sum_E"] / a["n_sweeps"], a["sum_M2"] / a["n_sweeps"]])
        r = np.array(rows)
        return r.mean(0), r.std(0, ddof=1) / math.sqrt(bins)

    h = sw.sw_create(XY, dim, L, 2, T, 4242)
    o = oracle.Oracle(XY, dim, L, 2, T, 4243)
    try:
        sw.sw_discard(h, 500)
        o.sweep(500, measure=False)
        sw.sw_measure(h)
        o.take_acc()

        def g():
            sw.sw_sweep(h, per)
            return sw.sw_measure(h)

        def c():
            o.sweep(per)
            return o.take_acc()
        gm, ge = binned(g)
        cm, ce = binned(c)
        for j in range(2):
            assert abs(gm[j] - cm[j]) < 3 * math.hypot(ge[j], ce[j]), (j, gm, cm, ge, ce)
    finally:
        sw.sw_destroy(h)
        o.close()


# ---------------------------------------------------------------- API behaviour
def test_resume_is_exact(sw):
    a = sw.sw_create(POTTS, 3, 20, 3, 1.7, 91)
    b = sw.sw_create(POTTS, 3, 20, 3, 1.7, 91)
    try:
        sw.sw_sweep(a, 9)
        sw.sw_set_spins(b, sw.sw_get_spins(a))
        sw.sw_set_sweep_counter(b, sw.sw_sweep_counter(a))
        sw.sw_sweep(a, 6)
        sw.sw_sweep(b, 6)
        assert np.array_equal(sw.sw_get_spins(a), sw.sw_get_spins(b))
    finally:
        sw.sw_destroy(a)
        sw.sw_destroy(b)


def test_user_stream_and_device_buffers(sw):
    import torch
    h = sw.sw_create(ISING, 3, 32, 2, 4.5, 12)
    try:
        st = torch.cuda.Stream()
        sw.sw_set_stream(h, st.cuda_stream)
        buf = torch.empty(32 ** 3, dtype=torch.int8, device="cuda")
        sw.sw_sweep(h, 3)
        sw.sw_get_spins_device(h, buf.data_ptr(), buf.numel())
        st.synchronize()
        assert np.array_equal(buf.cpu().numpy(), sw.sw_get_spins(h))
        flipped = (-buf).contiguous()
        sw.sw_set_spins_device(h, flipped.data_ptr(), flipped.numel())
        st.synchronize()
        assert np.array_equal(sw.sw_get_spins(h), flipped.cpu().numpy())
    finally:
        sw.sw_destroy(h)


def test_series_range_errors(sw):
    h = sw.sw_create(ISING, 2, 16, 2, 2.0, 1)
    try:
        sw.sw_discard(h, 3)
        sw.sw_sweep(h, 2)
        with pytest.raises(sw.SwError):
            sw.sw_get_series(h, 1, 1)          # discarded sweep: no record
        assert [r["sweep"] for r in sw.sw_get_series(h, 4, 2)] == [4, 5]
        with pytest.raises(sw.SwError):
            sw.sw_get_series(h, 6, 1)          # not done yet
    finally:
        sw.sw_destroy(h)


# ---------------------------------------------------------------- failure detection
def test_capped_loops_report_timeout_and_the_handle_recovers(sw):
    """Failure detection without a GPU fault: with the handle's loop cap at
    0 every union loop (shared-memory tile labeling, global merge), every
    compression walk and every label-equivalence iteration gives up at once.
    The kernels set the device error flag and return; the next synchronising
    call reports SW_ERR_TIMEOUT.  With the production cap restored the same
    handle labels correctly and sweeps bit-identically to the oracle."""
    dim, L, T, seed = 2, 256, 2.269185, 3
    N = L ** dim
    h = sw.sw_create(ISING, dim, L, 2, T, seed)
    try:
        on = inputs.pack_planes(np.ones((dim, N), bool), dim, L)
        sw.sw_set_loop_cap(h, 0)
        with pytest.raises(sw.SwError) as e:
            sw.sw_label_from_bonds(h, on)
        assert e.value.code == sw.SW_ERR_TIMEOUT
        sw.sw_sweep(h, 2)
        with pytest.raises(sw.SwError) as e:
            sw.sw_sync(h)
        assert e.value.code == sw.SW_ERR_TIMEOUT
        with pytest.raises(sw.SwError) as e:
            sw.sw_relabel(h, sw.SW_LABEL_EQUIVALENCE)
        assert e.value.code == sw.SW_ERR_TIMEOUT
        sw.sw_sync(h)                                   # the flag was cleared
        sw.sw_set_loop_cap(h, -1)
        assert (sw.sw_label_from_bonds(h, on) == 0).all()
        # resume from a known state: the handle sweeps exactly as the oracle
        o = oracle.Oracle(ISING, dim, L, 2, T, seed)
        try:
            sw.sw_set_spins(h, o.spins)
            sw.sw_set_sweep_counter(h, 0)
            sw.sw_measure(h)
            for k in range(1, 4):
                sw.sw_sweep(h, 1)
                o.sweep(1)
                assert np.array_equal(sw.sw_get_labels(h), o.labels), k
                assert np.array_equal(sw.sw_get_spins(h), o.spins), k
        finally:
            o.close()
    finally:
        sw.sw_destroy(h)
