"""Pins of the CPU oracle against references other than itself (CPU only).

Each group is chosen so that a plausible slip in the oracle fails it:
  * Philox: published known-answer vectors (any wrong constant, word order
    or round count changes every output word).
  * Labels: scipy connected components on random, structured and
    exhaustive masks (a wrong neighbour index, wrap or link direction).
  * Bonds: structure (never across unequal spins / opposite projections)
    and rates against the bond probability of Sec. 2 (a wrong factor of 2 in
    the exponent, or K vs 2K for Potts).
  * Flip: clusters uniform, draws unbiased, XY reflection invariants.
  * Moments: numpy evaluation of M, E; Potts M^2 through simplex vectors.
  * Stationary law: exact enumeration of small Ising / Potts lattices,
    Kaufman's exact L x L Ising energy, an independent XY Metropolis chain,
    and the exact identity q=2 Potts at T/2 == Ising at T.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from oracle import ISING, POTTS, XY
import exact
import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            out = oracle.philox(v[0:4], v[4:6])
            assert list(out) == v[6:10]
            rows += 1
    assert rows == 3


def test_philox_uniformity():
    # 2^16 draws from consecutive site counters: every output word uniform.
    words = np.array([oracle.philox([i, 7, 1, 0], [12345, 0]) for i in range(1 << 14)])
    for w in range(4):
        hist = np.bincount(words[:, w] >> 28, minlength=16)
        chi2 = ((hist - hist.mean()) ** 2 / hist.mean()).sum()
        assert chi2 < 45.0  # 15 dof, p ~ 1e-4


# ----------------------------------------------------------------- labels
@pytest.mark.parametrize("dim,L", [(2, 4), (2, 5), (2, 33), (2, 64), (3, 4), (3, 7), (3, 16)])
@pytest.mark.parametrize("density", [0.2, 0.5, 0.8])
def test_labels_equal_components(dim, L, density):
    planes = inputs.random_mask(dim, L, density, seed=dim * 1000 + L * 10 + int(density * 10))
    assert np.array_equal(oracle.labels(dim, L, planes), exact.components(dim, L, planes))


@pytest.mark.parametrize("dim,L", [(2, 4), (2, 48), (3, 5)])
def test_labels_structured(dim, L):
    N = L ** dim
    allon = inputs.pack_planes(np.ones((dim, N), bool), dim, L)
    assert (oracle.labels(dim, L, allon) == 0).all()
    alloff = inputs.pack_planes(np.zeros((dim, N), bool), dim, L)
    assert np.array_equal(oracle.labels(dim, L, alloff), np.arange(N))
    for axis in range(dim):
        m = inputs.stripe_mask(dim, L, axis)
        assert np.array_equal(oracle.labels(dim, L, m), exact.components(dim, L, m))
    if dim == 2:
        m = inputs.spiral_mask(L)
        lab = oracle.labels(dim, L, m)
        assert (lab == 0).all()


def test_labels_exhaustive_strip():
    # all 2^10 masks of the bonds inside a 2x4 open strip of an L=4 lattice
    L, dim = 4, 2
    inner = [(0, x + 4 * y) for y in range(2) for x in range(3)] + [(1, x) for x in range(4)]
    for m in range(1 << len(inner)):
        bits = np.zeros((dim, L * L), bool)
        for b, (d, i) in enumerate(inner):
            bits[d, i] = (m >> b) & 1
        planes = inputs.pack_planes(bits, dim, L)
        assert np.array_equal(oracle.labels(dim, L, planes), exact.components(dim, L, planes))


# ----------------------------------------------------------------- bonds
@pytest.mark.parametrize("model,q,T", [(ISING, 2, 2.269185), (ISING, 2, 4.0),
                                       (POTTS, 3, 0.994973), (POTTS, 8, 0.7)])
def test_bond_rate_and_structure(model, q, T):
    dim, L = 2, 64
    s = inputs.random_spins(model, L * L, q, seed=11)
    nbr = [exact.neighbours(dim, L, d) for d in range(dim)]
    equal = np.stack([s == s[nbr[d]] for d in range(dim)])
    n_eq, n_on = 0, 0
    for k in range(1, 41):
        bits = inputs.unpack_planes(oracle.bonds(model, dim, L, q, T, 99, k, s), dim, L)
        assert not (bits & ~equal).any()          # never across unequal spins
        n_eq += equal.sum()
        n_on += bits.sum()
    p = 1.0 - math.exp(-(2.0 if model == ISING else 1.0) / T)
    sigma = math.sqrt(n_eq * p * (1 - p))
    assert abs(n_on - n_eq * p) < 5 * sigma


def test_bond_threshold_extremes():
    assert oracle.bond_threshold(ISING, 1e6) < 2 ** 32 * 3e-6
    assert oracle.bond_threshold(ISING, 1e-3) == 2 ** 32 - 1
    assert oracle.bond_threshold(POTTS, 1e-3) == 2 ** 32 - 1


def test_zero_temperature_clusters_are_domains():
    # T -> 0: p -> 1, every bond between equal spins is active, so the SW
    # clusters are the connected equal-spin domains.
    for model, q, dim, L in [(ISING, 2, 2, 16), (POTTS, 3, 2, 9), (ISING, 2, 3, 6)]:
        s = inputs.random_spins(model, L ** dim, q, seed=5)
        planes = oracle.bonds(model, dim, L, q, 1e-3, 3, 1, s)
        bits = np.stack([s == s[exact.neighbours(dim, L, d)] for d in range(dim)])
        assert np.array_equal(inputs.unpack_planes(planes, dim, L), bits)
        assert np.array_equal(oracle.labels(dim, L, planes), exact.components(dim, L, planes))


def test_infinite_temperature_no_clusters():
    o = oracle.Oracle(ISING, 2, 16, 2, 1e9, 4)
    o.sweep(3)
    assert o.last_record()["nclusters"] == 256


def test_xy_bond_rate_and_structure():
    dim, L, T, seed = 2, 64, 0.9, 21
    th = inputs.random_spins(XY, L * L, 2, seed=3)
    nbr = [exact.neighbours(dim, L, d) for d in range(dim)]
    n_on, p_sum, var = 0, 0.0, 0.0
    for k in range(1, 31):
        phi = float(oracle.xy_phi(seed, k))
        x = np.cos(th.astype(np.float64) - phi)
        bits = inputs.unpack_planes(oracle.bonds(XY, dim, L, 2, T, seed, k, th), dim, L)
        for d in range(dim):
            prod = x * x[nbr[d]]
            assert not (bits[d] & (prod <= 0)).any()
            p = np.where(prod > 0, 1 - np.exp(-2.0 / T * prod), 0.0)
            n_on += bits[d].sum()
            p_sum += p.sum()
            var += (p * (1 - p)).sum()
    assert abs(n_on - p_sum) < 5 * math.sqrt(var)


def test_xy_phi_uniform():
    phis = np.array([oracle.xy_phi(77, k) for k in range(1, 4001)], dtype=np.float64)
    assert phis.min() >= 0 and phis.max() < 2 * np.pi
    hist = np.bincount((phis / (2 * np.pi) * 8).astype(int), minlength=8)
    assert ((hist - 500) ** 2 / 500).sum() < 30


# ----------------------------------------------------------------- flip
@pytest.mark.parametrize("model,q", [(ISING, 2), (POTTS, 3), (POTTS, 8)])
def test_flip_clusters_uniform_and_unbiased(model, q):
    dim, L, T = 2, 64, 0.8 if model == POTTS else 2.5
    s = inputs.random_spins(model, L * L, q, seed=8)
    counts = np.zeros(q if model == POTTS else 2)
    ncl_total = 0
    for k in range(1, 21):
        planes = oracle.bonds(model, dim, L, q, T, 5, k, s)
        lab = oracle.labels(dim, L, planes)
        new, ncl = oracle.flip(model, dim, L, q, 5, k, lab, s)
        roots = np.nonzero(lab == np.arange(L * L))[0]
        assert ncl == roots.size
        assert (new == new[lab]).all()                # each cluster uniform
        v = new[roots].astype(np.int64)
        counts += np.bincount((v + 1) // 2 if model == ISING else v, minlength=counts.size)
        ncl_total += ncl
        s = new
    expect = ncl_total / counts.size
    assert (((counts - expect) ** 2) / expect).sum() < 3 * counts.size + 20


def test_xy_flip_invariants():
    dim, L, T, seed, k = 2, 32, 1.0, 9, 4
    th = inputs.random_spins(XY, L * L, 2, seed=1)
    planes = oracle.bonds(XY, dim, L, 2, T, seed, k, th)
    lab = oracle.labels(dim, L, planes)
    new, _ = oracle.flip(XY, dim, L, 2, seed, k, lab, th)
    phi = float(oracle.xy_phi(seed, k))
    t0, t1 = th.astype(np.float64), new.astype(np.float64)
    assert ((t1 >= 0) & (t1 <= 2 * np.pi + 1e-6)).all()
    moved = ~np.isclose(np.cos(t1 - t0), 1.0, atol=1e-9) | ~np.isclose(np.sin(t1 - t0), 0.0, atol=1e-6)
    # reflected sites: projection on r changes sign, the perpendicular part stays
    assert np.allclose(np.cos(t1 - phi)[moved], -np.cos(t0 - phi)[moved], atol=2e-6)
    assert np.allclose(np.sin(t1 - phi)[moved], np.sin(t0 - phi)[moved], atol=2e-6)
    # whole clusters move together
    assert (moved == moved[lab]).all()
    # bond energy inside clusters is unchanged
    for d in range(dim):
        nb = exact.neighbours(dim, L, d)
        same = lab == lab[nb]
        assert np.allclose(np.cos(t1 - t1[nb])[same], np.cos(t0 - t0[nb])[same], atol=2e-6)


# ----------------------------------------------------------------- moments
@pytest.mark.parametrize("dim,L", [(2, 7), (3, 5)])
def test_moments_vs_numpy(dim, L):
    N = L ** dim
    s = inputs.random_spins(ISING, N, 2, seed=2)
    m = oracle.moments(ISING, dim, L, 2, s)
    assert m["M"] == s.sum() and m["E"] == exact.ising_energy(s, dim, L)
    for q in (3, 5):
        p = inputs.random_spins(POTTS, N, q, seed=3)
        m = oracle.moments(POTTS, dim, L, q, p)
        assert m["E"] == exact.potts_energy(p, dim, L)
        assert m["M2"] == pytest.approx(exact.potts_m2_simplex(p, q), rel=1e-12)
    th = inputs.random_spins(XY, N, 2, seed=4).astype(np.float64)
    m = oracle.moments(XY, dim, L, 2, th.astype(np.float32))
    E = -sum(np.cos(th - th[exact.neighbours(dim, L, d)]).sum() for d in range(dim))
    assert m["e_xy"] == pytest.approx(E, rel=1e-12, abs=1e-9)
    assert m["M2"] == pytest.approx(np.cos(th).sum() ** 2 + np.sin(th).sum() ** 2, rel=1e-12, abs=1e-9)


def test_potts_m2_closed_forms():
    q, L = 4, 8
    N = L * L
    assert oracle.moments(POTTS, 2, L, q, np.zeros(N, np.uint8))["M2"] == N * N
    even = (np.arange(N) % q).astype(np.uint8)
    assert oracle.moments(POTTS, 2, L, q, even)["M2"] == 0.0


# ----------------------------------------------------------------- stationary law
def _binned(o: oracle.Oracle, bins: int, per_bin: int):
    rows = []
    for _ in range(bins):
        o.sweep(per_bin)
        a = o.take_acc()
        n = a["n_sweeps"]
        rows.append([a["sum_E"] / n, a["sum_M2"] / n, a["sum_M4"] / n, a["sum_E2"] / n])
    r = np.array(rows)
    return r.mean(0), r.std(0, ddof=1) / math.sqrt(bins)


def _check(mean, err, exact_vals, keys, nsig=4.5):
    for j, key in enumerate(keys):
        if key is None:
            continue
        assert abs(mean[j] - exact_vals[key]) < nsig * err[j] + 1e-9, (key, mean[j], exact_vals[key], err[j])


@pytest.mark.parametrize("dim,L,T", [(2, 4, 1.5), (2, 4, 2.269185), (2, 4, 3.5), (2, 3, 2.0),
                                     (3, 2, 3.0), (3, 2, 6.0)])
def test_ising_stationary_law_enumeration(dim, L, T):
    ex = exact.enumerate_ising(dim, L, T)
    o = oracle.Oracle(ISING, dim, L, 2, T, seed=31 + L)
    o.sweep(500, measure=False)
    mean, err = _binned(o, 24, 6000)
    _check(mean, err, ex, ["E", "M2", "M4", "E2"])


@pytest.mark.parametrize("dim,L,q,T", [(2, 3, 3, 0.9949), (2, 3, 4, 0.9102), (2, 3, 3, 2.0),
                                       (3, 2, 3, 1.2)])
def test_potts_stationary_law_enumeration(dim, L, q, T):
    ex = exact.enumerate_potts(dim, L, q, T)
    o = oracle.Oracle(POTTS, dim, L, q, T, seed=41 + q)
    o.sweep(500, measure=False)
    mean, err = _binned(o, 24, 6000)
    _check(mean, err, ex, ["E", "M2", "M4", None])


def test_kaufman_matches_enumeration():
    for T in (1.5, 2.269185, 3.5):
        assert exact.kaufman_energy(4, T) == pytest.approx(exact.enumerate_ising(2, 4, T)["E"], rel=1e-10)


@pytest.mark.parametrize("L", [16, 32])
def test_ising_energy_vs_kaufman(L):
    T = 2.269185
    o = oracle.Oracle(ISING, 2, L, 2, T, seed=1000)
    o.sweep(200, measure=False)
    mean, err = _binned(o, 20, 1500 if L == 16 else 500)
    ex = exact.kaufman_energy(L, T)
    assert abs(mean[0] - ex) < 4.5 * err[0], (mean[0], ex, err[0])


def test_density_of_states_matches_brute_enumeration():
    # the bit-permutation enumeration against the configuration-array one
    for dim, L in [(2, 4), (2, 3), (3, 2)]:
        for T in (1.5, 3.0):
            a, b = exact.ising_moments_from_dos(dim, L, T), exact.enumerate_ising(dim, L, T)
            for k in ("E", "E2", "M2", "M4"):
                assert a[k] == pytest.approx(b[k], rel=1e-12), (dim, L, T, k)


@pytest.mark.parametrize("T", [3.0, 4.5115])
def test_ising_3x3x3_enumeration(T):
    """3D Ising on the 3x3x3 torus, the smallest 3D lattice whose +d and -d
    bonds of a site are different pairs (all 2^27 states enumerated)."""
    ex = exact.ising_moments_from_dos(3, 3, T)
    o = oracle.Oracle(ISING, 3, 3, 2, T, seed=333)
    o.sweep(500, measure=False)
    mean, err = _binned(o, 24, 6000)
    o.close()
    _check(mean, err, ex, ["E", "M2", "M4", "E2"])


def test_binder_ratio_4x4_enumeration():
    """U = <M^4>/<M^2>^2 (Sec. 3) from the oracle's accumulators against the
    exact ratio of the 4x4 Ising torus at T_c (jackknife error over bins)."""
    T = 2.0 / math.log(1.0 + math.sqrt(2.0))
    ex = exact.enumerate_ising(2, 4, T)
    o = oracle.Oracle(ISING, 2, 4, 2, T, seed=404)
    o.sweep(500, measure=False)
    o.take_acc()
    m2, m4 = [], []
    for _ in range(24):
        o.sweep(6000)
        a = o.take_acc()
        m2.append(a["sum_M2"] / a["n_sweeps"])
        m4.append(a["sum_M4"] / a["n_sweeps"])
    o.close()
    U, err = _jackknife_ratio(np.array(m4), np.array(m2))
    assert abs(U - ex["M4"] / ex["M2"] ** 2) < 4.5 * err, (U, ex["M4"] / ex["M2"] ** 2, err)


def _jackknife_ratio(m4, m2):
    """U = mean(m4)/mean(m2)^2 and its jackknife standard error over bins."""
    n = m4.size
    jk = ((m4.sum() - m4) / (n - 1)) / ((m2.sum() - m2) / (n - 1)) ** 2
    return m4.mean() / m2.mean() ** 2, math.sqrt((n - 1) / n * ((jk - jk.mean()) ** 2).sum())


def test_kaufman_energy_at_the_critical_point_tends_to_minus_sqrt2():
    """At T_c = 2/ln(1 + sqrt 2) the infinite-lattice energy per site of the
    square-lattice Ising model is -sqrt 2 (Onsager); Kaufman's finite tori
    approach it as 1/L.  A fit e(L) = e_inf + a/L + b/L^2 over L = 64, 128,
    256 gives e_inf to 1e-6."""
    Tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    Ls = np.array([64.0, 128.0, 256.0])
    e = np.array([exact.kaufman_energy(int(L), Tc) / L ** 2 for L in Ls])
    A = np.stack([np.ones(3), 1.0 / Ls, 1.0 / Ls ** 2], axis=1)
    e_inf = np.linalg.solve(A, e)[0]
    assert abs(e_inf + math.sqrt(2.0)) < 1e-6, e_inf
    assert np.all(np.diff(np.abs(e + math.sqrt(2.0))) < 0)


def test_oracle_energy_at_the_2d_ising_critical_point():
    """The oracle at T_c = 2/ln(1 + sqrt 2) on the 32 x 32 torus: <E>
    within 3 standard errors of Kaufman's exact value."""
    L, Tc = 32, 2.0 / math.log(1.0 + math.sqrt(2.0))
    o = oracle.Oracle(ISING, 2, L, 2, Tc, seed=2269)
    o.sweep(300, measure=False)
    mean, err = _binned(o, 20, 600)
    o.close()
    ex = exact.kaufman_energy(L, Tc)
    assert abs(mean[0] - ex) < 3.0 * err[0], (mean[0], ex, err[0])


def _binder(model, L, q, T, seed, bins=12, per=1500):
    o = oracle.Oracle(model, 2, L, q, T, seed)
    o.sweep(1000, measure=False)
    o.take_acc()
    m2, m4 = [], []
    for _ in range(bins):
        o.sweep(per)
        a = o.take_acc()
        m2.append(a["sum_M2"] / a["n_sweeps"])
        m4.append(a["sum_M4"] / a["n_sweeps"])
    o.close()
    return _jackknife_ratio(np.array(m4), np.array(m2))


@pytest.mark.parametrize("model,q,Tc", [
    (ISING, 2, 2.0 / math.log(1.0 + math.sqrt(2.0))),
    (POTTS, 3, 1.0 / math.log(1.0 + math.sqrt(3.0))),
    (POTTS, 4, 1.0 / math.log(1.0 + math.sqrt(4.0)))])
def test_binder_crossing_brackets_the_critical_point(model, q, Tc):
    """The ratio U of L = 16 and L = 32 cross at the 2D critical point:
    below it U falls with L (order), above it U rises (disorder).  The sign
    of U(32) - U(16) at 0.97 T_c and at 1.03 T_c, each at least 5 standard
    errors, brackets the crossing within 3% of T_c = 2/ln(1 + sqrt 2)
    (Ising) and 1/ln(1 + sqrt q) (Potts, duality).  A wrong factor in the
    bond probability (2K for Potts) or in T would move it by tens of %."""
    for f, sign in [(0.97, -1.0), (1.03, 1.0)]:
        u16, e16 = _binder(model, 16, q, f * Tc, seed=600 + q)
        u32, e32 = _binder(model, 32, q, f * Tc, seed=700 + q)
        assert sign * (u32 - u16) > 5.0 * math.hypot(e16, e32), (f, u16, e16, u32, e32)


def test_potts_q2_is_ising_at_half_temperature():
    # H_Potts(q=2) = (H_Ising + const)/2 per bond: Potts at T/2 has the Ising
    # bond probability 1 - exp(-2/T).  Init and draw maps: Ising +1 <-> 0.
    for dim, L in [(2, 32), (3, 8)]:
        T = 2.7
        a = oracle.Oracle(ISING, dim, L, 2, T, seed=55)
        b = oracle.Oracle(POTTS, dim, L, 2, T / 2, seed=55)
        assert oracle.bond_threshold(ISING, T) == oracle.bond_threshold(POTTS, T / 2)
        assert np.array_equal(a.spins == 1, b.spins == 0)
        for _ in range(15):
            a.sweep(1)
            b.sweep(1)
            assert np.array_equal(a.planes, b.planes)
            assert np.array_equal(a.labels, b.labels)
            assert np.array_equal(a.spins == 1, b.spins == 0)


@pytest.mark.parametrize("dim,L,T", [(2, 4, 1.0), (3, 2, 1.6)])
def test_xy_stationary_law_vs_metropolis(dim, L, T):
    ref = exact.xy_metropolis(dim, L, T, chains=400, sweeps=1500, burn=200, seed=17)
    o = oracle.Oracle(XY, dim, L, 2, T, seed=19)
    o.sweep(300, measure=False)
    mean, err = _binned(o, 20, 5000)
    for j, key in [(0, "E"), (1, "M2")]:
        sig = math.hypot(err[j], ref[key + "_err"])
        assert abs(mean[j] - ref[key]) < 4.5 * sig, (key, mean[j], ref[key], sig)


def test_resume_from_state_is_exact():
    # state = spins + sweep counter (+ seed): a restored copy continues identically
    a = oracle.Oracle(POTTS, 2, 24, 3, 1.0, seed=8)
    a.sweep(7)
    b = oracle.Oracle(POTTS, 2, 24, 3, 1.0, seed=8)
    b.spins = a.spins
    b.sweep_counter = a.sweep_counter
    a.sweep(5)
    b.sweep(5)
    assert np.array_equal(a.spins, b.spins)


# ----------------------------------------------------------------- clock model
CLOCK = oracle.CLOCK


def test_clock_q4_is_two_ising_models_at_twice_the_temperature():
    # cos(t_i - t_j) = (s_i s_j + u_i u_j)/2 with s = cos + sin, u = cos - sin
    # in {+1,-1}: the 4-state clock at T is two independent Ising models at 2T.
    T = 1.2
    ex = exact.enumerate_ising(2, 4, 2 * T)
    o = oracle.Oracle(CLOCK, 2, 4, 4, T, seed=12)
    o.sweep(300, measure=False)
    mean, err = _binned(o, 24, 6000)
    # E = (E_s + E_u)/2 and M^2 = (M_s^2 + M_u^2)/2 of the two Ising models
    assert abs(mean[0] - ex["E"]) < 4.5 * err[0] and abs(mean[1] - ex["M2"]) < 4.5 * err[1]
    # the larger lattice against Kaufman's exact energy at 2T (critical point)
    o = oracle.Oracle(CLOCK, 2, 16, 4, 2.269185 / 2, seed=13)
    o.sweep(200, measure=False)
    mean, err = _binned(o, 20, 1500)
    kf = exact.kaufman_energy(16, 2.269185)
    assert abs(mean[0] - kf) < 4.5 * err[0], (mean[0], kf, err[0])


@pytest.mark.parametrize("dim,L,q,T", [(2, 3, 3, 0.8), (2, 3, 5, 0.9), (3, 2, 6, 1.5)])
def test_clock_stationary_law_enumeration(dim, L, q, T):
    ex = exact.enumerate_clock(dim, L, q, T)
    o = oracle.Oracle(CLOCK, dim, L, q, T, seed=71 + q)
    o.sweep(300, measure=False)
    mean, err = _binned(o, 24, 5000)
    _check(mean, err, ex, ["E", "M2", "M4", None])


def test_clock_512_approaches_xy():
    dim, L, T = 2, 4, 1.0
    ref = exact.xy_metropolis(dim, L, T, chains=400, sweeps=1500, burn=200, seed=23)
    o = oracle.Oracle(CLOCK, dim, L, 512, T, seed=29)
    o.sweep(300, measure=False)
    mean, err = _binned(o, 20, 5000)
    for j, key in [(0, "E"), (1, "M2")]:
        sig = math.hypot(err[j], ref[key + "_err"])
        assert abs(mean[j] - ref[key]) < 4.5 * sig, (key, mean[j], ref[key], sig)


@pytest.mark.parametrize("q", [2, 3, 4, 6, 512, 1024])
def test_clock_fixed_point_tables(q):
    c, s = oracle.clock_fixed(q)
    a = 2 * np.pi * np.arange(q) / q
    assert np.all(np.abs(c - np.cos(a) * 2.0 ** 30) <= 0.5 + 1e-6)
    assert np.all(np.abs(s - np.sin(a) * 2.0 ** 30) <= 0.5 + 1e-6)
    if q % 4 == 0:                                 # exact quarter turns
        assert c[0] == 2 ** 30 and c[q // 4] == 0 and c[q // 2] == -2 ** 30 and s[q // 4] == 2 ** 30


@pytest.mark.parametrize("dim,L,q", [(2, 17, 512), (3, 6, 5), (2, 8, 4)])
def test_clock_moments_are_fixed_point_sums(dim, L, q):
    """mx, my, E of a random clock state from integer sums of the rounded
    tables, recomputed here with numpy's own trig (and, for q = 4, the exact
    integer values)."""
    p = inputs.random_spins(CLOCK, L ** dim, q, seed=q + L).astype(np.int64)
    a = 2 * np.pi * np.arange(q) / q
    C = np.rint(np.cos(a) * 2.0 ** 30).astype(np.int64)
    S = np.rint(np.sin(a) * 2.0 ** 30).astype(np.int64)
    eb = sum(int(C[(p - p[exact.neighbours(dim, L, d)]) % q].sum()) for d in range(dim))
    rec = oracle.moments(CLOCK, dim, L, q, p.astype(np.uint16))
    assert rec["mx"] == float(int(C[p].sum())) * 2.0 ** -30
    assert rec["my"] == float(int(S[p].sum())) * 2.0 ** -30
    assert rec["e_xy"] == -(float(eb) * 2.0 ** -30)
    assert rec["M2"] == rec["mx"] * rec["mx"] + rec["my"] * rec["my"]
    # against the plain floating definition
    th = a[p]
    assert abs(rec["mx"] - np.cos(th).sum()) < 1e-6 * p.size
    e = -sum(np.cos(th - th[exact.neighbours(dim, L, d)]).sum() for d in range(dim))
    assert abs(rec["e_xy"] - e) < 1e-6 * p.size * dim


def test_clock_bonds_and_reflection():
    dim, L, q, T, seed = 2, 48, 64, 0.8, 3
    s = inputs.random_spins(CLOCK, L * L, q, seed=4)
    n_on, p_sum, var = 0, 0.0, 0.0
    for k in range(1, 21):
        m = oracle.clock_mirror(seed, k, q)
        assert 0 <= m < 2 * q
        x = np.sin(np.pi * ((2 * s.astype(np.int64) - m) % (2 * q)) / q)
        bits = inputs.unpack_planes(oracle.bonds(CLOCK, dim, L, q, T, seed, k, s), dim, L)
        for d in range(dim):
            prod = x * x[exact.neighbours(dim, L, d)]
            assert not (bits[d] & (prod <= 0)).any()
            p = np.where(prod > 0, -np.expm1(-2.0 / T * prod), 0.0)
            n_on += bits[d].sum()
            p_sum += p.sum()
            var += (p * (1 - p)).sum()
        lab = oracle.labels(dim, L, oracle.bonds(CLOCK, dim, L, q, T, seed, k, s))
        new, _ = oracle.flip(CLOCK, dim, L, q, seed, k, lab, s)
        moved = new != s                          # sites on the mirror line stay put
        xn = np.sin(np.pi * ((2 * new.astype(np.int64) - m) % (2 * q)) / q)
        assert np.allclose(xn[moved], -x[moved], atol=1e-12)
        assert np.all((new[moved].astype(np.int64) + s[moved]) % q == m % q)
        s = new
    assert abs(n_on - p_sum) < 5 * math.sqrt(var)
