"""The error bounds behind the kernels' fast paths, checked on CPU with the
same float32 operations (numpy rounds each float32 operation to nearest;
the one transcendental, the GPU's __expf(x), is given the maximum error the
CUDA documentation states for it, 2 + floor(|1.173 x|) ulp).

XY bonds: the exp estimate stays far inside the 2^-16 margin of its
expm1f fallback (test_xy_exp_estimate_within_its_margin).

Clock model bonds: the kernel decides u < t[k_a][k_b] from the float
estimate pf = 1 - exp(-(2/T) x_a x_b) with x_k = float(sin(pi k / q)) and
reads the exact table entry only when |u - pf| <= 2^-16 + (2/T) 2^-20.  Its
claimed error bound is (2/T) 2.5e-7 + 4e-7: every pair of states must stay
inside it, the margin must be at least three times it, and a product that is
not positive in float must belong to a zero table entry."""
from __future__ import annotations

import math

import numpy as np
import pytest


def expf_error(arg, e):
    """Documented worst-case error of __expf(arg) around its float result e:
    2 + floor(|1.173 arg|) units in the last place of e."""
    n_ulp = 2.0 + np.floor(np.abs(1.173 * arg.astype(np.float64)))
    return n_ulp * np.spacing(e).astype(np.float64)


def exact_table(q: int, T: float):
    """Bond thresholds t[a][b] = floor(-expm1(-(2/T) x_a x_b) 2^32), 0 where
    x_a x_b <= 0, x_k = sin(pi k / q), all in double (the definition)."""
    k = np.arange(2 * q, dtype=np.float64)
    x = np.sin(np.pi * k / q)
    prod = x[:, None] * x[None, :]
    t = np.floor(-np.expm1(-(2.0 / T) * prod) * 4294967296.0)
    t = np.where(prod > 0.0, np.minimum(t, 4294967295.0), 0.0)
    return x, t


@pytest.mark.parametrize("q", [6, 64, 512, 1024])
@pytest.mark.parametrize("T", [0.15, 0.5, 2.20184, 50.0])
def test_clock_threshold_estimate_within_its_margin(q, T):
    x, t = exact_table(q, T)
    xf = x.astype(np.float32)
    prod = xf[:, None] * xf[None, :]                       # float32 products, rounded
    twoK = np.float32(2.0 / T)
    a = (twoK * prod).astype(np.float32)
    e = np.exp(-a).astype(np.float32)
    expf_extra = expf_error(-a, e)                           # __expf's documented bound
    pf = (np.float32(1.0) - e).astype(np.float32)
    pos = prod > 0
    err = np.abs(pf.astype(np.float64) - t / 4294967296.0) + expf_extra
    bound = float(twoK) * 2.5e-7 + 4e-7
    margin = 2.0 ** -16 + float(twoK) * 2.0 ** -20
    assert err[pos].max() <= bound
    assert margin >= 3.0 * bound
    # a product that is not positive in float has a zero threshold
    assert np.all(t[~pos] == 0.0)
    # the draw's float conversion adds at most 2^-25 (u < 1): inside the margin's slack
    assert margin - bound > 2.0 ** -25


@pytest.mark.parametrize("T", [0.05, 0.89, 2.20184, 50.0])
def test_xy_exp_estimate_within_its_margin(T):
    """XY bonds: from the (accurate) projection product, the kernel takes
    p from 1 - __expf(-2K prod) and calls expm1f only when the draw lies
    within 2^-16 of it; the estimate must stay far inside that margin for
    every product in (0, 1]."""
    prod = np.linspace(1e-7, 1.0, 2_000_001, dtype=np.float64).astype(np.float32)
    twoK = np.float32(2.0 / T)
    a = (twoK * prod).astype(np.float32)
    e = np.exp(-a).astype(np.float32)
    pf = (np.float32(1.0) - e).astype(np.float64)
    exact = -np.expm1(-a.astype(np.float64))
    assert (np.abs(pf - exact) + expf_error(-a, e)).max() < 2.0 ** -16 / 8


def test_invariant_divisor_multiplication_is_exact_for_small_lattices():
    """The small-lattice kernel divides by L, W and R*W with the
    multiply-high of Granlund & Montgomery: m = floor((2^32 - 1) / d) + 1 and
    floor(n / d) = (n * m) >> 32 for n * d < 2^32.  Every divisor up to the
    largest small lattice (8192 sites) with every dividend up to three times
    that (the kernel's largest, D * R * W) gives the exact quotient."""
    n = np.arange(3 * 8192, dtype=np.uint64)
    for d in range(2, 8193):
        m = np.uint64((2 ** 32 - 1) // d + 1)
        assert np.array_equal((n * m) >> np.uint64(32), n // np.uint64(d)), d
