"""The paper's labeler (label equivalence, Sec. 2) against the tile
union-find on the same bond planes, both through sw_relabel, both against
the oracle's canonical labels (needs a GB300)."""
from __future__ import annotations

import numpy as np
import pytest

import inputs
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


def both(sw, h):
    a, _, ia = sw.sw_relabel(h, sw.SW_LABEL_TILE_UF)
    b, _, ib = sw.sw_relabel(h, sw.SW_LABEL_EQUIVALENCE)
    assert ia == 1 and ib >= 1
    return a, b, ib


@pytest.mark.parametrize("dim,L", [(2, 4), (2, 33), (2, 64), (2, 130), (3, 4), (3, 9), (3, 32), (3, 37)])
@pytest.mark.parametrize("density", [0.2, 0.5, 0.75, 1.0])
def test_random_masks(sw, dim, L, density):
    h = sw.sw_create(ISING, dim, L, 2, 2.0, 1)
    try:
        m = inputs.random_mask(dim, L, density, seed=L * 11 + int(100 * density))
        ref = oracle.labels(dim, L, m)
        sw.sw_label_from_bonds(h, m)
        a, b, _ = both(sw, h)
        assert np.array_equal(a, ref)
        assert np.array_equal(b, ref)
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("dim,L", [(2, 8), (2, 64), (2, 96), (3, 6), (3, 24)])
def test_structured_masks(sw, dim, L):
    h = sw.sw_create(ISING, dim, L, 2, 2.0, 1)
    N = L ** dim
    try:
        off = inputs.pack_planes(np.zeros((dim, N), bool), dim, L)
        sw.sw_label_from_bonds(h, off)
        a, b, it = both(sw, h)
        assert np.array_equal(a, np.arange(N)) and np.array_equal(b, np.arange(N))
        assert it == 1                      # the first scan changes nothing
        on = inputs.pack_planes(np.ones((dim, N), bool), dim, L)
        sw.sw_label_from_bonds(h, on)
        a, b, _ = both(sw, h)
        assert (a == 0).all() and (b == 0).all()
        masks = [inputs.stripe_mask(dim, L, axis) for axis in range(dim)]
        if dim == 2:
            masks.append(inputs.spiral_mask(L))   # one long path: many iterations
        for m in masks:
            ref = oracle.labels(dim, L, m)
            sw.sw_label_from_bonds(h, m)
            a, b, _ = both(sw, h)
            assert np.array_equal(a, ref) and np.array_equal(b, ref)
    finally:
        sw.sw_destroy(h)


@pytest.mark.parametrize("model,dim,L,q,T", [
    (ISING, 3, 48, 2, 1 / 0.2216546),
    (ISING, 2, 64, 2, 2.269185314),
    (POTTS, 2, 50, 3, inputs.tc_2d_potts(3)),
    (XY, 3, 32, 2, 2.2),
])
def test_sweep_planes_and_state_untouched(sw, model, dim, L, q, T):
    """On the bonds of real sweeps both methods give the oracle's labels,
    and relabeling between sweeps leaves the run bit-identical."""
    seed = 77
    h = sw.sw_create(model, dim, L, q, T, seed)
    h2 = sw.sw_create(model, dim, L, q, T, seed)
    try:
        for _ in range(4):
            sw.sw_sweep(h, 1)
            sw.sw_sweep(h2, 1)
            planes = sw.sw_get_bonds(h)
            ref = oracle.labels(dim, L, planes)
            a, b, _ = both(sw, h)
            assert np.array_equal(a, ref) and np.array_equal(b, ref)
            assert np.array_equal(sw.sw_get_labels(h), ref)
        sw.sw_sweep(h, 3)
        sw.sw_sweep(h2, 3)
        assert np.array_equal(sw.sw_get_spins(h), sw.sw_get_spins(h2))
        assert sw.sw_get_series(h, 1, 7) == sw.sw_get_series(h2, 1, 7)
        assert sw.sw_measure(h) == sw.sw_measure(h2)
    finally:
        sw.sw_destroy(h)
        sw.sw_destroy(h2)


def test_critical_3d_L256(sw):
    """Full-size 3D Ising masks at K_c: both labelers, every site."""
    h = sw.sw_create(ISING, 3, 256, 2, 1 / 0.2216546, 1001)
    try:
        sw.sw_discard(h, 20)
        sw.sw_sweep(h, 1)
        ref = oracle.labels(3, 256, sw.sw_get_bonds(h))
        a, b, it = both(sw, h)
        assert np.array_equal(a, ref) and np.array_equal(b, ref)
        assert it < 200
    finally:
        sw.sw_destroy(h)


def test_bad_method(sw):
    h = sw.sw_create(ISING, 2, 16, 2, 2.0, 1)
    try:
        with pytest.raises(sw.SwError) as e:
            sw.sw_relabel(h, 7)
        assert e.value.code == sw.SW_ERR_BAD_ARG
    finally:
        sw.sw_destroy(h)
