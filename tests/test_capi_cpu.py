"""The C-ABI library loads and exports every function include/sw.h declares;
argument validation fails cleanly without touching a GPU (CPU only)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def swlib():
    from paper_1403_7560_gb300 import build, sw
    build.build()
    return sw


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sw_create", "sw_sweep", "sw_measure", "sw_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(swlib):
    lib = ctypes.CDLL(swlib.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps exactly the declared surface
    assert sorted(swlib._SIGNATURES) == declared_functions()


@pytest.mark.parametrize("args,needle", [
    ((4, 2, 16, 2, 2.0, 1), "model"),
    ((3, 2, 16, 1, 1.0, 1), "clock q"),
    ((3, 2, 16, 1025, 1.0, 1), "clock q"),
    ((0, 4, 16, 2, 2.0, 1), "dim"),
    ((0, 2, 3, 2, 2.0, 1), "L must"),
    ((0, 2, 16, 2, 0.0, 1), "T must"),
    ((0, 2, 16, 2, float("nan"), 1), "T must"),
    ((1, 2, 16, 1, 1.0, 1), "q must"),
    ((1, 2, 16, 257, 1.0, 1), "q must"),
    ((1, 3, 257, 256, 1.0, 1), "too large"),
    ((0, 3, 1700, 2, 4.5, 1), "too large"),
])
def test_create_rejects_bad_arguments(swlib, args, needle):
    with pytest.raises(swlib.SwError) as e:
        swlib.sw_create(*args)
    assert needle in str(e.value)
    assert e.value.code == swlib.SW_ERR_BAD_ARG


def test_null_handle_calls_fail_cleanly(swlib):
    lib = swlib.lib()
    assert lib.sw_sweep(None, 1) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_discard(None, 1) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_measure(None, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_sync(None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_num_sites(None) == 0
    assert lib.sw_relabel(None, swlib.SW_LABEL_EQUIVALENCE, None, None, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_set_spins_async(None, None, 0) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_get_spins_async(None, None, 0) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_get_record_async(None, 1, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_wait_io(None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_batch_set_config(None, 0, 0) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_batch_get_config(None, None, None, None, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_batch_autotune(None, 1, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_set_sweep_target(None, 5) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_set_loop_cap(None, 0) == swlib.SW_ERR_BAD_ARG
    lib.sw_destroy(None)
    assert swlib.sw_series_capacity() >= 1024


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1403_7560_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "sw_oracle" not in text and "liboracle" not in text


def test_device_bytes_accounting(swlib):
    """sw_device_bytes (host arithmetic, no GPU): the spins, bond planes and
    forest at least; tile buffers sized for every batch tile shape for
    Ising/Potts; the clock tables; 0 for invalid arguments."""
    db = swlib.sw_device_bytes
    N = 256 ** 3
    ising = db(swlib.SW_ISING, 3, 256, 2)
    assert ising >= N + 3 * N // 8 + 4 * N
    # the 32x8x8 tiles of a batch: 8192 tiles of 576 hooked words, counted for a batchable lattice
    assert ising >= N + 3 * N // 8 + 4 * N + 8192 * 576 * 4
    assert db(swlib.SW_XY, 3, 256, 2) >= 4 * N + 3 * N // 8 + 4 * N
    q = 512
    assert db(swlib.SW_CLOCK, 3, 64, q) - db(swlib.SW_CLOCK, 3, 64, 3) >= 4 * (2 * q) ** 2 - 4 * 36
    assert db(swlib.SW_ISING, 2, 64, 2) < db(swlib.SW_ISING, 2, 128, 2) < db(swlib.SW_ISING, 2, 256, 2)
    for bad in ((9, 2, 16, 2), (0, 4, 16, 2), (0, 2, 3, 2), (0, 3, 2000, 2)):
        assert db(*bad) == 0
    # lattices no batch can hold (XY, clock) still get the tile buffers of the
    # single-lattice tiles: 2D L = 4096 in 32x128 tiles, 4096 tiles of 160
    # hooked words (the 32x256 tiles would need only 2048 x 288)
    n2 = 4096 ** 2
    for model in (swlib.SW_XY, swlib.SW_CLOCK):
        spin = 4 if model == swlib.SW_XY else 2
        assert db(model, 2, 4096, 4) >= spin * n2 + 2 * n2 // 32 + 4 * n2 + 4096 * 160 * 4 + 4096 * 4


@pytest.mark.parametrize("dim,L,mask,labels,needle", [
    (1, 16, 1, 1, "dim"), (4, 16, 1, 1, "dim"), (2, 3, 1, 1, "L must"),
    (2, 16, 0, 1, "NULL"), (2, 16, 1, 0, "NULL"),
    (3, 129, 1, 1, "too large"),                   # 129^3 = 2,146,689 > 2^21 sites
    (2, 1449, 1, 1, "too large"),                  # 1449^2 = 2,099,601 > 2^21 sites
])
def test_noalloc_rejects_bad_arguments_before_any_gpu_work(swlib, dim, L, mask, labels, needle):
    """sw_label_from_bonds_noalloc validates dim, L, its buffers and the
    scratch limit before any CUDA call, so it fails cleanly on a machine
    without a GPU (the pointers are never dereferenced)."""
    lib = swlib.lib()
    rc = lib.sw_label_from_bonds_noalloc(dim, L, 16 if mask else None, 16 if labels else None, None)
    assert rc == swlib.SW_ERR_BAD_ARG
    assert needle in swlib.sw_last_error()


def test_noalloc_limit_is_exact(swlib):
    """The scratch holds 2^21 sites: 128^3 (exactly 2^21) and 1448^2 fit,
    the next cube and square do not and are refused on the host."""
    lib = swlib.lib()
    assert 128 ** 3 <= swlib.SW_NOALLOC_MAX_SITES < 129 ** 3
    assert 1448 ** 2 <= swlib.SW_NOALLOC_MAX_SITES < 1449 ** 2
    assert lib.sw_label_from_bonds_noalloc(3, 129, 16, 16, None) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_label_from_bonds_noalloc(2, 1449, 16, 16, None) == swlib.SW_ERR_BAD_ARG


def test_loop_cap_argument_range(swlib):
    """sw_set_loop_cap refuses a NULL handle and caps above the production
    cap; it needs no GPU to check either."""
    lib = swlib.lib()
    assert lib.sw_set_loop_cap(None, -1) == swlib.SW_ERR_BAD_ARG
    assert lib.sw_set_loop_cap(None, 1 << 23) == swlib.SW_ERR_BAD_ARG
