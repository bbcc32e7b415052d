"""Thin ctypes binding of the C ABI in include/sw.h (same names, argument
marshalling only).  Every step of the sweep runs in the CUDA library
libsw_gb300.so; if that library is missing this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SW_ISING, SW_POTTS, SW_XY, SW_CLOCK = 0, 1, 2, 3
SW_OK, SW_ERR_BAD_ARG, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_TIMEOUT, SW_ERR_RANGE = 0, -1, -2, -3, -4, -5

_lock = threading.Lock()
_lib = None


class SwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sw error {code}: {msg}")
        self.code = code


class sw_moments(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "n_sweeps", "sum_M2", "sum_M4", "sum_E", "sum_E2", "sum_nclusters",
        "U", "e_per_spin", "c_per_spin", "mean_cluster_size")]


class sw_record(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_uint64), ("M", ctypes.c_int64), ("E", ctypes.c_int64),
                ("nclusters", ctypes.c_int64), ("S2", ctypes.c_int64),
                ("mx", ctypes.c_double), ("my", ctypes.c_double), ("e_xy", ctypes.c_double),
                ("M2", ctypes.c_double), ("Ed", ctypes.c_double)]


# name -> (restype, argtypes); the full exported surface of include/sw.h
_vp, _sz, _u64, _i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
_SIGNATURES = {
    "sw_create": (_vp, [_i, _i, _i, _i, ctypes.c_double, _u64]),
    "sw_destroy": (None, [_vp]),
    "sw_last_error": (ctypes.c_char_p, []),
    "sw_sweep": (_i, [_vp, _i]),
    "sw_discard": (_i, [_vp, _i]),
    "sw_measure": (_i, [_vp, ctypes.POINTER(sw_moments)]),
    "sw_sync": (_i, [_vp]),
    "sw_set_loop_cap": (_i, [_vp, ctypes.c_longlong]),
    "sw_query": (_i, [_vp]),
    "sw_batch_query": (_i, [_vp]),
    "sw_set_stream": (_i, [_vp, _vp]),
    "sw_sweep_counter": (_u64, [_vp]),
    "sw_set_sweep_counter": (_i, [_vp, _u64]),
    "sw_num_sites": (_sz, [_vp]),
    "sw_spin_bytes": (_sz, [_vp]),
    "sw_bond_words": (_sz, [_vp]),
    "sw_get_spins": (_i, [_vp, _vp, _sz]),
    "sw_set_spins": (_i, [_vp, _vp, _sz]),
    "sw_get_spins_device": (_i, [_vp, _vp, _sz]),
    "sw_set_spins_device": (_i, [_vp, _vp, _sz]),
    "sw_get_labels": (_i, [_vp, _vp, _sz]),
    "sw_get_bonds": (_i, [_vp, _vp, _sz]),
    "sw_label_from_bonds": (_i, [_vp, _vp, _vp]),
    "sw_relabel": (_i, [_vp, _i, _vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_i)]),
    "sw_set_spins_async": (_i, [_vp, _vp, _sz]),
    "sw_get_spins_async": (_i, [_vp, _vp, _sz]),
    "sw_get_record_async": (_i, [_vp, _u64, ctypes.POINTER(sw_record)]),
    "sw_wait_io": (_i, [_vp]),
    "sw_get_series": (_i, [_vp, _u64, _sz, ctypes.POINTER(sw_record)]),
    "sw_series_capacity": (_sz, []),
    "sw_sweep_timed": (_i, [_vp, ctypes.POINTER(ctypes.c_float), _i]),
    "sw_label_from_bonds_noalloc": (_i, [_i, _i, _vp, _vp, _vp]),
    "sw_batch_create": (_vp, [_i]),
    "sw_batch_destroy": (None, [_vp]),
    "sw_batch_add": (_i, [_vp, _vp]),
    "sw_batch_remove": (_i, [_vp, _vp]),
    "sw_batch_sweep": (_i, [_vp, _i]),
    "sw_batch_set_stream": (_i, [_vp, _vp]),
    "sw_batch_size": (_sz, [_vp]),
    "sw_device_bytes": (_sz, [_i, _i, _i, _i]),
    "sw_set_sweep_target": (_i, [_vp, _u64]),
    "sw_batch_set_config": (_i, [_vp, _i, _i]),
    "sw_batch_get_config": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                 ctypes.POINTER(_i)]),
    "sw_batch_autotune": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_float)]),
}

SW_NOALLOC_MAX_SITES = 1 << 21
SW_LABEL_TILE_UF, SW_LABEL_EQUIVALENCE = 0, 1
SW_BATCH_TILE_SHAPES, SW_BATCH_SCHEDULES = 3, 8


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsw_gb300.so (build it first with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def sw_last_error() -> str:
    return lib().sw_last_error().decode()


def _check(rc: int):
    if rc != SW_OK:
        raise SwError(rc, sw_last_error())


def spin_dtype(model: int):
    return {SW_ISING: np.int8, SW_POTTS: np.uint8, SW_XY: np.float32, SW_CLOCK: np.uint16}[model]


class Handle:
    """An sw_handle* plus the arguments it was created with."""

    def __init__(self, ptr: int, model: int, dim: int, L: int, q: int, T: float, seed: int):
        self.ptr, self.model, self.dim, self.L, self.q, self.T, self.seed = ptr, model, dim, L, q, T, seed
        self.N = L ** dim

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def sw_create(model: int, dim: int, L: int, q: int, T: float, seed: int) -> Handle:
    ptr = lib().sw_create(model, dim, L, q, T, seed)
    if not ptr:
        raise SwError(SW_ERR_BAD_ARG, sw_last_error())
    return Handle(ptr, model, dim, L, q, T, seed)


def sw_destroy(h: Handle):
    if h is not None and h.ptr:
        lib().sw_destroy(h)
        h.ptr = 0


def sw_sweep(h: Handle, n: int):
    _check(lib().sw_sweep(h, n))


def sw_discard(h: Handle, n: int):
    _check(lib().sw_discard(h, n))


def sw_measure(h: Handle) -> dict:
    m = sw_moments()
    _check(lib().sw_measure(h, ctypes.byref(m)))
    return {f: getattr(m, f) for f, _ in sw_moments._fields_}


def sw_query(h: Handle) -> bool:
    """True once the work enqueued on the handle's stream has completed."""
    rc = lib().sw_query(h)
    if rc < 0:
        _check(rc)
    return rc == 1


def sw_set_loop_cap(h: Handle, cap: int):
    _check(lib().sw_set_loop_cap(h, int(cap)))


def sw_sync(h: Handle):
    _check(lib().sw_sync(h))


def sw_set_stream(h: Handle, stream: int):
    _check(lib().sw_set_stream(h, ctypes.c_void_p(stream)))


def sw_sweep_counter(h: Handle) -> int:
    return int(lib().sw_sweep_counter(h))


def sw_set_sweep_counter(h: Handle, k: int):
    _check(lib().sw_set_sweep_counter(h, k))


def sw_num_sites(h: Handle) -> int:
    return int(lib().sw_num_sites(h))


def sw_spin_bytes(h: Handle) -> int:
    return int(lib().sw_spin_bytes(h))


def sw_bond_words(h: Handle) -> int:
    return int(lib().sw_bond_words(h))


def sw_get_spins(h: Handle, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty(h.N, dtype=spin_dtype(h.model))
    _check(lib().sw_get_spins(h, out.ctypes.data, out.nbytes))
    return out


def sw_set_spins(h: Handle, spins: np.ndarray):
    s = np.ascontiguousarray(spins, dtype=spin_dtype(h.model))
    _check(lib().sw_set_spins(h, s.ctypes.data, s.nbytes))


def sw_get_spins_device(h: Handle, dev_ptr: int, nbytes: int):
    _check(lib().sw_get_spins_device(h, ctypes.c_void_p(dev_ptr), nbytes))


def sw_set_spins_device(h: Handle, dev_ptr: int, nbytes: int):
    _check(lib().sw_set_spins_device(h, ctypes.c_void_p(dev_ptr), nbytes))


def sw_get_labels(h: Handle) -> np.ndarray:
    out = np.empty(h.N, dtype=np.int32)
    _check(lib().sw_get_labels(h, out.ctypes.data, out.size))
    return out


def sw_get_bonds(h: Handle) -> np.ndarray:
    out = np.empty(sw_bond_words(h), dtype=np.uint32)
    _check(lib().sw_get_bonds(h, out.ctypes.data, out.size))
    return out


def sw_label_from_bonds(h: Handle, mask: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    if m.size != sw_bond_words(h):
        raise SwError(SW_ERR_BAD_ARG, "mask size != sw_bond_words")
    out = np.empty(h.N, dtype=np.int32)
    _check(lib().sw_label_from_bonds(h, m.ctypes.data, out.ctypes.data))
    return out


def sw_relabel(h: Handle, method: int, want_labels: bool = True):
    """Label the handle's current bond planes with SW_LABEL_TILE_UF or
    SW_LABEL_EQUIVALENCE; returns (labels or None, device ms, iterations)."""
    out = np.empty(h.N, dtype=np.int32) if want_labels else None
    ms = ctypes.c_float(0.0)
    it = ctypes.c_int(0)
    _check(lib().sw_relabel(h, method, out.ctypes.data if want_labels else None,
                            ctypes.byref(ms), ctypes.byref(it)))
    return out, float(ms.value), int(it.value)


def sw_set_spins_async(h: Handle, host: np.ndarray):
    """Enqueue the upload of `host` (a page-locked array, e.g. a numpy view
    of a pinned torch tensor, kept unchanged until sw_wait_io)."""
    _check(lib().sw_set_spins_async(h, host.ctypes.data, host.nbytes))


def sw_get_spins_async(h: Handle, host: np.ndarray):
    """Enqueue the download of the state into the page-locked array `host`
    (valid after sw_wait_io)."""
    _check(lib().sw_get_spins_async(h, host.ctypes.data, host.nbytes))


def sw_get_record_async(h: Handle, sweep: int, rec) -> None:
    """Enqueue the download of one sweep record into `rec`, a sw_record in
    page-locked memory (see record_buffer); valid after sw_wait_io."""
    _check(lib().sw_get_record_async(h, sweep, ctypes.byref(rec)))


def sw_wait_io(h: Handle):
    _check(lib().sw_wait_io(h))


def record_buffer(n: int):
    """n sw_record structs in page-locked host memory (kept alive by the
    returned object's `owner`)."""
    import torch
    t = torch.empty(n * ctypes.sizeof(sw_record), dtype=torch.uint8, pin_memory=True)
    arr = (sw_record * n).from_address(t.data_ptr())
    arr.owner = t
    return arr


def record_dict(rec) -> dict:
    return {f: getattr(rec, f) for f, _ in sw_record._fields_}


def sw_get_series(h: Handle, first: int, count: int) -> list[dict]:
    arr = (sw_record * max(count, 1))()
    _check(lib().sw_get_series(h, first, count, arr))
    return [{f: getattr(arr[k], f) for f, _ in sw_record._fields_} for k in range(count)]


def sw_sweep_timed(h: Handle) -> list[float]:
    """One measured sweep; device milliseconds of [bonds+tile labels, merge,
    flip, measurement]."""
    out = (ctypes.c_float * 4)()
    _check(lib().sw_sweep_timed(h, out, 4))
    return [float(v) for v in out]


def sw_label_from_bonds_noalloc(dim: int, L: int, dev_mask: int, dev_labels: int, stream: int = 0):
    """Labels of a device bond mask into a device int32 buffer, using the
    library's fixed scratch array instead of any allocation (pointers are
    device addresses, e.g. torch tensor data_ptr())."""
    _check(lib().sw_label_from_bonds_noalloc(dim, L, ctypes.c_void_p(dev_mask),
                                             ctypes.c_void_p(dev_labels), ctypes.c_void_p(stream)))


def sw_series_capacity() -> int:
    return int(lib().sw_series_capacity())


class Batch:
    """An sw_batch* (ragged batch of Ising/Potts lattices of one dimension)."""

    def __init__(self, ptr: int, dim: int):
        self.ptr, self.dim = ptr, dim

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def sw_batch_create(dim: int) -> Batch:
    ptr = lib().sw_batch_create(dim)
    if not ptr:
        raise SwError(SW_ERR_BAD_ARG, sw_last_error())
    return Batch(ptr, dim)


def sw_batch_destroy(b: Batch):
    if b is not None and b.ptr:
        lib().sw_batch_destroy(b)
        b.ptr = 0


def sw_batch_add(b: Batch, h: Handle):
    _check(lib().sw_batch_add(b, h))


def sw_batch_remove(b: Batch, h: Handle):
    _check(lib().sw_batch_remove(b, h))


def sw_batch_sweep(b: Batch, n: int):
    _check(lib().sw_batch_sweep(b, n))


def sw_batch_set_stream(b: Batch, stream: int):
    _check(lib().sw_batch_set_stream(b, ctypes.c_void_p(stream)))


def sw_batch_query(b: Batch) -> bool:
    """True once the batch's enqueued sweeps have completed."""
    rc = lib().sw_batch_query(b)
    if rc < 0:
        _check(rc)
    return rc == 1


def sw_batch_size(b: Batch) -> int:
    return int(lib().sw_batch_size(b))


def sw_set_sweep_target(h: Handle, target: int):
    """Batch sweeps of h stop when its sweep counter reaches target (0: none)."""
    _check(lib().sw_set_sweep_target(h, target))


def sw_batch_set_config(b: Batch, shape: int, schedule: int):
    _check(lib().sw_batch_set_config(b, shape, schedule))


def sw_batch_get_config(b: Batch) -> dict:
    """The batch's tile shape index, label schedule and tile extents."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().sw_batch_get_config(b, *[ctypes.byref(x) for x in v]))
    return {"shape": v[0].value, "schedule": v[1].value, "tile_y": v[2].value, "tile_z": v[3].value}


def sw_batch_autotune(b: Batch, sweeps: int) -> np.ndarray:
    """Times every (shape, schedule) on real sweeps of the batch and keeps the
    fastest; returns ms per sweep as [shape, schedule] (-1 where not tried)."""
    ms = (ctypes.c_float * (SW_BATCH_TILE_SHAPES * SW_BATCH_SCHEDULES))()
    _check(lib().sw_batch_autotune(b, sweeps, ms))
    return np.array(list(ms), dtype=np.float64).reshape(SW_BATCH_TILE_SHAPES, SW_BATCH_SCHEDULES)


def sw_device_bytes(model: int, dim: int, L: int, q: int) -> int:
    return int(lib().sw_device_bytes(model, dim, L, q))
