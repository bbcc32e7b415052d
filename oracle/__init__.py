"""CPU oracle for the Swendsen-Wang sweep (Komura & Okabe, Sec. 2).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
never does.  The arithmetic lives in ``sw_oracle.c`` (plain single-threaded
C, compiled with gcc without fast-math or FMA contraction); this module only
builds it and marshals numpy arrays through ctypes.

Pins: every function here is checked against something other than itself in
``tests/test_oracle_pins.py`` (Philox known answers, BFS components, exact
enumeration of small lattices, Kaufman's finite-lattice solution, the q=2
Potts / Ising identity, an independent XY Metropolis chain and closed forms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

ISING, POTTS, XY, CLOCK = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_sw.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sw_oracle.c into a shared library with gcc (IEEE semantics:
    no fast-math, no FMA contraction, so double sums round the same way on
    x86-64 and aarch64)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Record(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("E", ctypes.c_int64),
                ("nclusters", ctypes.c_int64), ("S2", ctypes.c_int64),
                ("mx", ctypes.c_double), ("my", ctypes.c_double),
                ("e_xy", ctypes.c_double), ("M2", ctypes.c_double),
                ("Ed", ctypes.c_double)]


class Acc(ctypes.Structure):
    _fields_ = [("n_sweeps", ctypes.c_double), ("sum_M2", ctypes.c_double),
                ("sum_M4", ctypes.c_double), ("sum_E", ctypes.c_double),
                ("sum_E2", ctypes.c_double), ("sum_nclusters", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, u32p, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_bond_threshold.argtypes = [ctypes.c_int, ctypes.c_double]
            L.oracle_bond_threshold.restype = ctypes.c_uint32
            L.oracle_xy_phi.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            L.oracle_xy_phi.restype = ctypes.c_float
            L.oracle_plane_words.argtypes = [ctypes.c_int, ctypes.c_int]
            L.oracle_plane_words.restype = ctypes.c_int64
            L.oracle_init.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint64, vp]
            L.oracle_bonds.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_uint64,
                                                            ctypes.c_uint32, vp, u32p]
            L.oracle_labels.argtypes = [ctypes.c_int, ctypes.c_int, u32p, i32p]
            L.oracle_flip.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint64, ctypes.c_uint32, i32p, vp]
            L.oracle_flip.restype = ctypes.c_int64
            L.oracle_moments.argtypes = [ctypes.c_int] * 4 + [vp, ctypes.POINTER(Record)]
            L.oracle_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_uint64]
            L.oracle_create.restype = vp
            L.oracle_destroy.argtypes = [vp]
            L.oracle_sweep.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            L.oracle_sweep_with_planes.argtypes = [vp, u32p, ctypes.c_int]
            L.oracle_spins.argtypes = [vp]
            L.oracle_spins.restype = vp
            L.oracle_planes.argtypes = [vp]
            L.oracle_planes.restype = vp
            L.oracle_label_array.argtypes = [vp]
            L.oracle_label_array.restype = vp
            L.oracle_sweep_counter.argtypes = [vp]
            L.oracle_sweep_counter.restype = ctypes.c_uint32
            L.oracle_set_sweep_counter.argtypes = [vp, ctypes.c_uint32]
            L.oracle_last_record.argtypes = [vp, ctypes.POINTER(Record)]
            L.oracle_take_acc.argtypes = [vp, ctypes.POINTER(Acc)]
            L.oracle_clock_thresholds.argtypes = [ctypes.c_int, ctypes.c_double, u32p]
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.oracle_clock_fixed.argtypes = [ctypes.c_int, i64p, i64p]
            L.oracle_clock_mirror.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]
            L.oracle_clock_mirror.restype = ctypes.c_uint32
            _lib = L
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def spin_dtype(model: int):
    return {ISING: np.int8, POTTS: np.uint8, XY: np.float32, CLOCK: np.uint16}[model]


def n_sites(dim: int, L: int) -> int:
    return L ** dim


def plane_words(dim: int, L: int) -> int:
    return int(lib().oracle_plane_words(dim, L))


# --------------------------------------------------------------------------
# Stand-alone steps (numpy in, numpy out)

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_u32p(c), _u32p(k), _u32p(out))
    return out


def bond_threshold(model: int, T: float) -> int:
    return int(lib().oracle_bond_threshold(model, T))


def xy_phi(seed: int, sweep: int) -> np.float32:
    return np.float32(lib().oracle_xy_phi(seed, sweep))


def clock_fixed(q: int):
    """Fixed-point tables round(2^30 cos(2 pi p / q)), round(2^30 sin(...))."""
    c = np.zeros(q, dtype=np.int64)
    s = np.zeros(q, dtype=np.int64)
    p64 = ctypes.POINTER(ctypes.c_int64)
    lib().oracle_clock_fixed(q, c.ctypes.data_as(p64), s.ctypes.data_as(p64))
    return c, s


def clock_thresholds(q: int, T: float) -> np.ndarray:
    t = np.zeros((2 * q, 2 * q), dtype=np.uint32)
    lib().oracle_clock_thresholds(q, T, _u32p(t))
    return t


def clock_mirror(seed: int, sweep: int, q: int) -> int:
    return int(lib().oracle_clock_mirror(seed, sweep, q))


def init_spins(model, dim, L, q, seed) -> np.ndarray:
    s = np.zeros(n_sites(dim, L), dtype=spin_dtype(model))
    lib().oracle_init(model, dim, L, q, seed, s.ctypes.data)
    return s


def bonds(model, dim, L, q, T, seed, sweep, spins) -> np.ndarray:
    s = np.ascontiguousarray(spins, dtype=spin_dtype(model))
    planes = np.zeros(plane_words(dim, L), dtype=np.uint32)
    lib().oracle_bonds(model, dim, L, q, T, seed, sweep, s.ctypes.data, _u32p(planes))
    return planes


def labels(dim, L, planes) -> np.ndarray:
    p = np.ascontiguousarray(planes, dtype=np.uint32)
    assert p.size == plane_words(dim, L)
    out = np.zeros(n_sites(dim, L), dtype=np.int32)
    if lib().oracle_labels(dim, L, _u32p(p), _i32p(out)) != 0:
        raise MemoryError("oracle_labels")
    return out


def flip(model, dim, L, q, seed, sweep, lab, spins):
    """Returns (new spins, number of clusters)."""
    s = np.array(spins, dtype=spin_dtype(model), copy=True)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    ncl = lib().oracle_flip(model, dim, L, q, seed, sweep, _i32p(lab), s.ctypes.data)
    return s, int(ncl)


def moments(model, dim, L, q, spins) -> dict:
    s = np.ascontiguousarray(spins, dtype=spin_dtype(model))
    r = Record()
    lib().oracle_moments(model, dim, L, q, s.ctypes.data, ctypes.byref(r))
    return {f: getattr(r, f) for f, _ in Record._fields_}


# --------------------------------------------------------------------------
# A whole run

class Oracle:
    """Single-threaded SW run with the same state and accumulators as the
    CUDA library's handle."""

    def __init__(self, model, dim, L, q, T, seed):
        self.model, self.dim, self.L, self.q, self.T, self.seed = model, dim, L, q, T, seed
        self.N = n_sites(dim, L)
        self._h = lib().oracle_create(model, dim, L, q, T, seed)
        if not self._h:
            raise ValueError("oracle_create: bad arguments")

    def close(self):
        if self._h:
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def sweep(self, n: int = 1, measure: bool = True):
        if lib().oracle_sweep(self._h, n, int(measure)) != 0:
            raise MemoryError("oracle_sweep")

    def sweep_with_planes(self, planes, measure: bool = True):
        p = np.ascontiguousarray(planes, dtype=np.uint32)
        assert p.size == plane_words(self.dim, self.L)
        if lib().oracle_sweep_with_planes(self._h, _u32p(p), int(measure)) != 0:
            raise MemoryError("oracle_sweep")

    def _view(self, ptr, count, dtype):
        buf = (ctypes.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
        return np.frombuffer(buf, dtype=dtype).copy()

    @property
    def spins(self) -> np.ndarray:
        return self._view(lib().oracle_spins(self._h), self.N, spin_dtype(self.model))

    @spins.setter
    def spins(self, value):
        v = np.ascontiguousarray(value, dtype=spin_dtype(self.model))
        assert v.size == self.N
        ctypes.memmove(lib().oracle_spins(self._h), v.ctypes.data, v.nbytes)

    @property
    def planes(self) -> np.ndarray:
        return self._view(lib().oracle_planes(self._h), plane_words(self.dim, self.L), np.uint32)

    @property
    def labels(self) -> np.ndarray:
        return self._view(lib().oracle_label_array(self._h), self.N, np.int32)

    @property
    def sweep_counter(self) -> int:
        return int(lib().oracle_sweep_counter(self._h))

    @sweep_counter.setter
    def sweep_counter(self, k: int):
        lib().oracle_set_sweep_counter(self._h, k)

    def last_record(self) -> dict:
        r = Record()
        lib().oracle_last_record(self._h, ctypes.byref(r))
        return {f: getattr(r, f) for f, _ in Record._fields_}

    def take_acc(self) -> dict:
        a = Acc()
        lib().oracle_take_acc(self._h, ctypes.byref(a))
        return {f: getattr(a, f) for f, _ in Acc._fields_}
