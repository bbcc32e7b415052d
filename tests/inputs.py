"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds none of the SW arithmetic: only numpy random states, masks and the
workload table (model, dimension, L, temperature, seed, sweep counts) used by
the tests and the benchmark.
"""
from __future__ import annotations

import math

import numpy as np

ISING, POTTS, XY = 0, 1, 2

# Critical couplings quoted for the workloads.
TC_2D_ISING = 2.0 / math.log(1.0 + math.sqrt(2.0))      # 2.269185...
K_3D_ISING = 0.2216546                                   # Sec. 3 (Bloete et al.)
K_3D_XY = 0.4541652                                      # near 1/2.20184 (Sec. 3)


def tc_2d_potts(q: int) -> float:
    return 1.0 / math.log(1.0 + math.sqrt(q))


# name -> (model, dim, L, q, T, seed, discard sweeps, measured sweeps)
WORKLOADS = {
    "ising2d_L64": (ISING, 2, 64, 2, 2.269185, 1000, 200, 1000),
    "ising3d_L256": (ISING, 3, 256, 2, 1.0 / K_3D_ISING, 1001, 100, 1000),
    "xy3d_L256": (XY, 3, 256, 2, 1.0 / K_3D_XY, 1002, 0, 1000),
}


def spin_dtype(model: int):
    return {ISING: np.int8, POTTS: np.uint8, XY: np.float32}[model]


def random_spins(model: int, n: int, q: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if model == ISING:
        return (rng.integers(0, 2, n, dtype=np.int8) * 2 - 1).astype(np.int8)
    if model == POTTS:
        return rng.integers(0, q, n).astype(np.uint8)
    return (rng.random(n, dtype=np.float32) * np.float32(2 * np.pi)).astype(np.float32) % np.float32(2 * np.pi)


def row_words(L: int) -> int:
    return (L + 31) // 32


def plane_words(dim: int, L: int) -> int:
    return dim * L ** (dim - 1) * row_words(L)


def pack_planes(bits: np.ndarray, dim: int, L: int) -> np.ndarray:
    """bits: bool array [dim, N] (bond (i,d) active) -> bit-plane words."""
    R = L ** (dim - 1)
    W = row_words(L)
    b = bits.reshape(dim, R, L)
    pad = np.zeros((dim, R, W * 32), dtype=bool)
    pad[:, :, :L] = b
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    words = (pad.reshape(dim, R, W, 32).astype(np.uint64) * weights).sum(axis=-1)
    return words.astype(np.uint32).reshape(-1)


def unpack_planes(planes: np.ndarray, dim: int, L: int) -> np.ndarray:
    R = L ** (dim - 1)
    W = row_words(L)
    w = np.asarray(planes, dtype=np.uint32).reshape(dim, R, W, 1)
    bits = ((w >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).reshape(dim, R, W * 32)
    return bits[:, :, :L].reshape(dim, L ** dim)


def random_mask(dim: int, L: int, density: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return pack_planes(rng.random((dim, L ** dim)) < density, dim, L)


def stripe_mask(dim: int, L: int, axis: int) -> np.ndarray:
    """Every bond along `axis` on, all others off: lines that wrap the torus."""
    bits = np.zeros((dim, L ** dim), dtype=bool)
    bits[axis] = True
    return pack_planes(bits, dim, L)


def spiral_mask(L: int) -> np.ndarray:
    """2D: one long path that winds inward through the whole lattice."""
    bits = np.zeros((2, L * L), dtype=bool)
    x0, y0, x1, y1 = 0, 0, L - 1, L - 1
    path = []
    while x0 <= x1 and y0 <= y1:
        path += [(x, y0) for x in range(x0, x1 + 1)]
        path += [(x1, y) for y in range(y0 + 1, y1 + 1)]
        if y0 < y1:
            path += [(x, y1) for x in range(x1 - 1, x0 - 1, -1)]
        if x0 < x1:
            path += [(x0, y) for y in range(y1 - 1, y0, -1)]
        x0, y0, x1, y1 = x0 + 1, y0 + 1, x1 - 1, y1 - 1
    for (xa, ya), (xb, yb) in zip(path, path[1:]):
        if ya == yb:
            x = min(xa, xb)
            bits[0, x + L * ya] = True
        else:
            y = min(ya, yb)
            bits[1, xa + L * y] = True
    return pack_planes(bits, 2, L)
