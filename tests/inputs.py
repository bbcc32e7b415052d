"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds none of the SW arithmetic: only numpy random states, masks and the
workload table (model, dimension, L, temperature, seed, sweep counts) used by
the tests and the benchmark.
"""
from __future__ import annotations

import math

import numpy as np

ISING, POTTS, XY, CLOCK = 0, 1, 2, 3

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
    return {ISING: np.int8, POTTS: np.uint8, XY: np.float32, CLOCK: np.uint16}[model]


def random_spins(model: int, n: int, q: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if model == ISING:
        return (rng.integers(0, 2, n, dtype=np.int8) * 2 - 1).astype(np.int8)
    if model == POTTS:
        return rng.integers(0, q, n).astype(np.uint8)
    if model == CLOCK:
        return rng.integers(0, q, n).astype(np.uint16)
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


# ---------------------------------------------------------------- batch / serving
TC_3D_ISING = 1.0 / K_3D_ISING      # 4.511524
TC_3D_XY = 2.20184


def ragged_batch(n: int = 256, seed: int = 1003):
    """The ragged-batch workload: n 2D lattices, model uniform over
    {Ising, Potts q=3, Potts q=4}, L uniform over {32, 48, ..., 1024},
    T uniform in [0.8 Tc, 1.2 Tc], one seed per lattice.
    Returns a list of (model, dim, L, q, T, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = int(rng.integers(0, 3))
        model, q = (ISING, 2) if kind == 0 else (POTTS, 3 if kind == 1 else 4)
        L = 16 * int(rng.integers(2, 65))
        tc = TC_2D_ISING if model == ISING else tc_2d_potts(q)
        T = tc * float(rng.uniform(0.8, 1.2))
        out.append((model, 2, L, q, T, int(rng.integers(1, 2 ** 62))))
    return out


def small_batch(n: int = 256, seed: int = 1005):
    """Many small lattices: n 2D lattices, model uniform over {Ising, Potts
    q=3, Potts q=4}, L uniform over [16, 90] (at most 8192 sites, all of
    them within the one-CTA path's 2D limit),
    T uniform in [0.8 Tc, 1.2 Tc], one seed per lattice.
    Returns a list of (model, dim, L, q, T, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = int(rng.integers(0, 3))
        model, q = (ISING, 2) if kind == 0 else (POTTS, 3 if kind == 1 else 4)
        L = int(rng.integers(16, 91))
        tc = TC_2D_ISING if model == ISING else tc_2d_potts(q)
        T = tc * float(rng.uniform(0.8, 1.2))
        out.append((model, 2, L, q, T, int(rng.integers(1, 2 ** 62))))
    return out


def served_stream(n: int, seed: int = 1004, rate: float | None = None, max_L2: int = 4096,
                  max_L3: int = 256, sweeps=(100, 5000)):
    """The served request stream: n jobs, class uniform over {2D Ising, 3D
    Ising, 2D Potts q=3, 4, 8, 3D XY}, L log-uniform in [16, max_L2] (2D) or
    [16, max_L3] (3D), T = Tc (1 + U(-0.02, 0.02)), sweeps log-uniform in
    the given range, Poisson arrivals at `rate` jobs/s (all at t = 0 when
    rate is None).  Returns dicts with the job fields."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for k in range(n):
        kind = int(rng.integers(0, 6))
        if kind == 0:
            model, dim, q, tc = ISING, 2, 2, TC_2D_ISING
        elif kind == 1:
            model, dim, q, tc = ISING, 3, 2, TC_3D_ISING
        elif kind in (2, 3, 4):
            q = (3, 4, 8)[kind - 2]
            model, dim, tc = POTTS, 2, tc_2d_potts(q)
        else:
            model, dim, q, tc = XY, 3, 2, TC_3D_XY
        hi = max_L2 if dim == 2 else max_L3
        L = int(round(math.exp(rng.uniform(math.log(16), math.log(hi)))))
        T = tc * (1.0 + float(rng.uniform(-0.02, 0.02)))
        nsw = int(round(math.exp(rng.uniform(math.log(sweeps[0]), math.log(sweeps[1])))))
        if rate:
            t += float(rng.exponential(1.0 / rate))
        jobs.append(dict(id=k, model=model, dim=dim, L=L, q=q, T=T,
                         seed=int(rng.integers(1, 2 ** 62)), sweeps=nsw, arrival=t))
    return jobs
