"""Independent references the oracle is pinned against.

Nothing here calls the oracle or the CUDA path.  Each function is a textbook
definition or a library routine: connected components (scipy), exact
enumeration of small lattices, Kaufman's finite-lattice partition function of
the 2D Ising torus, the simplex-vector form of the Potts magnetization and a
single-site Metropolis chain for the XY model.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from inputs import unpack_planes


def neighbours(dim: int, L: int, d: int) -> np.ndarray:
    """Index of the +d neighbour of every site (periodic)."""
    idx = np.arange(L ** dim).reshape((L,) * dim)  # axes (z, y, x) / (y, x)
    axis = dim - 1 - d
    return np.roll(idx, -1, axis=axis).reshape(-1)


def components(dim: int, L: int, planes) -> np.ndarray:
    """Canonical component labels (minimum site index) of the active-bond
    graph, via scipy's connected_components."""
    N = L ** dim
    bits = unpack_planes(planes, dim, L)
    rows, cols = [], []
    for d in range(dim):
        i = np.nonzero(bits[d])[0]
        rows.append(i)
        cols.append(neighbours(dim, L, d)[i])
    r = np.concatenate(rows) if rows else np.zeros(0, int)
    c = np.concatenate(cols) if cols else np.zeros(0, int)
    g = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(N, N))
    _, comp = connected_components(g, directed=False)
    first = np.full(comp.max() + 1, N, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(N))
    return first[comp].astype(np.int32)


def ising_energy(s: np.ndarray, dim: int, L: int) -> np.ndarray:
    """E = -sum_<ij> s_i s_j for a batch of configurations s[..., N]."""
    s = s.astype(np.int64)
    return -sum((s * s[..., neighbours(dim, L, d)]).sum(-1) for d in range(dim))


def potts_energy(s: np.ndarray, dim: int, L: int) -> np.ndarray:
    """E = sum_<ij> (1 - delta(s_i, s_j))."""
    return sum((s != s[..., neighbours(dim, L, d)]).sum(-1) for d in range(dim))


def potts_m2_simplex(s: np.ndarray, q: int) -> np.ndarray:
    """|sum_i e_{s_i}|^2 with e_k the q vertices of a regular simplex in
    R^(q-1) scaled so that e_a . e_b = (q delta_ab - 1)/(q - 1)."""
    basis = np.eye(q) - 1.0 / q                 # centred vertices in R^q
    basis /= np.linalg.norm(basis[0])
    vec = basis[s.astype(np.int64)].sum(axis=-2)
    return (vec ** 2).sum(-1)


def enumerate_ising(dim: int, L: int, T: float) -> dict:
    N = L ** dim
    states = ((np.arange(2 ** N)[:, None] >> np.arange(N)) & 1).astype(np.int8) * 2 - 1
    E = ising_energy(states, dim, L).astype(np.float64)
    M = states.sum(-1).astype(np.float64)
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return {"E": (w * E).sum() / Z, "E2": (w * E * E).sum() / Z,
            "M2": (w * M ** 2).sum() / Z, "M4": (w * M ** 4).sum() / Z}


def enumerate_potts(dim: int, L: int, q: int, T: float) -> dict:
    N = L ** dim
    states = np.array(list(itertools.product(range(q), repeat=N)), dtype=np.uint8)
    E = potts_energy(states, dim, L).astype(np.float64)
    M2 = potts_m2_simplex(states, q)
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return {"E": (w * E).sum() / Z, "M2": (w * M2).sum() / Z,
            "M4": (w * M2 ** 2).sum() / Z}


def kaufman_lnZ(L: int, K, mp):
    """ln Z of the L x L periodic Ising model (B. Kaufman, Phys. Rev. 76,
    1232 (1949)), in the form Z = 1/2 (2 sinh 2K)^(N/2) (Z1+Z2+Z3+Z4) with
    cosh g_l = cosh 2K coth 2K - cos(l pi / L) and g_0 = 2K + ln tanh K."""
    K = mp.mpf(K)
    c = mp.cosh(2 * K) / mp.tanh(2 * K)

    def g(l):
        if l == 0:
            return 2 * K + mp.log(mp.tanh(K))
        return mp.acosh(c - mp.cos(mp.pi * l / L))

    z1 = z2 = z3 = z4 = mp.mpf(1)
    for r in range(L):
        go, ge = g(2 * r + 1), g(2 * r)
        z1 *= 2 * mp.cosh(L * go / 2)
        z2 *= 2 * mp.sinh(L * go / 2)
        z3 *= 2 * mp.cosh(L * ge / 2)
        z4 *= 2 * mp.sinh(L * ge / 2)
    return mp.log(mp.mpf(1) / 2) + (L * L / mp.mpf(2)) * mp.log(2 * mp.sinh(2 * K)) + mp.log(z1 + z2 + z3 + z4)


def kaufman_energy(L: int, T: float) -> float:
    """<E> = -d ln Z / dK at K = 1/T."""
    import mpmath as mp
    mp.mp.dps = 40
    return float(-mp.diff(lambda k: kaufman_lnZ(L, k, mp), mp.mpf(1) / mp.mpf(T)))


def xy_metropolis(dim: int, L: int, T: float, chains: int, sweeps: int, burn: int,
                  seed: int, step: float = 2.0) -> dict:
    """Single-site Metropolis for H = -sum cos(theta_i - theta_j), run as
    many independent chains with checkerboard updates (L even).  Returns the
    mean and standard error (over chains) of E and M^2."""
    assert L % 2 == 0
    rng = np.random.default_rng(seed)
    N = L ** dim
    th = rng.random((chains, N)) * 2 * np.pi
    nb = [neighbours(dim, L, d) for d in range(dim)]
    inv = [np.argsort(n) for n in nb]                      # -d neighbours
    coords = np.indices((L,) * dim).reshape(dim, -1).sum(0)
    parity = [np.nonzero(coords % 2 == p)[0] for p in (0, 1)]
    eacc = np.zeros(chains)
    macc = np.zeros(chains)
    nmeas = 0
    for sweep in range(burn + sweeps):
        for sites in parity:
            old = th[:, sites]
            new = old + (rng.random(old.shape) - 0.5) * 2 * step
            dE = np.zeros_like(old)
            for d in range(dim):
                for nbr in (nb[d][sites], inv[d][sites]):
                    tj = th[:, nbr]
                    dE += -np.cos(new - tj) + np.cos(old - tj)
            acc = rng.random(old.shape) < np.exp(-np.maximum(dE, 0) / T)
            th[:, sites] = np.where(acc, new, old) % (2 * np.pi)
        if sweep >= burn:
            E = -sum(np.cos(th - th[:, nb[d]]).sum(-1) for d in range(dim))
            M2 = np.cos(th).sum(-1) ** 2 + np.sin(th).sum(-1) ** 2
            eacc += E
            macc += M2
            nmeas += 1
    e, m = eacc / nmeas, macc / nmeas
    return {"E": e.mean(), "E_err": e.std(ddof=1) / math.sqrt(chains),
            "M2": m.mean(), "M2_err": m.std(ddof=1) / math.sqrt(chains)}


def enumerate_clock(dim: int, L: int, q: int, T: float) -> dict:
    """Exact <E>, <M^2>, <M^4> of the q-state clock model
    H = -sum cos(theta_i - theta_j), theta = 2 pi p / q, by enumeration."""
    N = L ** dim
    states = (np.arange(q ** N)[:, None] // (q ** np.arange(N))) % q
    th = 2 * np.pi * states / q
    E = -sum(np.cos(th - th[:, neighbours(dim, L, d)]).sum(-1) for d in range(dim))
    M2 = np.cos(th).sum(-1) ** 2 + np.sin(th).sum(-1) ** 2
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return {"E": (w * E).sum() / Z, "M2": (w * M2).sum() / Z, "M4": (w * M2 ** 2).sum() / Z}


_DOS_CACHE: dict = {}


def ising_density_of_states(dim: int, L: int, chunk_bits: int = 22) -> np.ndarray:
    """g[u, n]: the number of Ising configurations of the periodic L^dim
    lattice with u unsatisfied (antiparallel) bonds and n up spins, by
    enumeration of all 2^N states as N-bit integers (N <= 32).  The +d
    neighbour of every site is a fixed bit permutation, applied to a whole
    chunk of states with shifts and masks; u is the popcount of the state
    xor its permuted copy.  Cached per lattice."""
    key = (dim, L)
    if key in _DOS_CACHE:
        return _DOS_CACHE[key]
    N = L ** dim
    assert N <= 32
    groups = []
    for d in range(dim):
        nb = neighbours(dim, L, d)
        by_shift: dict = {}
        for i in range(N):
            by_shift[int(nb[i]) - i] = by_shift.get(int(nb[i]) - i, 0) | (1 << i)
        groups.append([(delta, np.uint32(mask)) for delta, mask in by_shift.items()])
    nbonds = dim * N
    hist = np.zeros((nbonds + 1) * (N + 1), dtype=np.int64)
    step = 1 << min(chunk_bits, N)
    for start in range(0, 1 << N, step):
        S = np.arange(start, start + step, dtype=np.uint64).astype(np.uint32)
        u = np.zeros(step, dtype=np.int64)
        for d in range(dim):
            R = np.zeros(step, dtype=np.uint32)
            for delta, mask in groups[d]:
                # bit i of R is bit nb(i) = i + delta of S
                R |= ((S >> np.uint32(delta)) if delta > 0 else (S << np.uint32(-delta))) & mask
            u += np.bitwise_count(S ^ R).astype(np.int64)
        n_up = np.bitwise_count(S).astype(np.int64)
        hist += np.bincount(u * (N + 1) + n_up, minlength=hist.size)
    g = hist.reshape(nbonds + 1, N + 1)
    _DOS_CACHE[key] = g
    return g


def ising_moments_from_dos(dim: int, L: int, T: float) -> dict:
    """Exact <E>, <E^2>, <M^2>, <M^4> of the Ising model (E = -sum s_i s_j,
    M = sum s_i) from the enumerated density of states."""
    g = ising_density_of_states(dim, L).astype(np.float64)
    N = L ** dim
    nbonds = dim * N
    E = -(nbonds - 2.0 * np.arange(nbonds + 1))[:, None]
    M = (2.0 * np.arange(N + 1) - N)[None, :]
    w = g * np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return {"E": (w * E).sum() / Z, "E2": (w * E * E).sum() / Z,
            "M2": (w * M ** 2).sum() / Z, "M4": (w * M ** 4).sum() / Z}
