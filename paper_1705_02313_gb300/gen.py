"""Seeded synthetic parity-game generators.

This module produces inputs only. It holds none of the solver's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.

Every random draw comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the 64-bit output
function as published by Vigna), used as a counter-based generator keyed by
(seed, stream, index, draw). Host code anywhere can therefore regenerate any
single vertex's data without generating the rest.

Game layout (CSR, int32): ``offsets[n+1]``, ``targets[m]``, ``owner[n]``
(uint8, 0 = Even, 1 = Odd) and ``pri[n]`` (int32). Each edge list is sorted
ascending and holds distinct targets; self-loops are allowed.

The paper measured on a suite of verification games that is not available
here; these generators are the stand-in (random games with permuted priorities,
ladder games, long successor chains, and batches of games of log-uniform size).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers: one per kind of draw
S_DEGREE, S_TARGET, S_OWNER, S_PRIORITY, S_BACKEDGE, S_CHAIN, S_BATCH = 1, 2, 3, 4, 5, 6, 7


def splitmix64(x):
    """SplitMix64: the value returned by the generator whose state is ``x``
    before the call (state advanced by the golden gamma, then mixed)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draw(seed, stream, index, j):
    """Counter-based draw: 64 random bits for (seed, stream, index, j)."""
    with np.errstate(over="ignore"):
        k = splitmix64(np.uint64(seed) ^ (np.uint64(stream) << np.uint64(56)))
        a = splitmix64(k ^ np.asarray(index, dtype=np.uint64))
        return splitmix64(a ^ np.asarray(j, dtype=np.uint64))


def uniform_below(bits, n):
    """Map 64 random bits to an integer in [0, n) using the top 32 bits."""
    n = np.asarray(n, dtype=np.uint64)
    return ((np.asarray(bits, dtype=np.uint64) >> np.uint64(32)) * n) >> np.uint64(32)


def batch_seed(i):
    """Seed of game ``i`` in a batch or a request stream."""
    return int(splitmix64(np.uint64(0x5EED) ^ np.uint64(i)))


@dataclass
class Game:
    n: int
    offsets: np.ndarray  # int32 [n+1]
    targets: np.ndarray  # int32 [m]
    owner: np.ndarray    # uint8 [n]
    pri: np.ndarray      # int32 [n]

    @property
    def m(self) -> int:
        return int(self.offsets[-1])

    def arrays(self):
        return self.offsets, self.targets, self.owner, self.pri


def permuted_priorities(n, seed):
    """A random permutation of 0..n-1: vertex v gets the rank of its key
    SplitMix64(seed, v) among all keys, ties broken by v."""
    keys = draw(seed, S_PRIORITY, np.arange(n, dtype=np.uint64), 0)
    order = np.argsort(keys, kind="stable")
    pri = np.empty(n, dtype=np.int32)
    pri[order] = np.arange(n, dtype=np.int32)
    return pri


def random_owners(n, seed, p_odd=0.5):
    bits = draw(seed, S_OWNER, np.arange(n, dtype=np.uint64), 0)
    thr = np.uint64(min(int(p_odd * 2.0**64), 2**64 - 1))
    return (bits < thr).astype(np.uint8)


def _distinct_targets(n, deg, seed):
    """For each vertex v, ``deg[v]`` distinct uniform targets in [0, n),
    sorted ascending. Slot j's r-th attempt uses counter j + 64 r; a draw that
    repeats an earlier slot of the same vertex is redrawn."""
    nv = deg.shape[0]
    dmax = int(deg.max()) if nv else 0
    slots = np.full((nv, max(dmax, 1)), np.iinfo(np.int64).max, dtype=np.int64)
    vid = np.arange(nv, dtype=np.uint64)
    for j in range(dmax):
        active = deg > j
        idx = np.nonzero(active)[0]
        attempt = 0
        pending = idx
        while pending.size:
            cand = uniform_below(draw(seed, S_TARGET, vid[pending], j + 64 * attempt), n).astype(np.int64)
            dup = np.zeros(pending.size, dtype=bool)
            for i in range(j):
                dup |= slots[pending, i] == cand
            ok = pending[~dup]
            slots[ok, j] = cand[~dup]
            pending = pending[dup]
            attempt += 1
    slots.sort(axis=1)
    mask = np.arange(slots.shape[1])[None, :] < deg[:, None]
    return slots[mask].astype(np.int32)


def _csr_from_degrees(deg):
    off = np.zeros(deg.shape[0] + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    if off[-1] >= 2**31:
        raise ValueError("edge count exceeds int32 CSR")
    return off.astype(np.int32)


def level_priorities(n, levels, seed):
    """Priorities drawn uniformly from 0..levels-1 (few distinct priorities,
    as in the verification games the paper measures)."""
    return uniform_below(draw(seed, S_PRIORITY, np.arange(n, dtype=np.uint64), 0), levels).astype(np.int32)


def random_game(n, dmin, dmax, seed=0, p_odd=0.5, levels=0):
    """Random game: out-degree uniform in [dmin, dmax] (capped at n), distinct
    uniform targets, owner Odd with probability p_odd, priorities a random
    permutation of 0..n-1 (levels = 0) or uniform over 0..levels-1."""
    if n <= 0:
        raise ValueError("n must be positive")
    dmin, dmax = min(dmin, n), min(dmax, n)
    v = np.arange(n, dtype=np.uint64)
    deg = (dmin + uniform_below(draw(seed, S_DEGREE, v, 0), dmax - dmin + 1)).astype(np.int64)
    off = _csr_from_degrees(deg)
    tgt = _distinct_targets(n, deg, seed)
    pri = level_priorities(n, levels, seed) if levels else permuted_priorities(n, seed)
    return Game(n, off, tgt, random_owners(n, seed, p_odd), pri)


def ladder_game(n, seed=0, p_odd=0.5):
    """Ladder / long-chain game: vertex i has the edge i -> i+1 and one back
    edge to j uniform in [0, i). Vertex 0 has only 0 -> 1; vertex n-1 has only
    its back edge. Owners and priorities as in the random game."""
    if n < 2:
        raise ValueError("ladder needs n >= 2")
    i = np.arange(n, dtype=np.int64)
    deg = np.full(n, 2, dtype=np.int64)
    deg[0] = 1
    deg[n - 1] = 1
    off = _csr_from_degrees(deg)
    back = uniform_below(draw(seed, S_BACKEDGE, i[1:].astype(np.uint64), 0), i[1:].astype(np.uint64)).astype(np.int64)
    tgt = np.empty(int(off[-1]), dtype=np.int64)
    tgt[0] = 1
    mid = np.arange(1, n - 1)
    tgt[off[mid]] = back[mid - 1]
    tgt[off[mid] + 1] = mid + 1
    tgt[off[n - 1]] = back[n - 2]
    return Game(n, off, tgt.astype(np.int32), random_owners(n, seed, p_odd), permuted_priorities(n, seed))


def chain_profile(n, seed=0, extra_degree=1):
    """A long successor chain for valuation-only runs: an all-Even game whose
    strategy sends pi[i] -> pi[i+1] along a random permutation pi, with
    pi[n-1] -> sink. Each vertex also has ``extra_degree`` random edges
    (merged with the chain edge when they coincide). Returns (game, sigma)
    with sigma[v] = -1 meaning the sink."""
    keys = draw(seed, S_CHAIN, np.arange(n, dtype=np.uint64), 0)
    pi = np.argsort(keys, kind="stable").astype(np.int64)
    nxt = np.full(n, -1, dtype=np.int64)
    nxt[pi[:-1]] = pi[1:]
    rows = [pi[:-1]]
    cols = [pi[1:]]
    if extra_degree:
        extra = _distinct_targets(n, np.full(n, extra_degree, dtype=np.int64), seed).astype(np.int64)
        rows.append(np.repeat(np.arange(n, dtype=np.int64), extra_degree))
        cols.append(extra)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    key = np.unique(rows * n + cols)
    rows, cols = key // n, key % n
    deg = np.bincount(rows, minlength=n).astype(np.int64)
    if (deg == 0).any():  # only the chain's last vertex, without extra edges
        lone = np.nonzero(deg == 0)[0]
        key = np.unique(np.concatenate([key, lone * n + lone]))
        rows, cols = key // n, key % n
        deg = np.bincount(rows, minlength=n).astype(np.int64)
    off = _csr_from_degrees(deg)
    owner = np.zeros(n, dtype=np.uint8)
    game = Game(n, off, cols.astype(np.int32), owner, permuted_priorities(n, seed))
    return game, nxt.astype(np.int32)


def log_uniform_sizes(count, lo, hi, seed=0):
    """``count`` sizes log-uniform in [lo, hi] (integers)."""
    u = (draw(seed, S_BATCH, np.arange(count, dtype=np.uint64), 0) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)
    sizes = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(sizes, lo, hi)


def batch_games(count, lo, hi, dmin, dmax, p_odd=0.5, seed=0):
    """A batch of random games; game i uses seed ``batch_seed(i)`` and a
    log-uniform size in [lo, hi]."""
    sizes = log_uniform_sizes(count, lo, hi, seed)
    return [random_game(int(sizes[i]), dmin, dmax, seed=batch_seed(i), p_odd=p_odd) for i in range(count)]


def named_config(name, seed=0):
    """The workloads measured by this project, by name."""
    if name == "random-1k":          # n = 1,000, out-degree U[1,4]
        return random_game(1000, 1, 4, seed)
    if name == "random-1m":          # n = 1,000,000, out-degree U[2,8]
        return random_game(1_000_000, 2, 8, seed)
    if name == "random-10m":         # n = 10,000,000, out-degree U[2,5]
        return random_game(10_000_000, 2, 5, seed)
    if name == "ladder-10m":         # n = 10,000,000 ladder
        return ladder_game(10_000_000, seed)
    raise KeyError(name)


# ---------------------------------------------------------------------------
# native generator (csrc/gen_host.c): the same random games, generated by C
# worker threads straight into caller buffers

_GEN = None


def _gen_lib():
    global _GEN
    if _GEN is None:
        from . import build
        path = build.build_gen()
        lib = ctypes.CDLL(path)
        i64, u64p, i64p, vp = ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p, ctypes.c_void_p
        lib.pggen_edge_counts.argtypes = [i64, i64p, u64p, i64, i64, i64p, ctypes.c_int]
        lib.pggen_fill_batch.argtypes = [i64, i64p, u64p, i64, i64, ctypes.c_uint64, i64p, i64p, vp, vp, vp, vp,
                                         ctypes.c_int]
        lib.pggen_fill_game.argtypes = [i64, i64, i64, ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp, vp,
                                        ctypes.c_int, i64]
        _GEN = lib
    return _GEN


def _owner_threshold(p_odd):
    return min(int(p_odd * 2.0**64), 2**64 - 1)


def _threads(nthreads):
    return int(nthreads or os.cpu_count() or 1)


def _addr(x):
    return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data


def native_random_game(n, dmin, dmax, seed=0, p_odd=0.5, nthreads=0, levels=0):
    """random_game(n, dmin, dmax, seed, p_odd, levels), generated by the C generator."""
    lib = _gen_lib()
    sizes = np.array([n], np.int64)
    seeds = np.array([seed], np.uint64)
    m = np.zeros(1, np.int64)
    if lib.pggen_edge_counts(1, sizes.ctypes.data, seeds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), dmin, dmax,
                             m.ctypes.data, 1):
        raise ValueError("bad generator arguments")
    if m[0] >= 2**31:
        raise ValueError("edge count exceeds int32 CSR")
    off = np.empty(n + 1, np.int32)
    tgt = np.empty(int(m[0]), np.int32)
    own = np.empty(n, np.uint8)
    pri = np.empty(n, np.int32)
    if lib.pggen_fill_game(n, dmin, dmax, seed, _owner_threshold(p_odd), off.ctypes.data, tgt.ctypes.data,
                           own.ctypes.data, pri.ctypes.data, _threads(nthreads), levels):
        raise ValueError("generator failed")
    return Game(n, off, tgt, own, pri)


def native_batch(count, lo, hi, dmin, dmax, p_odd=0.5, seed=0, nthreads=0, alloc=None, indices=None):
    """The batch of batch_games(count, lo, hi, dmin, dmax, p_odd, seed), packed
    in the pg_solve_batch layout. ``alloc(shape_len, numpy_dtype)`` may supply
    the four data buffers (for example pinned host tensors); by default numpy
    arrays are used. ``indices`` (optional) packs only those games of the
    batch, in that order (one rank's share). Returns (vtx_base, edge_base,
    offsets, targets, owner, pri)."""
    lib = _gen_lib()
    sizes = log_uniform_sizes(count, lo, hi, seed).astype(np.int64)
    ids = np.arange(count, dtype=np.int64) if indices is None else np.asarray(indices, dtype=np.int64)
    sizes = np.ascontiguousarray(sizes[ids])
    count = int(ids.size)
    seeds = np.array([batch_seed(int(i)) for i in ids], np.uint64)
    seeds_p = seeds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    ecount = np.zeros(count, np.int64)
    nt = _threads(nthreads)
    if lib.pggen_edge_counts(count, sizes.ctypes.data, seeds_p, dmin, dmax, ecount.ctypes.data, nt):
        raise ValueError("bad generator arguments")
    vtx_base = np.zeros(count + 1, np.int64)
    edge_base = np.zeros(count + 1, np.int64)
    np.cumsum(sizes, out=vtx_base[1:])
    np.cumsum(ecount, out=edge_base[1:])
    nv, ne = int(vtx_base[-1]), int(edge_base[-1])
    alloc = alloc or (lambda length, dt: np.empty(length, dt))
    off = alloc(nv + count, np.int32)
    tgt = alloc(ne, np.int32)
    own = alloc(nv, np.uint8)
    pri = alloc(nv, np.int32)
    if lib.pggen_fill_batch(count, sizes.ctypes.data, seeds_p, dmin, dmax, _owner_threshold(p_odd),
                            vtx_base.ctypes.data, edge_base.ctypes.data, _addr(off), _addr(tgt), _addr(own),
                            _addr(pri), nt):
        raise ValueError("generator failed")
    return vtx_base, edge_base, off, tgt, own, pri
