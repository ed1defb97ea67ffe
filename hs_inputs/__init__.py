"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs.  It holds none of the sorting arithmetic and
serves the CUDA path and the CPU oracle alike; both receive the same host
arrays.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast Splittable
Pseudorandom Number Generators", OOPSLA 2014) used as a counter-based
generator: the i-th 64-bit output of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)`` with the published finaliser
``mix``.  Every draw is therefore a pure function of (seed, index), which keeps
chunked generation of very large arrays deterministic.

Distributions (the paper's workloads are random, sorted and nearly sorted
arrays; it gives no generator parameters):

* ``random``: uniform over the full int32 range.
* ``sorted``: ascending, spread over the full int32 range; built as a running
  sum of random gaps (no sort involved), so it has the density of a sorted
  uniform draw and may contain equal neighbours.
* ``nearly``: ``sorted``, then for ``floor(0.01 n)`` draws (i, j), each uniform
  in [0, n), a[i] and a[j] are swapped, in draw order.
* pair keys: 2^16 distinct values; u uniform in [0, 65535] mapped through the
  injection ``u -> (u * M) xor C (mod 2^32)`` with M odd and C drawn from the
  generator, viewed as int32; values are the original indices.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_U64 = 0xFFFFFFFFFFFFFFFF
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

SEED_BASE = 0x5EED0000


_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libhsgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles gen.c (the fast form of these generators) with plain gcc."""
    src = os.path.join(_HERE, "gen.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _clib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u64, i64, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        L.hsg_u32.argtypes = [u64, u64, u64, vp]
        L.hsg_sorted.argtypes = [u64, i64, vp]
        L.hsg_nearly.argtypes = [u64, i64, vp]
        L.hsg_segmented.argtypes = [u64, i64, vp, vp, vp]
        for f in (L.hsg_u32, L.hsg_sorted, L.hsg_nearly, L.hsg_segmented):
            f.restype = None
        _lib = L
    return _lib


def config_seed(config_id: int, salt: int = 0) -> int:
    """Seed of a workload: SEED_BASE + config id, plus an optional salt."""
    return (SEED_BASE + int(config_id) + (int(salt) << 32)) & 0xFFFFFFFFFFFFFFFF


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of stream ``seed`` as uint64."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        return _mix(z)


def _stream_u32(seed: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """Low 32 bits of the first n outputs, generated in chunks."""
    out = np.empty(n, np.uint32) if out is None else out
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        out[s:s + c] = (splitmix64(seed, s, c) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of each output."""
    return (splitmix64(seed, 0, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive), as int64 (floor of a scaled double)."""
    span = hi - lo + 1
    return lo + np.minimum((uniform01(seed, n) * span).astype(np.int64), span - 1)


def random_i32(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    if n:
        _clib().hsg_u32(seed & _U64, 0, n, out.ctypes.data)
    return out


def sorted_i32(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    if n:
        _clib().hsg_sorted(seed & _U64, n, out.ctypes.data)
    return out


def nearly_sorted_i32(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    if n:
        _clib().hsg_nearly(seed & _U64, n, out.ctypes.data)
    return out


def np_random_i32(n: int, seed: int) -> np.ndarray:
    """numpy form of random_i32 (the definition the C form must match)."""
    return _stream_u32(seed, n).view(np.int32)


def np_sorted_i32(n: int, seed: int) -> np.ndarray:
    """Ascending keys spanning [INT32_MIN, INT32_MAX] with random gaps."""
    if n == 0:
        return np.empty(0, np.int32)
    max_gap = max(1, (1 << 33) // n)  # mean gap ~ 2^32 / n
    out = np.empty(n, np.int32)
    acc = 0
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        gaps = (splitmix64(seed, s, c) % np.uint64(max_gap)).astype(np.int64)
        run = np.cumsum(gaps) + acc
        acc = int(run[-1])
        out[s:s + c] = np.clip(run - (1 << 31), -(1 << 31), (1 << 31) - 1).astype(np.int32)
    return out


def np_nearly_sorted_i32(n: int, seed: int) -> np.ndarray:
    a = np_sorted_i32(n, seed)
    k = n // 100
    if k == 0:
        return a
    draws = splitmix64(seed ^ 0x6E6561726C79, 0, 2 * k) % np.uint64(n)
    ii = draws[0::2].astype(np.int64).tolist()
    jj = draws[1::2].astype(np.int64).tolist()
    for i, j in zip(ii, jj):
        a[i], a[j] = a[j], a[i]
    return a


def keys(n: int, dist: str, seed: int) -> np.ndarray:
    """int32 keys of one distribution: 'random', 'sorted' or 'nearly'."""
    if dist == "random":
        return random_i32(n, seed)
    if dist == "sorted":
        return sorted_i32(n, seed)
    if dist == "nearly":
        return nearly_sorted_i32(n, seed)
    raise ValueError(dist)


def keys_i64(n: int, dist: str, seed: int) -> np.ndarray:
    """int64 keys: 'random' is each SplitMix64 output as a signed 64-bit word
    (uniform over the int64 range); 'sorted' is a running sum of random gaps
    spread over the int64 range (no sort involved); 'nearly' is the sorted
    keys with floor(n/100) sequential swaps of uniform pairs.  The sorted keys
    start near INT64_MIN and span about half the range."""
    if dist == "random":
        return splitmix64(seed ^ 0x693634, 0, n).view(np.int64).copy()
    if dist not in ("sorted", "nearly"):
        raise ValueError(dist)
    max_gap = np.uint64(max(1, (1 << 64) // max(n, 1) - 1))
    gaps = splitmix64(seed ^ 0x67617073, 0, n) % max_gap
    run = np.cumsum(gaps, dtype=np.uint64)  # below 2^64: n gaps of less than 2^64/n
    a = (run + np.uint64(1 << 63)).view(np.int64)  # shift to start near INT64_MIN
    if dist == "sorted":
        return a
    k = n // 100
    if k:
        draws = splitmix64(seed ^ 0x6E6561726C79, 0, 2 * k) % np.uint64(n)
        for i, j in zip(draws[0::2].astype(np.int64).tolist(), draws[1::2].astype(np.int64).tolist()):
            a[i], a[j] = a[j], a[i]
    return a


def pair_keys_16bit(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Keys from 2^16 distinct int32 values and values = original index."""
    u = (random_i32(n, seed).view(np.uint32) & np.uint32(0xFFFF)).astype(np.uint32)
    h = splitmix64(seed ^ 0x7061697273, 0, 2)
    mult = np.uint32((int(h[0]) & 0xFFFFFFFF) | 1)
    xor = np.uint32(int(h[1]) & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        k = ((u * mult) ^ xor).astype(np.uint32).view(np.int32)
    v = np.arange(n, dtype=np.int32)
    return k, v


def segment_sizes(num_segs: int, seed: int, lo: int = 3, hi: int = 65536) -> np.ndarray:
    """floor(exp(U(ln lo, ln(hi+1)))) clamped to [lo, hi] (log-uniform sizes)."""
    u = uniform01(seed, num_segs)
    s = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    return np.clip(s, lo, hi)


DISTS = ("random", "sorted", "nearly")


def segmented(num_segs: int, seed: int, lo: int = 3, hi: int = 65536,
              sizes: np.ndarray | None = None):
    """Concatenated segments with a per-segment distribution (C form of
    np_segmented).  Returns (keys, offsets[num_segs+1], dist_ids)."""
    sizes = segment_sizes(num_segs, seed, lo, hi) if sizes is None else np.asarray(sizes, np.int64)
    off = np.zeros(sizes.size + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    dist_ids = np.ascontiguousarray(uniform_int(seed ^ 0x64697374, sizes.size, 0, 2), np.int64)
    out = np.empty(int(off[-1]), np.int32)
    if sizes.size:
        _clib().hsg_segmented(seed & _U64, sizes.size, off.ctypes.data, dist_ids.ctypes.data,
                              out.ctypes.data)
    return out, off, dist_ids


def np_segmented(num_segs: int, seed: int, lo: int = 3, hi: int = 65536,
                 sizes: np.ndarray | None = None):
    """Concatenated segments with a per-segment distribution drawn uniformly
    from (random, sorted, nearly).  Returns (keys, offsets[num_segs+1], dist_ids).

    Random segments take their keys from one stream over the whole buffer.
    Sorted and nearly sorted segments are running sums of random gaps (one
    stream over their positions), each spread over the int32 range; nearly
    sorted ones then get floor(0.01 * size) sequential swaps of uniform pairs
    (one stream of draws, segment by segment)."""
    sizes = segment_sizes(num_segs, seed, lo, hi) if sizes is None else np.asarray(sizes, np.int64)
    num_segs = sizes.size
    off = np.zeros(num_segs + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    dist_ids = uniform_int(seed ^ 0x64697374, num_segs, 0, 2)
    out = np.empty(int(off[-1]), np.int32)
    _stream_u32(seed ^ 0x6B657973, out.size, out.view(np.uint32))
    sel = np.nonzero((dist_ids != 0) & (sizes > 0))[0]
    if sel.size:
        ssz = sizes[sel]
        starts = off[sel]
        # positions of all selected segments, segment by segment
        rel = np.arange(int(ssz.sum()), dtype=np.int64) - np.repeat(np.cumsum(ssz) - ssz, ssz)
        pos = np.repeat(starts, ssz) + rel
        max_gap = np.repeat(np.maximum(1, (1 << 33) // ssz), ssz).astype(np.uint64)
        gaps = (splitmix64(seed ^ 0x67617073, 0, pos.size) % max_gap).astype(np.int64)
        run = np.cumsum(gaps)
        first = np.cumsum(ssz) - ssz  # index of each segment's first position in `pos`
        base = np.repeat(run[first] - gaps[first], ssz)
        out[pos] = np.clip(run - base - (1 << 31), -(1 << 31), (1 << 31) - 1).astype(np.int32)
        near = sel[dist_ids[sel] == 2]
        k = sizes[near] // 100
        if k.sum() > 0:
            draws = splitmix64(seed ^ 0x6E656172, 0, 2 * int(k.sum()))
            seg_of = np.repeat(np.arange(near.size), k)
            span = sizes[near][seg_of].astype(np.uint64)
            b = off[near][seg_of]
            ii = (b + (draws[0::2] % span).astype(np.int64)).tolist()
            jj = (b + (draws[1::2] % span).astype(np.int64)).tolist()
            for i, j in zip(ii, jj):
                out[i], out[j] = out[j], out[i]
    return out, off, dist_ids


def log_uniform_sizes(n: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Sizes floor(exp(U(ln lo, ln(hi+1)))) clamped to [lo, hi]."""
    return segment_sizes(n, seed, lo, hi)


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = uniform01(seed, n)
    return np.cumsum(-np.log1p(-u) / rate_per_s)
