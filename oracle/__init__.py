"""Plain CPU oracle for the hybrid network-leaf sorts (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C,
single-threaded) through ctypes and shares no code with the CUDA library.

Algorithm 1 (Optimized Merge Sort with Sorting Networks) and Algorithm 2
(Optimized Quick Sort with Sorting Networks) are implemented step by step in
``oracle.c``; network sets follow Table 3 (Sorting Network Configurations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c"), os.path.join(HERE, "oracle.h")]

# Table 3 configurations as bitmasks (bit k: network of size k available).
NETSETS = {
    "none": 0x000,
    "PowerOf2": (1 << 4) | (1 << 8),
    "Even": (1 << 4) | (1 << 6) | (1 << 8),
    "Odd": (1 << 3) | (1 << 5) | (1 << 7),
    "3": 1 << 3,
    "3To4": (1 << 3) | (1 << 4),
    "3To5": (1 << 3) | (1 << 4) | (1 << 5),
    "3To8": 0x1F8,
    "6To8": (1 << 6) | (1 << 7) | (1 << 8),
    # VarSortk: any subarray of 2..k elements is a leaf, sorted by the size-k
    # network on a copy padded with +infinity (flag 0x10000 plus size bit k).
    "VarSort3": 0x10000 | (1 << 3),
    "VarSort4": 0x10000 | (1 << 4),
    "VarSort5": 0x10000 | (1 << 5),
}


class Counters(ctypes.Structure):
    _fields_ = [
        ("merge_calls", ctypes.c_uint64),
        ("net_calls", ctypes.c_uint64 * 9),
        ("partition_calls", ctypes.c_uint64),
        ("max_depth", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {
            "merge_calls": int(self.merge_calls),
            "net_calls": {k: int(self.net_calls[k]) for k in range(3, 9) if self.net_calls[k]},
            "partition_calls": int(self.partition_calls),
            "max_depth": int(self.max_depth),
        }


def build(force: bool = False) -> str:
    """Compiles oracle.c into a shared library (plain gcc, portable flags)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        lib_m = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in SOURCES):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
         "-o", tmp, SOURCES[0]])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        cp = ctypes.POINTER(Counters)
        L.or_network.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.or_network.restype = ctypes.c_int
        L.or_apply_network.argtypes = [ctypes.c_int, i32p]
        L.or_apply_network.restype = None
        L.or_merge.argtypes = [i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i32p]
        L.or_merge.restype = None
        L.or_merge_sort.argtypes = [i32p, ctypes.c_int64, ctypes.c_uint32, cp]
        L.or_merge_sort.restype = ctypes.c_int
        L.or_merge_sort_i64.argtypes = [i64p, ctypes.c_int64, ctypes.c_uint32, cp]
        L.or_merge_sort_i64.restype = ctypes.c_int
        L.or_median_of_three.argtypes = [i32p, ctypes.c_int64, ctypes.c_int64]
        L.or_median_of_three.restype = ctypes.c_int64
        L.or_hoare_partition.argtypes = [i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        L.or_hoare_partition.restype = ctypes.c_int64
        L.or_quick_sort.argtypes = [i32p, ctypes.c_int64, ctypes.c_uint32, cp]
        L.or_quick_sort.restype = ctypes.c_int
        L.or_merge_sort_pairs.argtypes = [i32p, i32p, ctypes.c_int64, ctypes.c_uint32, cp]
        L.or_merge_sort_pairs.restype = ctypes.c_int
        L.or_segsort.argtypes = [i32p, i64p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32]
        L.or_segsort.restype = ctypes.c_int
        L.or_is_sorted.argtypes = [i32p, ctypes.c_int64]
        L.or_is_sorted.restype = ctypes.c_int
        L.or_count_less.argtypes = [i32p, ctypes.c_int64, ctypes.c_int32]
        L.or_count_less.restype = ctypes.c_int64
        L.or_count_less_equal.argtypes = [i32p, ctypes.c_int64, ctypes.c_int32]
        L.or_count_less_equal.restype = ctypes.c_int64
        _lib = L
    return _lib


def _i32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i64(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def netset_mask(netset) -> int:
    return NETSETS[netset] if isinstance(netset, str) else int(netset)


def network(m: int) -> list[tuple[int, int]]:
    """Comparator list (lo, hi) of the oracle's size-m network."""
    buf = (ctypes.c_int * 64)()
    cnt = lib().or_network(m, buf, 32)
    if cnt < 0:
        raise ValueError(f"no network of size {m}")
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(cnt)]


def apply_network(m: int, a: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    assert out.size == m
    lib().or_apply_network(m, _i32(out))
    return out


def merge(a: np.ndarray, left: int, mid: int, right: int) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    tmp = np.empty(max(1, right - left + 1), np.int32)
    lib().or_merge(_i32(out), left, mid, right, _i32(tmp))
    return out


def merge_sort(a: np.ndarray, netset="6To8", counters: bool = False):
    """Algorithm 1 on a copy of ``a``; returns the sorted copy (and counters)."""
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    c = Counters()
    rc = lib().or_merge_sort(_i32(out), out.size, netset_mask(netset), ctypes.byref(c))
    if rc:
        raise ValueError(f"or_merge_sort failed ({rc})")
    return (out, c.as_dict()) if counters else out


def merge_sort_i64(a: np.ndarray, netset="6To8", counters: bool = False):
    """Algorithm 1 on a copy of the int64 array ``a``; returns the sorted copy
    (and counters)."""
    out = np.ascontiguousarray(a, dtype=np.int64).copy()
    c = Counters()
    rc = lib().or_merge_sort_i64(_i64(out), out.size, netset_mask(netset), ctypes.byref(c))
    if rc:
        raise ValueError(f"or_merge_sort_i64 failed ({rc})")
    return (out, c.as_dict()) if counters else out


def quick_sort(a: np.ndarray, netset="6To8", counters: bool = False):
    """Algorithm 2 on a copy of ``a``; returns the sorted copy (and counters)."""
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    c = Counters()
    rc = lib().or_quick_sort(_i32(out), out.size, netset_mask(netset), ctypes.byref(c))
    if rc:
        raise ValueError(f"or_quick_sort failed ({rc})")
    return (out, c.as_dict()) if counters else out


def merge_sort_pairs(keys: np.ndarray, vals: np.ndarray, netset="6To8"):
    """Stable key/value Algorithm 1; returns sorted copies (keys, vals)."""
    k = np.ascontiguousarray(keys, dtype=np.int32).copy()
    v = np.ascontiguousarray(vals, dtype=np.int32).copy()
    assert k.size == v.size
    rc = lib().or_merge_sort_pairs(_i32(k), _i32(v), k.size, netset_mask(netset), None)
    if rc:
        raise ValueError(f"or_merge_sort_pairs failed ({rc})")
    return k, v


def median_of_three(a: np.ndarray, low: int, high: int):
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    m = lib().or_median_of_three(_i32(out), low, high)
    return out, int(m)


def hoare_partition(a: np.ndarray, low: int, high: int, pivot_index: int):
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    j = lib().or_hoare_partition(_i32(out), low, high, pivot_index)
    return out, int(j)


def segsort(a: np.ndarray, offsets: np.ndarray, algo: str = "merge", netset="6To8",
            threads: int = 1) -> np.ndarray:
    """Sorts every segment a[off[i]:off[i+1]] on a copy (Algorithm 1 or 2
    per segment).  threads > 1 hands disjoint ranges of whole segments to
    that many host threads (the segments are independent; ctypes releases
    the GIL during each call), which changes nothing in the arithmetic."""
    out = np.ascontiguousarray(a, dtype=np.int32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    mode, mask = 0 if algo == "merge" else 1, netset_mask(netset)

    def run(s0: int, s1: int) -> int:
        if s1 <= s0:
            return 0
        sub = out[off[s0]:off[s1]]
        o = np.ascontiguousarray(off[s0:s1 + 1] - off[s0])
        return lib().or_segsort(_i32(sub), _i64(o), s1 - s0, mode, mask)

    if threads <= 1 or nseg < 2 * threads:
        rcs = [run(0, nseg)]
    else:
        import concurrent.futures as cf
        # ranges of about equal key counts
        cuts = np.searchsorted(off, np.linspace(off[0], off[-1], threads + 1)[1:-1])
        bounds = [0] + sorted(set(int(c) for c in cuts)) + [nseg]
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            rcs = list(ex.map(lambda ab: run(*ab), zip(bounds[:-1], bounds[1:])))
    if any(rcs):
        raise ValueError(f"or_segsort failed ({[r for r in rcs if r]})")
    return out


def is_sorted(a: np.ndarray) -> bool:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return bool(lib().or_is_sorted(_i32(a), a.size))


def count_less(a: np.ndarray, v: int) -> int:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return int(lib().or_count_less(_i32(a), a.size, int(v)))


def count_less_equal(a: np.ndarray, v: int) -> int:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return int(lib().or_count_less_equal(_i32(a), a.size, int(v)))
