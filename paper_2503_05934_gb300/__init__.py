"""hsort: hybrid network-leaf sorting of int32 keys on a GB300 (sm_103a).

A thin Python binding over the C-ABI library declared in ``include/hsort.h``.
Functions keep the C names; they only marshal torch tensors (device memory
and streams) into pointers.  Every step of every sort runs in the library's
CUDA kernels; if the library is missing, calls raise.

Network sets follow Table 3 of the paper (Sorting Network Configurations);
the algorithms are Algorithm 1 (merge) and Algorithm 2 (quick).
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import HsortError, Plan, SortPlan, check, lib

NETSETS = {
    "none": 0x000, "3": 0x008, "3To4": 0x018, "3To5": 0x038, "6To8": 0x1C0,
    "3To8": 0x1F8, "PowerOf2": 0x110, "Even": 0x150, "Odd": 0x0A8,
    "VarSort3": 0x10008, "VarSort4": 0x10010, "VarSort5": 0x10020,
}
ALGOS = {"merge": 0, "quick": 1}

__all__ = [
    "NETSETS", "ALGOS", "HsortError", "lib", "netset_mask", "algo_id",
    "hs_sort_workspace_bytes", "hs_sort_i32", "hs_sort_pairs_i32", "hs_sort_i64",
    "hs_sort_i64_workspace_bytes",
    "hs_sort_host_workspace_bytes", "hs_sort_i32_host", "hs_launch_count",
    "hs_prof_enable", "hs_prof_select", "hs_prof_reset", "hs_prof_read", "hs_version", "hs_set_option",
    "hs_sort_i32_noalloc", "NOALLOC_MAX_KEYS", "hs_device_check", "hs_bulk_wait_selftest",
    "Plan", "make_plan",
    "hs_segsort_workspace_bytes", "hs_segsort_i32", "hs_sort_i32_many", "Graph",
    "hs_segsort_capture", "hs_segsort_autotune", "hs_tune_cache_save", "hs_tune_cache_load",
    "Server", "hs_merge_split", "SortPlan", "hs_sort_autotune", "hs_sort_plan_for", "hs_tune_cache_clear", "hs_segsort_plan_for",
]


def netset_mask(netset) -> int:
    return NETSETS[netset] if isinstance(netset, str) else int(netset)


def algo_id(algo) -> int:
    return ALGOS[algo] if isinstance(algo, str) else int(algo)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


def _check_i32(t: torch.Tensor, name: str, device: bool = True) -> None:
    if t.dtype != torch.int32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous int32 tensor")
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def hs_sort_workspace_bytes(n: int, with_values: bool = False, algo="merge") -> int:
    return int(lib().hs_sort_workspace_bytes(n, 1 if with_values else 0, algo_id(algo)))


def _workspace(nbytes: int, device, ws: torch.Tensor | None) -> torch.Tensor:
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError("workspace tensor too small")
        return ws
    return torch.empty(max(nbytes, 16), dtype=torch.uint8, device=device)


def hs_sort_i32(keys: torch.Tensor, algo="merge", netset="6To8", ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Sorts ``keys`` (CUDA int32, contiguous) in place; returns ``keys``."""
    _check_i32(keys, "keys")
    n = keys.numel()
    need = hs_sort_workspace_bytes(n, False, algo)
    ws = _workspace(need, keys.device, ws)
    check(lib().hs_sort_i32(keys.data_ptr() if n else None, n, algo_id(algo), netset_mask(netset),
                            ws.data_ptr(), ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys


def hs_sort_pairs_i32(keys: torch.Tensor, vals: torch.Tensor, algo="merge", netset="6To8",
                      ws: torch.Tensor | None = None, stream=None):
    """Stable in-place key/value sort; returns (keys, vals)."""
    _check_i32(keys, "keys")
    _check_i32(vals, "vals")
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals differ in length")
    n = keys.numel()
    need = hs_sort_workspace_bytes(n, True, algo)
    ws = _workspace(need, keys.device, ws)
    check(lib().hs_sort_pairs_i32(keys.data_ptr() if n else None, vals.data_ptr() if n else None,
                                  n, algo_id(algo), netset_mask(netset), ws.data_ptr(),
                                  ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys, vals


def hs_sort_i64_workspace_bytes(n: int) -> int:
    return int(lib().hs_sort_i64_workspace_bytes(n))


def hs_sort_i64(keys: torch.Tensor, algo="merge", netset="6To8", ws: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Sorts ``keys`` (CUDA int64, contiguous) in place; returns ``keys``."""
    if keys.dtype != torch.int64 or not keys.is_contiguous() or not keys.is_cuda:
        raise ValueError("keys must be a contiguous int64 CUDA tensor")
    n = keys.numel()
    ws = _workspace(hs_sort_i64_workspace_bytes(n), keys.device, ws)
    check(lib().hs_sort_i64(keys.data_ptr() if n else None, n, algo_id(algo), netset_mask(netset),
                            ws.data_ptr(), ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys


def hs_sort_host_workspace_bytes(n: int, algo="merge") -> int:
    return int(lib().hs_sort_host_workspace_bytes(n, algo_id(algo)))


def hs_sort_i32_host(keys: torch.Tensor, algo="merge", netset="6To8", ws: torch.Tensor = None,
                     stream=None, device=None) -> torch.Tensor:
    """Host-buffer form: ``keys`` is a CPU int32 tensor (ideally pinned),
    sorted in place through the device; blocks until done."""
    _check_i32(keys, "keys", device=False)
    if keys.is_cuda:
        raise ValueError("hs_sort_i32_host takes a host tensor")
    n = keys.numel()
    need = hs_sort_host_workspace_bytes(n, algo)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    ws = _workspace(need, dev, ws)
    check(lib().hs_sort_i32_host(keys.data_ptr() if n else None, n, algo_id(algo),
                                 netset_mask(netset), ws.data_ptr(),
                                 ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys


def _i64_dev(t: torch.Tensor, name: str) -> None:
    if t.dtype != torch.int64 or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{name} must be a contiguous int64 CUDA tensor")


def make_plan(netset="6To8", block_threads=256, ctas_per_sm=0) -> Plan:
    return Plan(netset_mask(netset), int(block_threads), int(ctas_per_sm), 0)


def hs_segsort_workspace_bytes(n_keys: int, num_segs: int) -> int:
    return int(lib().hs_segsort_workspace_bytes(n_keys, num_segs))


def hs_segsort_i32(keys: torch.Tensor, offsets: torch.Tensor, algo="merge", netset="6To8",
                   plan: Plan | None = None, ws: torch.Tensor | None = None, stream=None):
    """Sorts every segment keys[offsets[i]:offsets[i+1]] in place, one launch."""
    _check_i32(keys, "keys")
    _i64_dev(offsets, "offsets")
    n, s = keys.numel(), offsets.numel() - 1
    ws = _workspace(hs_segsort_workspace_bytes(n, s), keys.device, ws)
    check(lib().hs_segsort_i32(keys.data_ptr(), n, offsets.data_ptr(), s, algo_id(algo),
                               netset_mask(netset), ctypes.byref(plan) if plan else None,
                               ws.data_ptr(), ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys


def hs_sort_i32_many(keys: torch.Tensor, offsets_host, algo="merge", netset="6To8",
                     ws: torch.Tensor | None = None, stream=None):
    """One hs_sort_i32 call per segment (offsets on the host)."""
    import numpy as np
    _check_i32(keys, "keys")
    off = np.ascontiguousarray(offsets_host, dtype=np.int64)
    longest = int(np.max(np.diff(off))) if off.size > 1 else 0
    ws = _workspace(hs_sort_workspace_bytes(longest, False, algo), keys.device, ws)
    check(lib().hs_sort_i32_many(keys.data_ptr(), keys.numel(), off.ctypes.data, off.size - 1,
                                 algo_id(algo), netset_mask(netset), ws.data_ptr(),
                                 ws.numel() * ws.element_size(), _stream_ptr(stream)))
    return keys


class Graph:
    """A captured batched sort (hs_graph); replay with launch()."""

    def __init__(self, handle: int, keep: tuple):
        self.handle = handle
        self._keep = keep  # buffers the graph reads and writes

    def launch(self, stream=None) -> None:
        check(lib().hs_graph_launch(self.handle, _stream_ptr(stream)))

    def destroy(self) -> None:
        if self.handle:
            lib().hs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hs_segsort_capture(keys: torch.Tensor, offsets: torch.Tensor, plan: Plan | None = None,
                       ws: torch.Tensor | None = None) -> Graph:
    _check_i32(keys, "keys")
    _i64_dev(offsets, "offsets")
    n, s = keys.numel(), offsets.numel() - 1
    ws = _workspace(hs_segsort_workspace_bytes(n, s), keys.device, ws)
    h = ctypes.c_void_p()
    check(lib().hs_segsort_capture(keys.data_ptr(), n, offsets.data_ptr(), s,
                                   ctypes.byref(plan) if plan else None, ws.data_ptr(),
                                   ws.numel() * ws.element_size(), ctypes.byref(h)))
    return Graph(h.value, (keys, offsets, ws))


def hs_segsort_autotune(keys: torch.Tensor, offsets: torch.Tensor, ws: torch.Tensor | None = None,
                        stream=None):
    """Returns (Plan, milliseconds) of the fastest candidate; keys unchanged."""
    _check_i32(keys, "keys")
    _i64_dev(offsets, "offsets")
    n, s = keys.numel(), offsets.numel() - 1
    ws = _workspace(int(lib().hs_segsort_autotune_workspace_bytes(n, s)), keys.device, ws)
    plan = Plan()
    ms = ctypes.c_double()
    check(lib().hs_segsort_autotune(keys.data_ptr(), n, offsets.data_ptr(), s, ws.data_ptr(),
                                    ws.numel() * ws.element_size(), _stream_ptr(stream),
                                    ctypes.byref(plan), ctypes.byref(ms)))
    return plan, float(ms.value)


def hs_sort_autotune(keys: torch.Tensor, netset="6To8", ws: torch.Tensor | None = None,
                     stream=None):
    """Times the single-array merge path's plans on ``keys``; returns (SortPlan,
    milliseconds) of the fastest and caches it for this size bucket; keys unchanged."""
    _check_i32(keys, "keys")
    n = keys.numel()
    ws = _workspace(int(lib().hs_sort_autotune_workspace_bytes(n)), keys.device, ws)
    plan = SortPlan()
    ms = ctypes.c_double()
    with torch.cuda.device(keys.device):
        check(lib().hs_sort_autotune(keys.data_ptr() if n else None, n, netset_mask(netset),
                                     ws.data_ptr(), ws.numel() * ws.element_size(),
                                     _stream_ptr(stream), ctypes.byref(plan), ctypes.byref(ms)))
    return plan, float(ms.value)


def hs_segsort_plan_for(n_keys: int, num_segs: int, netset="6To8") -> Plan:
    """The plan hs_segsort_i32 takes with no plan given for these sizes and set."""
    plan = Plan()
    check(lib().hs_segsort_plan_for(n_keys, num_segs, netset_mask(netset), ctypes.byref(plan)))
    return plan


def hs_sort_plan_for(n: int, netset="6To8", keys: torch.Tensor | None = None) -> SortPlan:
    """The plan the merge path takes now for ``n`` keys (aligned unless ``keys`` says
    otherwise).  Host only; reads the cache of the current CUDA device."""
    plan = SortPlan()
    check(lib().hs_sort_plan_for(keys.data_ptr() if keys is not None else None, n,
                                 netset_mask(netset), ctypes.byref(plan)))
    return plan


def hs_tune_cache_save(path: str) -> None:
    check(lib().hs_tune_cache_save(path.encode()))


def hs_tune_cache_load(path: str) -> None:
    check(lib().hs_tune_cache_load(path.encode()))


def hs_tune_cache_clear() -> None:
    lib().hs_tune_cache_clear()


class Server:
    """Continuous-batching sort server (hs_server_*) on the current device."""

    def __init__(self, budget_bytes: int):
        h = ctypes.c_void_p()
        check(lib().hs_server_create(int(budget_bytes), ctypes.byref(h)))
        self.handle = h.value

    def submit(self, keys: torch.Tensor, netset="6To8", algo="merge") -> int:
        _check_i32(keys, "keys")
        t = ctypes.c_uint64()
        n = keys.numel()
        check(lib().hs_server_submit(self.handle, keys.data_ptr() if n else None, n,
                                     algo_id(algo), netset_mask(netset), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int) -> tuple[int, float]:
        st = ctypes.c_int()
        lat = ctypes.c_double()
        check(lib().hs_server_wait(self.handle, ticket, ctypes.byref(st), ctypes.byref(lat)))
        return int(st.value), float(lat.value)

    def stats(self) -> dict:
        b, r, u = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t()
        check(lib().hs_server_stats(self.handle, ctypes.byref(b), ctypes.byref(r), ctypes.byref(u)))
        return {"batches": b.value, "batched_requests": r.value, "bytes_in_use": u.value}

    def replay(self, arrival_s, key_ptrs, sizes, netset="6To8"):
        """Submits requests at the given offsets (s) from now; returns
        (latencies_s, makespan_s)."""
        import numpy as np
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        ptrs = np.ascontiguousarray(key_ptrs, dtype=np.uint64)
        ns = np.ascontiguousarray(sizes, dtype=np.uint64)
        lat = np.zeros(arr.size, np.float64)
        mk = ctypes.c_double()
        check(lib().hs_server_replay(self.handle, arr.ctypes.data, ptrs.ctypes.data, ns.ctypes.data,
                                     arr.size, netset_mask(netset), lat.ctypes.data,
                                     ctypes.byref(mk)))
        return lat, float(mk.value)

    def destroy(self) -> None:
        if self.handle:
            lib().hs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


NOALLOC_MAX_KEYS = 4194304


def hs_sort_i32_noalloc(keys: torch.Tensor, netset="6To8", stream=None) -> torch.Tensor:
    """Merge-sorts ``keys`` in place with the library's built-in scratch (no
    workspace, no device allocation); ``keys.numel()`` <= NOALLOC_MAX_KEYS."""
    _check_i32(keys, "keys")
    n = keys.numel()
    # The library picks the scratch array of the current device: make it the
    # keys' device for the call (and take that device's stream by default).
    with torch.cuda.device(keys.device):
        check(lib().hs_sort_i32_noalloc(keys.data_ptr() if n else None, n, netset_mask(netset),
                                        _stream_ptr(stream)))
    return keys


def hs_launch_count() -> int:
    return int(lib().hs_launch_count())


def hs_prof_enable(on: bool = True) -> None:
    lib().hs_prof_enable(1 if on else 0)


def hs_prof_select(kernel: str | None) -> None:
    """Time only launches of `kernel` (None: every kernel)."""
    check(lib().hs_prof_select(kernel.encode() if kernel else None))


def hs_prof_reset() -> None:
    lib().hs_prof_reset()


def hs_prof_read(kernel: str) -> tuple[int, float]:
    """(launches, total milliseconds) of one kernel since the last reset."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    check(lib().hs_prof_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def hs_device_check(stream=None) -> None:
    """Waits for the stream and raises if a kernel reported a timed-out wait."""
    check(lib().hs_device_check(_stream_ptr(stream)))


def hs_bulk_wait_selftest(polls: int, stream=None) -> None:
    """Launches the bounded-wait diagnostic (a bulk-copy wait that can never
    complete, limited to `polls` polls); hs_device_check then reports it."""
    check(lib().hs_bulk_wait_selftest(int(polls), _stream_ptr(stream)))


def hs_merge_split(keys, starts, lens, rank: int, samp=None):
    """Host build of the four-way levels' K-way merge-path split: for output
    rank ``rank`` of the stable merge of runs ``keys[starts[i]:starts[i]+lens[i]]``
    (numpy int32, K = 2, 4 or 8 runs), the number of elements each run
    contributes to the first ``rank`` outputs.  ``samp`` (every 32nd key)
    makes the search read positions that are multiples of 32 from it."""
    import numpy as np
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    st = np.ascontiguousarray(starts, dtype=np.int64)
    ln = np.ascontiguousarray(lens, dtype=np.int64)
    if st.size != ln.size:
        raise ValueError("starts and lens differ in length")
    sp = None if samp is None else np.ascontiguousarray(samp, dtype=np.int32)
    out = np.zeros(ln.size, dtype=np.int64)
    rc = lib().hs_merge_split(keys.ctypes.data if keys.size else None,
                              sp.ctypes.data if sp is not None else None,
                              st.ctypes.data, ln.ctypes.data, int(ln.size), int(rank),
                              out.ctypes.data)
    if rc != 0:
        raise ValueError("hs_merge_split: invalid arguments")
    return out


def hs_set_option(name: str, value: int) -> None:
    check(lib().hs_set_option(name.encode(), int(value)))


def hs_version() -> str:
    return lib().hs_version().decode()
