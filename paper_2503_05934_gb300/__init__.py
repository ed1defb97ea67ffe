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

from ._lib import HsortError, check, lib

NETSETS = {
    "none": 0x000, "3": 0x008, "3To4": 0x018, "3To5": 0x038, "6To8": 0x1C0,
    "3To8": 0x1F8, "PowerOf2": 0x110, "Even": 0x150, "Odd": 0x0A8,
}
ALGOS = {"merge": 0, "quick": 1}

__all__ = [
    "NETSETS", "ALGOS", "HsortError", "lib", "netset_mask", "algo_id",
    "hs_sort_workspace_bytes", "hs_sort_i32", "hs_sort_pairs_i32",
    "hs_sort_host_workspace_bytes", "hs_sort_i32_host", "hs_launch_count",
    "hs_prof_enable", "hs_prof_reset", "hs_prof_read", "hs_version", "hs_set_option",
    "hs_sort_i32_noalloc", "NOALLOC_MAX_KEYS",
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


NOALLOC_MAX_KEYS = 4194304


def hs_sort_i32_noalloc(keys: torch.Tensor, netset="6To8", stream=None) -> torch.Tensor:
    """Merge-sorts ``keys`` in place with the library's built-in scratch (no
    workspace, no device allocation); ``keys.numel()`` <= NOALLOC_MAX_KEYS."""
    _check_i32(keys, "keys")
    n = keys.numel()
    check(lib().hs_sort_i32_noalloc(keys.data_ptr() if n else None, n, netset_mask(netset),
                                    _stream_ptr(stream)))
    return keys


def hs_launch_count() -> int:
    return int(lib().hs_launch_count())


def hs_prof_enable(on: bool = True) -> None:
    lib().hs_prof_enable(1 if on else 0)


def hs_prof_reset() -> None:
    lib().hs_prof_reset()


def hs_prof_read(kernel: str) -> tuple[int, float]:
    """(launches, total milliseconds) of one kernel since the last reset."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    check(lib().hs_prof_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def hs_set_option(name: str, value: int) -> None:
    check(lib().hs_set_option(name.encode(), int(value)))


def hs_version() -> str:
    return lib().hs_version().decode()
