"""ctypes loader for the in-tree CUDA library ``_build/libhsort.so``.

There is no fallback: if the library is missing or fails to load, every call
raises.  The C declarations mirror ``include/hsort.h``.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhsort.so")

HS_OK = 0
STATUS = {0: "HS_OK", 1: "HS_ERR_INVALID_ARG", 2: "HS_ERR_UNSUPPORTED", 3: "HS_ERR_NO_MEMORY",
          4: "HS_ERR_CUDA", 5: "HS_ERR_TIMEOUT", 6: "HS_ERR_OVER_BUDGET"}

_c_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_u32 = ctypes.c_uint32
_int = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "hs_sort_workspace_bytes": (_sz, [_sz, _int, _int]),
    "hs_sort_i32": (_int, [_vp, _sz, _int, _u32, _vp, _sz, _vp]),
    "hs_sort_pairs_i32": (_int, [_vp, _vp, _sz, _int, _u32, _vp, _sz, _vp]),
    "hs_sort_i64_workspace_bytes": (_sz, [_sz]),
    "hs_sort_i64": (_int, [_vp, _sz, _int, _u32, _vp, _sz, _vp]),
    "hs_sort_host_workspace_bytes": (_sz, [_sz, _int]),
    "hs_sort_i32_host": (_int, [_vp, _sz, _int, _u32, _vp, _sz, _vp]),
    "hs_sort_i32_noalloc": (_int, [_vp, _sz, _u32, _vp]),
    "hs_segsort_workspace_bytes": (_sz, [_sz, _sz]),
    "hs_segsort_i32": (_int, [_vp, _sz, _vp, _sz, _int, _u32, _vp, _vp, _sz, _vp]),
    "hs_sort_i32_many": (_int, [_vp, _sz, _vp, _sz, _int, _u32, _vp, _sz, _vp]),
    "hs_segsort_capture": (_int, [_vp, _sz, _vp, _sz, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "hs_graph_launch": (_int, [_vp, _vp]),
    "hs_graph_destroy": (None, [_vp]),
    "hs_segsort_autotune_workspace_bytes": (_sz, [_sz, _sz]),
    "hs_segsort_autotune": (_int, [_vp, _sz, _vp, _sz, _vp, _sz, _vp, _vp,
                                   ctypes.POINTER(ctypes.c_double)]),
    "hs_sort_autotune_workspace_bytes": (_sz, [_sz]),
    "hs_sort_autotune": (_int, [_vp, _sz, _u32, _vp, _sz, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "hs_sort_plan_for": (_int, [_vp, _sz, _u32, _vp]),
    "hs_segsort_plan_for": (_int, [_sz, _sz, _u32, _vp]),
    "hs_tune_cache_save": (_int, [ctypes.c_char_p]),
    "hs_tune_cache_load": (_int, [ctypes.c_char_p]),
    "hs_tune_cache_clear": (None, []),
    "hs_server_create": (_int, [_sz, ctypes.POINTER(_vp)]),
    "hs_server_submit": (_int, [_vp, _vp, _sz, _int, _u32, ctypes.POINTER(ctypes.c_uint64)]),
    "hs_server_wait": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_int),
                              ctypes.POINTER(ctypes.c_double)]),
    "hs_server_stats": (_int, [_vp, ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_sz)]),
    "hs_server_replay": (_int, [_vp, _vp, _vp, _vp, _sz, _u32, _vp,
                                ctypes.POINTER(ctypes.c_double)]),
    "hs_server_destroy": (None, [_vp]),
    "hs_status_str": (ctypes.c_char_p, [_int]),
    "hs_last_error": (ctypes.c_char_p, []),
    "hs_version": (ctypes.c_char_p, []),
    "hs_launch_count": (ctypes.c_uint64, []),
    "hs_prof_enable": (None, [_int]),
    "hs_prof_select": (_int, [ctypes.c_char_p]),
    "hs_prof_reset": (None, []),
    "hs_prof_read": (_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(ctypes.c_double)]),
    "hs_set_option": (_int, [ctypes.c_char_p, ctypes.c_int64]),
    "hs_device_check": (_int, [_vp]),
    "hs_bulk_wait_selftest": (_int, [_u32, _vp]),
    "hs_keys_tile": (_sz, [_u32, _sz]),
    "hs_pairs_tile": (_sz, [_u32]),
    "hs_i64_tile": (_sz, [_u32, _sz]),
    "hs_network_pairs": (_int, [_int, ctypes.POINTER(ctypes.c_int), _int]),
    "hs_network_apply": (_int, [_int, _c_i32p]),
    "hs_merge_split": (_int, [_vp, _vp, _vp, _vp, _int, ctypes.c_int64, _vp]),
}


class Plan(ctypes.Structure):
    """hs_plan: leaf network set and persistent-kernel shape of the batched form."""
    _fields_ = [("netset", ctypes.c_uint32), ("block_threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"netset": int(self.netset), "block_threads": int(self.block_threads),
                "ctas_per_sm": int(self.ctas_per_sm)}


class SortPlan(ctypes.Structure):
    """hs_sort_plan: block-sort CTA size and merge fan-in of the single-array merge path."""
    _fields_ = [("blocksort_threads", ctypes.c_int32), ("merge_fanin", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self) -> dict:
        return {"blocksort_threads": int(self.blocksort_threads),
                "merge_fanin": int(self.merge_fanin)}


class HsortError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Loads the library once; raises if it is absent (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"hsort CUDA library not built: {LIB_PATH} is missing "
                              "(run paper_2503_05934_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != HS_OK:
        msg = lib().hs_last_error().decode(errors="replace")
        raise HsortError(status, msg)
