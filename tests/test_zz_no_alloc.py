"""hs_sort_i32_noalloc, the allocation-free merge sort.

It serves callers that cannot allocate device memory (a plugin whose host
application owns all device allocations, code under a fixed device-memory
budget, latency-critical paths that must not risk a synchronising cudaMalloc).
Instead of a caller-provided workspace it uses one scratch array built into
the library, so its results must equal those of hs_sort_i32 with a workspace,
call after call, whatever the previous call left in that array.

This file is collected last on purpose, and it also passes when run alone in
a fresh process (the first call does the per-device set-up)."""
import ctypes

import numpy as np
import pytest

import hs_inputs as g
import oracle
from helpers import hs_module

pytestmark = pytest.mark.gpu

MAX_KEYS = 4194304
NETS_6TO8 = 0x1C0


def _noalloc(L, t, n, stream):
    return L.hs_sort_i32_noalloc(ctypes.c_void_p(t.data_ptr()), n, NETS_6TO8,
                                 ctypes.c_void_p(stream))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    hs = hs_module()
    L = hs.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # Two calls in a row: the largest allowed size, then a smaller ragged one
    # that runs over the scratch contents the first call left behind.
    for n, seed in [(MAX_KEYS, 41), (1_000_003, 42)]:
        a = g.random_i32(n, seed)
        want = torch.from_numpy(a).cuda()
        hs.hs_sort_i32(want, "merge", "6To8")  # existing entry point, own workspace
        got = torch.from_numpy(a).cuda()
        st = _noalloc(L, got, n, stream)
        assert st == 0, L.hs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), n
        assert np.all(np.diff(got.cpu().numpy().astype(np.int64)) >= 0)
        # and directly against the oracle's Algorithm 1
        assert np.array_equal(got.cpu().numpy(), oracle.merge_sort(a, "6To8")), n


def test_noalloc_python_binding_uses_the_keys_device():
    """The Python binding runs the call with the keys' device current (its
    scratch array and stream are that device's), and sorts as the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    hs = hs_module()
    a = g.random_i32(300_001, 43)
    t = torch.from_numpy(a).cuda()
    hs.hs_sort_i32_noalloc(t, "6To8")
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), oracle.merge_sort(a, "6To8"))


def test_noalloc_rejects_sizes_above_the_limit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    L = hs_module().lib()
    t = torch.zeros(8, dtype=torch.int32, device="cuda")
    # n is checked before the pointer is used or anything is launched.
    assert L.hs_sort_i32_noalloc(ctypes.c_void_p(t.data_ptr()), MAX_KEYS + 1, NETS_6TO8, None) == 1
    assert b"HS_NOALLOC_MAX_KEYS" in L.hs_last_error()
