"""GPU parity of the quick path (Algorithm 2: median-of-three partitions with
network leaves) against the CPU oracle; keys have a unique sorted output, so
every case must match the oracle bit for bit."""
import numpy as np
import pytest

import hs_inputs as g
import oracle
from helpers import check_sorted_permutation, hs_module, to_dev

pytestmark = pytest.mark.gpu

PAPER_NETSETS = ["none", "3To5", "6To8", "3To8"]


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return hs_module()


def gpu_quick(hs, a, netset="6To8", offset=0):
    import torch
    t = to_dev(a, offset)
    hs.hs_sort_i32(t, "quick", netset)
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [25_000, 100_000, 1_000_000])
@pytest.mark.parametrize("dist", g.DISTS)
@pytest.mark.parametrize("netset", PAPER_NETSETS)
def test_paper_sizes_quick(hs, n, dist, netset):
    a = g.keys(n, dist, g.config_seed(1, salt=n))
    assert np.array_equal(gpu_quick(hs, a, netset), oracle.quick_sort(a, netset))


@pytest.mark.parametrize("netset", list(oracle.NETSETS))
def test_edge_sizes_quick(hs, netset):
    L = max([k for k in range(3, 9) if (oracle.NETSETS[netset] >> k) & 1] or [1])
    T = 1024 * L
    ST = 1024 * (3 if L == 1 else 2 * L - 1)  # the single-CTA sort's tile: the base case up to it
    sizes = sorted(set(range(0, 12)) | {T - 1, T, T + 1, 2 * T + 1, 8191, 8192, 8193,
                                        ST - 1, ST, ST + 1, 8192 * 3 + 1, (1 << 17) + 3, 500_001})
    for n in sizes:
        a = g.random_i32(n, 300 + n)
        assert np.array_equal(gpu_quick(hs, a, netset), oracle.quick_sort(a, netset)), n


@pytest.mark.parametrize("netset", ["6To8", "none", "3To5"])
def test_degenerate_quick(hs, netset):
    n = 300_007
    cases = {
        "all_equal": np.full(n, -5, np.int32),
        "two_values": np.where(g.random_i32(n, 3) > 0, 1, 0).astype(np.int32),
        "few_values": (g.random_i32(n, 4) % 5).astype(np.int32),
        "extremes": np.where(g.random_i32(n, 5) > 0, 2**31 - 1, -2**31).astype(np.int32),
        "reverse": np.arange(n, 0, -1, dtype=np.int32),
        "sorted": np.arange(n, dtype=np.int32),
        "organ_pipe": np.concatenate([np.arange(n // 2), np.arange(n - n // 2, 0, -1)]).astype(np.int32),
    }
    for name, a in cases.items():
        assert np.array_equal(gpu_quick(hs, a, netset), oracle.quick_sort(a, netset)), name


def test_unaligned_quick(hs):
    a = g.random_i32(400_003, 9)
    assert np.array_equal(gpu_quick(hs, a, "6To8", offset=3), np.sort(a))


@pytest.mark.parametrize("cap", [0, 1, 2, 5])
def test_depth_guard_fallback(hs, cap):
    """With the level cap forced low, the segments still open are finished by
    the merge path; the result must not change."""
    a = g.keys(600_000, "nearly", 12)
    hs.hs_set_option("quick_max_levels", cap)
    try:
        out = gpu_quick(hs, a, "6To8")
    finally:
        hs.hs_set_option("quick_max_levels", -1)
    assert np.array_equal(out, oracle.quick_sort(a, "6To8"))


def test_full_size_quick_2p28(hs):
    """2^28 uniform keys through the quick path (the benchmark's quick
    workload, same seed), equal element by element to the oracle's
    Algorithm 2."""
    n = 1 << 28
    a = g.random_i32(n, g.config_seed(2))
    out = gpu_quick(hs, a, "6To8")
    assert np.array_equal(out, oracle.quick_sort(a, "6To8"))


def test_large_quick_2p26(hs):
    import torch
    n = 1 << 26
    a = g.random_i32(n, g.config_seed(2, salt=7))
    t = to_dev(a)
    hs.hs_sort_i32(t, "quick", "6To8")
    torch.cuda.synchronize()
    out = t.cpu().numpy()
    del t
    check_sorted_permutation(a, out, samples=4)


@pytest.mark.parametrize("netset", ["6To8", "3To5", "none"])
def test_two_way_partition_option(hs, netset):
    """Option quick_partition = 2 (Algorithm 2's 2-way form, equal keys
    alternating sides): the oracle's Algorithm 2 (Hoare's scan) result on
    every distribution, few distinct keys, all-equal keys and sizes around
    the chunk and tile."""
    hs.hs_set_option("quick_partition", 2)
    try:
        for n in [7937, 8192, 8193, 100_000, 1_000_003]:
            for dist in g.DISTS:
                a = g.keys(n, dist, 7000 + n)
                assert np.array_equal(gpu_quick(hs, a, netset), oracle.quick_sort(a, netset)), (n, dist)
        for a in [np.full(300_001, 7, np.int32), (g.random_i32(500_000, 3) % 4).astype(np.int32),
                  np.concatenate([np.full(50_000, -1, np.int32), g.random_i32(50_000, 4)])]:
            assert np.array_equal(gpu_quick(hs, a, netset), np.sort(a))
    finally:
        hs.hs_set_option("quick_partition", 3)
