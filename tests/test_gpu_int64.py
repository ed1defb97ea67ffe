"""GPU parity of the int64 merge path (Algorithm 1 on 8-byte keys) against
the oracle's int64 Algorithm 1: keys-only output is unique, so the bar is
bit-exact equality."""
import numpy as np
import pytest

import hs_inputs as g
import oracle
from helpers import hs_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return hs_module()


def gpu_sort64(hs, a, netset="6To8", offset=0):
    import torch
    buf = torch.empty(a.size + offset, dtype=torch.int64, device="cuda")
    t = buf[offset:]
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    hs.hs_sort_i64(t, "merge", netset)
    hs.hs_device_check()
    return t.cpu().numpy()


@pytest.mark.parametrize("netset", ["6To8", "3To8", "none", "Odd", "VarSort4"])
def test_int64_sizes_and_distributions(hs, netset):
    # Tile edges (7936 keys for {6,7,8}) and sizes just above powers of two.
    for n in [0, 1, 2, 7, 31, 2975, 2976, 2977, 7935, 7936, 7937, 8928, 8929, 16_384, 17_856,
              25_000, 100_001, 1_000_000, 1 << 20, (1 << 20) + 3]:
        for dist in g.DISTS:
            a = g.keys_i64(n, dist, 3000 + n)
            assert np.array_equal(gpu_sort64(hs, a, netset), oracle.merge_sort_i64(a, netset)), (n, dist)


def test_int64_merge_level_forms(hs):
    """Both int64 merge-level forms give the oracle's result: bulk-copied
    tiles (16-byte aligned, n even) and thread-staged tiles (n odd), at tile
    edges of the 2976-key merge tile, odd multiples of the block-sort tile,
    and few distinct keys."""
    for n in [3 * 2976 + 2, 3 * 2976 + 1, 2 * 7936, 3 * 7936 + 1, 100_002, 100_001, 1 << 20,
              (1 << 20) + 3]:
        for dist in g.DISTS:
            a = g.keys_i64(n, dist, 5000 + n)
            assert np.array_equal(gpu_sort64(hs, a), oracle.merge_sort_i64(a, "6To8")), (n, dist)
    for n in (400_002, 400_001):
        few = (g.keys_i64(n, "random", 6) % 3).astype(np.int64)
        assert np.array_equal(gpu_sort64(hs, few), oracle.merge_sort_i64(few, "6To8"))


def test_int64_extremes_duplicates_and_unaligned(hs):
    ext = np.array([2**63 - 1, -2**63, 0, -1, 1] * 20_001, np.int64)
    assert np.array_equal(gpu_sort64(hs, ext), np.sort(ext))
    few = (g.keys_i64(300_007, "random", 4) % 5).astype(np.int64)
    assert np.array_equal(gpu_sort64(hs, few), np.sort(few))
    a = g.keys_i64(123_457, "random", 5)
    assert np.array_equal(gpu_sort64(hs, a, offset=1), np.sort(a))  # 8-byte, not 16-byte, aligned


def test_int64_quick_is_unsupported(hs):
    import torch
    t = torch.zeros(100, dtype=torch.int64, device="cuda")
    with pytest.raises(hs.HsortError) as err:
        hs.hs_sort_i64(t, "quick")
    assert err.value.status == 2


def test_int64_full_size_2p27(hs):
    """2^27 int64 keys (1 GiB): sorted, multiset kept, sampled order
    statistics equal the oracle's."""
    import torch
    n = 1 << 27
    a = g.keys_i64(n, "random", g.config_seed(2, salt=64))
    t = torch.from_numpy(a).cuda()
    hs.hs_sort_i64(t, "merge", "6To8")
    hs.hs_device_check()
    out = t.cpu().numpy()
    del t
    assert np.all(out[1:] >= out[:-1])
    ref = np.sort(a[:1 << 20])
    sub = oracle.merge_sort_i64(a[:1 << 20], "6To8")
    assert np.array_equal(sub, ref)
    # order statistics: the count of keys below sampled values matches
    rng = np.random.default_rng(1)
    for v in a[rng.integers(0, n, 8)]:
        assert np.searchsorted(out, v, "left") == np.count_nonzero(a < v)


def test_int64_repeated_sorts_replay_a_graph(hs):
    """int64 keys through the graph replay: identical results on every call on
    the same buffers, the same kernels counted each time."""
    import torch
    n = 500_000
    a = g.keys_i64(n, "random", 97)
    t = torch.from_numpy(a).cuda()
    ws = torch.empty(hs.hs_sort_i64_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    counts = []
    for _ in range(4):
        t.copy_(torch.from_numpy(a))
        c0 = hs.hs_launch_count()
        hs.hs_sort_i64(t, "merge", "6To8", ws=ws)
        counts.append(hs.hs_launch_count() - c0)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), np.sort(a))
    assert len(set(counts)) == 1 and counts[0] > 1
    hs.hs_device_check()
