"""GPU parity of the merge path (Algorithm 1) against the CPU oracle.

Every case compares the CUDA result with the oracle element by element on
the same seeded input; keys and stable pairs have a unique correct output, so
the bar is bit-exact equality.  Full-size cases (2^28 keys, 2^27 pairs) are
checked by properties that hold at any size plus oracle order statistics."""
import numpy as np
import pytest

import hs_inputs as g
import oracle
from helpers import (check_sorted_permutation, check_stable_pairs_index_values, hs_module,
                     to_dev)

pytestmark = pytest.mark.gpu

ALL_NETSETS = list(oracle.NETSETS)
PAPER_NETSETS = ["none", "3To5", "6To8", "3To8"]


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return hs_module()


def gpu_sort(hs, a, algo="merge", netset="6To8", offset=0):
    import torch
    t = to_dev(a, offset)
    hs.hs_sort_i32(t, algo, netset)
    hs.hs_device_check()  # no kernel gave up on a bounded wait
    return t.cpu().numpy()


def gpu_sort_pairs(hs, k, v, netset="6To8", offset=0):
    import torch
    tk, tv = to_dev(k, offset), to_dev(v, offset)
    hs.hs_sort_pairs_i32(tk, tv, "merge", netset)
    hs.hs_device_check()
    return tk.cpu().numpy(), tv.cpu().numpy()


def test_ten_thousand_uniform_6to8(hs):
    """n = 10,000 uniform over the int32 range, {6,7,8} leaves, against the
    oracle's classical merge sort and its 6To8 hybrid."""
    a = g.random_i32(10_000, g.config_seed(0))
    out = gpu_sort(hs, a, "merge", "6To8")
    assert np.array_equal(out, oracle.merge_sort(a, "none"))
    assert np.array_equal(out, oracle.merge_sort(a, "6To8"))


@pytest.mark.parametrize("n", [25_000, 100_000, 1_000_000])
@pytest.mark.parametrize("dist", g.DISTS)
@pytest.mark.parametrize("netset", PAPER_NETSETS)
def test_paper_sizes_merge(hs, n, dist, netset):
    a = g.keys(n, dist, g.config_seed(1, salt=n))
    assert np.array_equal(gpu_sort(hs, a, "merge", netset), oracle.merge_sort(a, netset))


def _edge_sizes(netset):
    T = 1024 * max([k for k in range(3, 9) if (oracle.NETSETS[netset] >> k) & 1] or [1])
    sizes = set(range(0, 18)) | {31, 32, 33, 1023, 1024, 1025}
    sizes |= {T - 1, T, T + 1, 2 * T - 1, 2 * T, 2 * T + 1, 3 * T + 5, 4 * T - 3}
    sizes |= {(1 << k) + d for k in (14, 15, 16, 17, 20) for d in (-1, 0, 1)}
    sizes |= {4096 * 3 + 7, 70_001}
    # around the single-CTA small-array tile: 1024 threads x (2L - 1) keys
    # (x 3 for the classical set)
    L = max([k for k in range(3, 9) if (oracle.NETSETS[netset] >> k) & 1] or [1])
    small = 1024 * (3 if L == 1 else 2 * L - 1)
    sizes |= {small - 1, small, small + 1}
    return sorted(sizes)


@pytest.mark.parametrize("netset", ALL_NETSETS)
def test_edge_sizes_all_netsets(hs, netset):
    for n in _edge_sizes(netset):
        a = g.random_i32(n, 77 + n)
        assert np.array_equal(gpu_sort(hs, a, "merge", netset), np.sort(a)), n
        assert np.array_equal(gpu_sort(hs, a, "merge", netset), oracle.merge_sort(a, netset)), n


@pytest.mark.parametrize("netset", ["6To8", "none", "Odd", "3To5"])
def test_degenerate_inputs(hs, netset):
    n = 50_003
    cases = {
        "all_equal": np.full(n, 7, np.int32),
        "all_max": np.full(n, 2**31 - 1, np.int32),
        "extremes": np.where(g.random_i32(n, 1) > 0, 2**31 - 1, -2**31).astype(np.int32),
        "reverse": np.arange(n, 0, -1, dtype=np.int32),
        "sorted": np.arange(n, dtype=np.int32),
        "three_values": (g.random_i32(n, 2) % 3).astype(np.int32),
        "max_then_min": np.concatenate([np.full(n // 2, 2**31 - 1, np.int32),
                                        np.full(n - n // 2, -2**31, np.int32)]),
    }
    for name, a in cases.items():
        assert np.array_equal(gpu_sort(hs, a, "merge", netset), oracle.merge_sort(a, netset)), name


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_pointer_scalar_path(hs, offset):
    for n in [5, 8193, 100_000, 300_001]:
        a = g.random_i32(n, offset * 1000 + n)
        assert np.array_equal(gpu_sort(hs, a, "merge", "6To8", offset=offset), np.sort(a))


def test_small_words_bruteforce(hs):
    """Every word of length <= 8 over {0,1,2}, each offset into its own key
    band and the whole set shuffled: one sort must rebuild every word's sorted
    block, with heavy duplication inside each band."""
    import itertools
    words = []
    for n in range(1, 9):
        words += [np.array(t, np.int64) for t in itertools.product(range(3), repeat=n)]
    flat = np.concatenate([(i << 2) + w for i, w in enumerate(words)]).astype(np.int64)
    flat = (flat - (1 << 20)).astype(np.int32)
    perm = np.random.default_rng(5).permutation(flat.size)
    a = flat[perm]
    for netset in ["6To8", "3To8", "none", "PowerOf2"]:
        assert np.array_equal(gpu_sort(hs, a, "merge", netset), oracle.merge_sort(a, netset))


@pytest.mark.parametrize("netset", ["6To8", "3To8", "none", "Even"])
def test_pairs_against_oracle(hs, netset):
    for n in [1, 2, 7, 8, 9, 1000, 8191, 8192, 8193, 100_000, 1_000_003]:
        k, v = g.pair_keys_16bit(n, 900 + n)
        k = (k % 97).astype(np.int32)  # heavy ties make stability visible
        ko, vo = gpu_sort_pairs(hs, k, v, netset)
        ek, ev = oracle.merge_sort_pairs(k, v, netset)
        assert np.array_equal(ko, ek), n
        assert np.array_equal(vo, ev), n


def test_pairs_unaligned(hs):
    k, v = g.pair_keys_16bit(200_001, 4)
    ko, vo = gpu_sort_pairs(hs, k, v, "6To8", offset=1)
    ek, ev = oracle.merge_sort_pairs(k, v, "6To8")
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)


def test_pairs_copy_forms_keep_results(hs):
    """The pair sort's two forms give the oracle's stable order: bulk-copied
    block-sort tiles and merge tiles (16-byte aligned keys and values,
    n % 4 == 0) and thread-staged ones (an unaligned start or n % 4 != 0),
    at sizes around the 7936-pair block-sort tile and the 3968-pair merge
    tile, with few distinct keys (long equal runs across tiles) and
    arbitrary values."""
    rng = np.random.default_rng(40)
    for n in [2, 7, 31, 3967, 3968, 3969, 7935, 7936, 7937, 7940, 15_871, 15_872, 15_873,
              3 * 7936, 61_441, 250_003, 1 << 20]:
        for kinds in ["few", "wide"]:
            if kinds == "few":
                k = rng.integers(0, 5, n).astype(np.int32)
            else:
                k = rng.integers(-(1 << 31), 1 << 31, n, dtype=np.int64).astype(np.int32)
            v = rng.integers(-(1 << 31), 1 << 31, n, dtype=np.int64).astype(np.int32)
            ek, ev = oracle.merge_sort_pairs(k, v, "6To8")
            for off in ([0, 3] if n < 300_000 else [0]):
                ko, vo = gpu_sort_pairs(hs, k, v, "6To8", offset=off)
                assert np.array_equal(ko, ek), (n, kinds, off)
                assert np.array_equal(vo, ev), (n, kinds, off)


@pytest.mark.parametrize("fanin", [4, 2])
def test_pairs_four_way_levels(hs, fanin):
    """Four-way pair levels (forced at every size) against the oracle's
    stable order: odd and even numbers of doublings, ragged last groups, few
    distinct keys (equal keys spread over all four runs of a group, where
    the run order decides), descending blocks and arbitrary values; binary
    levels on the same inputs."""
    rng = np.random.default_rng(91 + fanin)
    T = int(hs.lib().hs_pairs_tile(hs.netset_mask("6To8")))
    sizes = sorted({2 * T, 3 * T + 4, 4 * T, 5 * T + 8, 8 * T, 9 * T + 12, 16 * T + 4,
                    33 * T - 8, 64 * T + 100, (1 << 21) + 4 * 333})
    hs.hs_set_option("merge_fanin", fanin)
    try:
        for n in sizes:
            for kind in ["few", "wide", "blocks"]:
                if kind == "few":
                    k = rng.integers(0, 3, n).astype(np.int32)
                elif kind == "wide":
                    k = rng.integers(-(1 << 31), 1 << 31, n, dtype=np.int64).astype(np.int32)
                else:
                    k = ((n - np.arange(n)) // 4000).astype(np.int32)
                v = rng.integers(-(1 << 31), 1 << 31, n, dtype=np.int64).astype(np.int32)
                ek, ev = oracle.merge_sort_pairs(k, v, "6To8")
                ko, vo = gpu_sort_pairs(hs, k, v, "6To8")
                assert np.array_equal(ko, ek), (n, kind)
                assert np.array_equal(vo, ev), (n, kind)
    finally:
        hs.hs_set_option("merge_fanin", 0)


@pytest.mark.parametrize("netset", ["none", "3To5", "Odd", "3To4", "6To8", "3", "PowerOf2"])
def test_pairs_all_netsets_small_words(hs, netset):
    """Every word over {0, 1, 2} of length 1..8, concatenated (ties
    everywhere), sorted as stable pairs under every leaf size."""
    import itertools
    segs = [np.array(t, np.int32) for m in range(1, 9) for t in itertools.product(range(3), repeat=m)]
    k = np.concatenate(segs)
    v = np.arange(k.size, dtype=np.int32)[::-1].copy()
    ko, vo = gpu_sort_pairs(hs, k, v, netset)
    ek, ev = oracle.merge_sort_pairs(k, v, "6To8")
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)


def test_host_buffer_entry(hs):
    import torch
    a = g.random_i32(1_000_000, 31)
    h = torch.from_numpy(a.copy()).pin_memory()
    hs.hs_sort_i32_host(h, "merge", "6To8")
    assert np.array_equal(h.numpy(), oracle.merge_sort(a, "6To8"))


@pytest.mark.parametrize("n", [1 << 22, (1 << 22) + 12_345, 5 * (1 << 22) + 2, 3 * (1 << 23),
                               (1 << 26) + 4 * 12_345, 5 * (1 << 24) + 2])
def test_host_buffer_entry_chunked(hs, n):
    """Host sorts of 2^22 keys or more copy in by chunks and block sort each
    chunk on arrival, from 2^26 keys on also with its first merge levels
    (chunks of whole runs), then run the remaining levels: the result must
    equal the oracle's order statistics and numpy's sort (pinned and pageable
    buffers; the last two sizes take chunk-local levels, aligned and not a
    multiple of four)."""
    import torch
    a = g.random_i32(n, 40 + n)
    h = torch.from_numpy(a.copy()).pin_memory()
    hs.hs_sort_i32_host(h, "merge", "6To8")
    want = np.sort(a)
    assert np.array_equal(h.numpy(), want)
    p = torch.from_numpy(a.copy())  # pageable
    hs.hs_sort_i32_host(p, "merge", "3To5")
    assert np.array_equal(p.numpy(), want)


@pytest.mark.parametrize("fanin", [2, 4])
@pytest.mark.parametrize("netset", ["6To8", "none"])
def test_host_buffer_pipeline_options(hs, fanin, netset):
    """The chunked host-buffer sort (chunks sorted on side streams, the last
    level copied out in parts) under both fan-ins and the smallest block-sort
    tile, against the oracle."""
    import torch
    hs.hs_set_option("merge_fanin", fanin)
    try:
        for n in [1 << 22, (1 << 22) + 4 * 777, 9 * (1 << 20) + 3]:
            a = g.random_i32(n, 60 + n + fanin)
            h = torch.from_numpy(a.copy()).pin_memory()
            hs.hs_sort_i32_host(h, "merge", netset)
            assert np.array_equal(h.numpy(), oracle.merge_sort(a, netset)), n
    finally:
        hs.hs_set_option("merge_fanin", 0)


def test_bulk_copy_wait_gives_up_with_a_status(hs):
    """A bulk-copy wait that can never complete (an mbarrier armed for bytes
    no copy delivers) ends after its poll limit with HS_ERR_TIMEOUT from
    hs_device_check, not a hang; the context stays usable and the status word
    is clear afterwards."""
    hs.hs_bulk_wait_selftest(1000)
    with pytest.raises(hs.HsortError) as err:
        hs.hs_device_check()
    assert err.value.status == 5  # HS_ERR_TIMEOUT
    hs.hs_device_check()  # cleared
    a = g.random_i32(100_000, 17)
    assert np.array_equal(gpu_sort(hs, a, "merge", "6To8"), np.sort(a))


@pytest.mark.parametrize("fanin", [0, 4])
def test_workspace_reuse_and_launch_count(hs, fanin):
    """Three sorts through one workspace; the launch count follows the level
    plan: binary levels below 2^27 keys by default, four-way levels when
    forced."""
    import torch
    n = 1 << 20
    ws = torch.empty(hs.hs_sort_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    hs.hs_set_option("merge_fanin", fanin)
    before = hs.hs_launch_count()
    try:
        for seed in range(3):
            a = g.random_i32(n, seed)
            t = to_dev(a)
            hs.hs_sort_i32(t, "merge", "6To8", ws=ws)
            torch.cuda.synchronize()
            assert np.array_equal(t.cpu().numpy(), np.sort(a))
    finally:
        hs.hs_set_option("merge_fanin", 0)
    # 1 block sort, then the global levels over the block-sort tile the
    # library reports for this n: four-way levels take two doublings each
    # (partition + merge launches), after one binary level when their number
    # is odd; binary levels of this size (265 tiles, within L2) search their
    # own splits: one launch each
    tile = int(hs.lib().hs_keys_tile(hs.netset_mask("6To8"), n))
    levels = 0
    while tile << levels < n:
        levels += 1
    binary, four = (levels % 2, levels // 2) if fanin == 4 else (levels, 0)
    assert hs.hs_launch_count() - before == 3 * (1 + binary + 2 * four)


def _four_way_inputs(n, seed):
    """Key patterns that stress the four-way split: uniform, few distinct
    values (equal keys spanning all four runs of a group), sorted, reversed,
    descending blocks (later runs of a group hold smaller keys), all equal,
    and only the two extreme values."""
    a = g.random_i32(n, seed)
    blocks = max(1, n // 5000)
    desc = (np.arange(n, dtype=np.int64) // 5000)
    return {
        "uniform": a,
        "few": (a % 3).astype(np.int32),
        "sorted": np.sort(a),
        "reverse": np.sort(a)[::-1].copy(),
        "desc_blocks": ((blocks - desc) * 1000 + (a % 1000)).astype(np.int32),
        "all_equal": np.full(n, -5, np.int32),
        "extremes": np.where(a > 0, 2**31 - 1, -2**31).astype(np.int32),
    }


@pytest.mark.parametrize("netset", ["6To8", "3To5"])
def test_four_way_levels(hs, netset):
    """Four-way merge levels (two of Algorithm 1's merge levels per pass)
    against the oracle and against binary levels only: odd and even numbers
    of doublings, last groups with one to four runs, partial last runs, and
    the key patterns of _four_way_inputs."""
    mask = hs.netset_mask(netset)
    cases = []
    for base in [1 << 16, 1 << 20, 3 << 20]:
        T = int(hs.lib().hs_keys_tile(mask, base))
        cases += [2 * T, 3 * T + 4, 4 * T, 4 * T + 8, 5 * T, 7 * T - 4, 8 * T, 9 * T + 12,
                  16 * T + 4, 17 * T + 4, 33 * T - 8, 64 * T + 100]
    cases += [(1 << 22) + 4 * 12_345, 3 << 22]
    cases = sorted({c for c in cases if c % 4 == 0})
    try:
        for n in cases:
            for name, a in _four_way_inputs(n, n).items():
                want = oracle.merge_sort(a, netset)
                for fanin in (4, 2):
                    hs.hs_set_option("merge_fanin", fanin)
                    assert np.array_equal(gpu_sort(hs, a, "merge", netset), want), (n, name, fanin)
    finally:
        hs.hs_set_option("merge_fanin", 0)


def test_four_way_levels_unaligned_and_ragged(hs):
    """Unaligned starts and lengths that are not multiples of four take the
    binary generic levels; the result is the same."""
    for n in [4 * 8928 + 1, 16 * 8928 + 3, (1 << 20) + 2]:
        a = g.random_i32(n, 3 * n)
        want = oracle.merge_sort(a, "6To8")
        assert np.array_equal(gpu_sort(hs, a, "merge", "6To8"), want), n
        assert np.array_equal(gpu_sort(hs, a, "merge", "6To8", offset=1), want), n


def test_tail_not_multiple_of_four(hs):
    """Aligned buffers whose length is not a multiple of 4: the bulk-copy merge
    loads the last keys with plain loads."""
    for n in [8192 * 2 + 1, 8192 * 2 + 2, 8192 * 2 + 3, 8192 * 5 + 3, 7936 * 3 + 1, 7936 * 4 + 2,
              1_000_001, 1_000_002, (1 << 22) + 3]:
        a = g.random_i32(n, 5000 + n)
        assert np.array_equal(gpu_sort(hs, a, "merge", "6To8"), np.sort(a)), n


def test_many_duplicates_and_runs(hs):
    """Long runs of equal keys across tile and run boundaries."""
    n = 3 * (1 << 20) + 17
    for mod in [1, 2, 7, 4096]:
        a = (g.random_i32(n, mod) % mod).astype(np.int32)
        assert np.array_equal(gpu_sort(hs, a, "merge", "6To8"), np.sort(a)), mod


@pytest.mark.parametrize("shape", [-1, 2, 4])
@pytest.mark.parametrize("fanin", [2, 4])
def test_shapes_and_fanin_keep_results(hs, shape, fanin):
    """Block-sort shape (256 or 288 threads, or the per-size rule) and the
    merge fan-in change speed, not results: aligned arrays (bulk-copied
    tiles, sampled partitions), unaligned ones (thread-staged tiles, the
    generic levels) and n % 4 != 0, on uniform keys, few distinct keys and
    presorted runs, under four network sets."""
    hs.hs_set_option("blocksort_shape", shape)
    hs.hs_set_option("merge_fanin", fanin)
    try:
        for netset in ["6To8", "3To5", "none", "Odd"]:
            for n in [1, 7, 7936, 7937, 8928, 8929, 16385, 17856, 17860, 100_003, 1 << 20]:
                a = g.random_i32(n, n + 10 * (shape + 1) + fanin)
                want = oracle.merge_sort(a, netset)
                assert np.array_equal(gpu_sort(hs, a, "merge", netset), want), (netset, n)
                if n > 8000:
                    assert np.array_equal(gpu_sort(hs, a, "merge", netset, offset=1), want), (netset, n)
        for n in [9000, 65_536, 250_000]:
            for kind in ["few", "sorted"]:
                a = g.random_i32(n, n + shape)
                a = (a % 3).astype(np.int32) if kind == "few" else g.keys(n, "nearly", n + shape)
                assert np.array_equal(gpu_sort(hs, a, "merge", "6To8"), np.sort(a)), (n, kind)
    finally:
        hs.hs_set_option("blocksort_shape", -1)
        hs.hs_set_option("merge_fanin", 0)


def test_profiling_counters(hs):
    import torch
    hs.hs_prof_reset()
    hs.hs_prof_enable(True)
    hs.hs_set_option("merge_fanin", 4)  # four-way levels at this size too
    try:
        t = to_dev(g.random_i32(1 << 18, 1))
        hs.hs_sort_i32(t, "merge", "6To8")
        torch.cuda.synchronize()
        n_bs, ms_bs = hs.hs_prof_read("blocksort_keys")
        n_mk, ms_mk = hs.hs_prof_read("merge_keys")
        n_m4, ms_m4 = hs.hs_prof_read("merge4_keys")
    finally:
        hs.hs_prof_enable(False)
        hs.hs_set_option("merge_fanin", 0)
    tile = int(hs.lib().hs_keys_tile(hs.netset_mask("6To8"), 1 << 18))
    levels = 0
    while tile << levels < (1 << 18):
        levels += 1
    # binary level first when the number of doublings is odd, then four-way
    assert levels == 5
    assert n_bs == 1 and n_mk == 1 and n_m4 == 2 and min(ms_bs, ms_mk, ms_m4) > 0


def test_profiling_one_kernel(hs):
    """hs_prof_select restricts the event timing to one kernel."""
    import torch
    hs.hs_prof_reset()
    hs.hs_prof_select("merge_keys")
    hs.hs_prof_enable(True)
    try:
        t = to_dev(g.random_i32(1 << 18, 2))
        hs.hs_sort_i32(t, "merge", "6To8")
        torch.cuda.synchronize()
        n_bs, _ = hs.hs_prof_read("blocksort_keys")
        n_mk, ms_mk = hs.hs_prof_read("merge_keys")
    finally:
        hs.hs_prof_enable(False)
        hs.hs_prof_select(None)
    assert n_bs == 0 and n_mk > 0 and ms_mk > 0


def test_full_size_keys_2p28(hs):
    """2^28 uniform int32 keys, {6,7,8}: the benchmark's workload (same seed)
    and launch configuration, equal element by element to the oracle's
    Algorithm 1 on the whole array; sortedness, multiset fingerprint and
    sampled order statistics as well."""
    import torch
    n = 1 << 28
    a = g.random_i32(n, g.config_seed(2))
    t = to_dev(a)
    hs.hs_sort_i32(t, "merge", "6To8")
    hs.hs_device_check()
    out = t.cpu().numpy()
    del t
    assert np.array_equal(out, oracle.merge_sort(a, "6To8"))
    check_sorted_permutation(a, out, samples=6)


def test_above_2p31_keys(hs):
    """2^31 + 49,380 uniform keys (8 GiB, a multiple of four: the tiled
    binary and four-way levels), past every 32-bit index: sorted, multiset
    fingerprint kept, sampled order statistics from the oracle's counts."""
    import torch
    n = (1 << 31) + 49_380
    a = g.random_i32(n, g.config_seed(2, salt=31))
    t = to_dev(a)
    hs.hs_sort_i32(t, "merge", "6To8")
    hs.hs_device_check()
    out = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    check_sorted_permutation(a, out, samples=4)


def test_full_size_pairs_2p27(hs):
    """2^27 stable pairs, keys from 2^16 distinct values, value = index (the
    benchmark's pair workload): equal element by element to the oracle's
    stable Algorithm 1, and a complete stability check."""
    import torch
    n = 1 << 27
    k, v = g.pair_keys_16bit(n, g.config_seed(2, salt=1))
    tk, tv = to_dev(k), to_dev(v)
    hs.hs_sort_pairs_i32(tk, tv, "merge", "6To8")
    torch.cuda.synchronize()
    ko, vo = tk.cpu().numpy(), tv.cpu().numpy()
    del tk, tv
    ek, ev = oracle.merge_sort_pairs(k, v, "6To8")
    assert np.array_equal(ko, ek) and np.array_equal(vo, ev)
    check_stable_pairs_index_values(k, ko, vo)


def _sort_calls(hs, src, buf, ws, calls):
    """Sorts a fresh copy of src in the same buffer `calls` times; returns the
    launches each call counted."""
    import torch
    counts = []
    for _ in range(calls):
        buf.copy_(src)
        c0 = hs.hs_launch_count()
        hs.hs_sort_i32(buf, "merge", "6To8", ws=ws)
        counts.append(hs.hs_launch_count() - c0)
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy(), np.sort(src.cpu().numpy()))
    return counts


def test_repeated_sorts_replay_a_graph(hs):
    """The second call with the same arrays captures the sort into a CUDA graph
    and later calls replay it: identical results and the same kernels counted
    as the direct launches (a replay does all the work again)."""
    import torch
    n = 1 << 20
    src = to_dev(g.random_i32(n, 91))
    buf = torch.empty_like(src)
    ws = torch.empty(hs.hs_sort_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    hs.hs_set_option("sort_graphs", 0)
    try:
        direct = _sort_calls(hs, src, buf, ws, 2)
    finally:
        hs.hs_set_option("sort_graphs", 1)
    assert direct == [8, 8]  # block sort + seven binary levels that search their own splits
    assert _sort_calls(hs, src, buf, ws, 5) == [8] * 5
    # A changed option is a new configuration: older graphs are not replayed.
    hs.hs_set_option("blocksort_shape", 2)
    try:
        assert _sort_calls(hs, src, buf, ws, 4) == [9] * 4  # 7936-key tiles: eight levels
    finally:
        hs.hs_set_option("blocksort_shape", -1)
    assert _sort_calls(hs, src, buf, ws, 3) == [8] * 3
    # Another array of the same size is another signature, and still exact.
    other = to_dev(g.keys(n, "nearly", 92))
    buf2 = torch.empty_like(other)
    assert _sort_calls(hs, other, buf2, ws, 3) == [8] * 3
    hs.hs_device_check()


def test_merge_sort_inside_a_caller_graph(hs):
    """The merge path is asynchronous: a caller can capture it into its own
    CUDA graph (the library then launches directly into the capture) and
    replay it on new data."""
    import torch
    n = 300_000
    src = to_dev(g.random_i32(n, 93))
    buf = src.clone()
    ws = torch.empty(hs.hs_sort_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    hs.hs_sort_i32(buf, "merge", "6To8", ws=ws)  # warm-up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        hs.hs_sort_i32(buf, "merge", "6To8", ws=ws)
    for seed in (94, 95):
        a = g.random_i32(n, seed)
        buf.copy_(torch.from_numpy(a))
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy(), np.sort(a))
    hs.hs_device_check()


def test_repeated_pair_sorts_replay_a_graph(hs):
    """Stable pairs through the graph replay: every call on the same buffers
    (the third on replaying a captured graph) gives the oracle's stable order
    and counts the same kernels."""
    import torch
    n = 300_000
    k, v = g.pair_keys_16bit(n, 96)
    ws = torch.empty(hs.hs_sort_workspace_bytes(n, True), dtype=torch.uint8, device="cuda")
    tk, tv = to_dev(k), to_dev(v)
    want_k, want_v = oracle.merge_sort_pairs(k, v, "6To8")
    counts = []
    for _ in range(4):
        tk.copy_(torch.from_numpy(k))
        tv.copy_(torch.from_numpy(v))
        c0 = hs.hs_launch_count()
        hs.hs_sort_pairs_i32(tk, tv, "merge", "6To8", ws=ws)
        counts.append(hs.hs_launch_count() - c0)
        torch.cuda.synchronize()
        assert np.array_equal(tk.cpu().numpy(), want_k)
        assert np.array_equal(tv.cpu().numpy(), want_v)
    assert len(set(counts)) == 1 and counts[0] > 1
    hs.hs_device_check()
