"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

* Networks: the 0-1 principle (Knuth, TAOCP vol. 3, Theorem 5.3.4Z) over all
  2^m 0/1 inputs, every permutation of m <= 8 distinct keys, and the
  comparator counts of size-optimal networks.
* Merge, MedianOfThree, HoarePartition: brute force over all small arrays on a
  three-letter alphabet, checked against the properties that define them.
* Algorithms 1 and 2: equality with numpy's sort (a library routine) and
  numpy's stable argsort for pairs.
* Algorithm 1's recursion: the leaf-size histogram from the closed form of
  halving splits (depth-k subarrays have floor(n/2^k) or ceil(n/2^k) keys),
  and binary-tree invariants (Merge calls = leaves - 1).
"""
import itertools
import os

import numpy as np
import pytest

import hs_inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALL_NETSETS = list(oracle.NETSETS)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# ---------------------------------------------------------------- networks

def test_table3_netsets_match_paper():
    names = set()
    for row in _read_golden("table3_netsets.txt"):
        name, sizes = row.split(":")
        words = sizes.split()
        if words[0] == "var":  # VarSortk: dynamic network for any size up to k
            mask = 0x10000 | (1 << int(words[1]))
        else:
            mask = sum(1 << int(w) for w in words)
        assert oracle.NETSETS[name] == mask, name
        names.add(name)
    assert names | {"none"} == set(oracle.NETSETS)  # the 11 configurations + classical


@pytest.mark.parametrize("m", range(3, 9))
def test_network_comparator_count(m):
    want = {int(a): int(b) for a, b in (r.split() for r in _read_golden("network_sizes.txt"))}
    net = oracle.network(m)
    assert len(net) == want[m]
    assert all(0 <= i < j < m for i, j in net)


@pytest.mark.parametrize("m", range(2, 9))
def test_network_zero_one_principle(m):
    for bits in range(1 << m):
        a = np.array([(bits >> k) & 1 for k in range(m)], np.int32)
        out = oracle.apply_network(m, a)
        assert np.all(np.diff(out) >= 0), (m, a, out)
        assert out.sum() == a.sum()


@pytest.mark.parametrize("m", range(3, 9))
def test_network_all_permutations(m):
    perms = np.array(list(itertools.permutations(range(m))), np.int32)
    # Apply through Algorithm 1 with S = {m}: a segment of size m goes straight
    # to the network (the "size matches" branch).
    off = np.arange(0, perms.size + 1, m, dtype=np.int64)
    out = oracle.segsort(perms.ravel() * 7 - 3, off, "merge", 1 << m).reshape(-1, m)
    assert np.array_equal(out, np.broadcast_to(np.arange(m) * 7 - 3, out.shape))
    # And a direct call on a few with negative / extreme keys.
    ext = np.array([2**31 - 1, -2**31, 0, -1, 1, 2**31 - 2, -2**31 + 1, 5][:m], np.int32)
    for p in list(itertools.permutations(range(m)))[:50]:
        assert np.array_equal(oracle.apply_network(m, ext[list(p)]), np.sort(ext))


# ------------------------------------------------------- merge / partition

def _words(n, alphabet=3):
    for t in itertools.product(range(alphabet), repeat=n):
        yield np.array(t, np.int32)


def test_merge_bruteforce():
    for total in range(2, 9):
        for w in _words(total):
            for split in range(1, total):
                a = np.concatenate([np.sort(w[:split]), np.sort(w[split:])])
                padded = np.concatenate([[9], a, [9]]).astype(np.int32)
                out = oracle.merge(padded, 1, split, total)
                assert out[0] == 9 and out[-1] == 9
                assert np.array_equal(out[1:-1], np.sort(w))


def test_median_of_three_bruteforce():
    for n in range(1, 8):
        for w in _words(n):
            for low in range(n):
                for high in range(low, n):
                    out, mid = oracle.median_of_three(w, low, high)
                    assert mid == low + (high - low) // 2
                    assert out[low] <= out[mid] <= out[high]
                    idx = sorted({low, mid, high})
                    assert sorted(out[idx].tolist()) == sorted(w[idx].tolist())
                    rest = [i for i in range(n) if i not in idx]
                    assert np.array_equal(out[rest], w[rest])


def test_hoare_partition_bruteforce():
    for n in range(2, 9):
        for w in _words(n):
            for pivot_index in range(n - 1):  # any pivot position except the last
                out, j = oracle.hoare_partition(w, 0, n - 1, pivot_index)
                pivot = w[pivot_index]
                assert 0 <= j < n - 1
                assert out[: j + 1].max() <= pivot <= out[j + 1:].min()
                assert np.array_equal(np.sort(out), np.sort(w))


# -------------------------------------------------------- full sort outputs

EDGE_SIZES = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 15, 16, 17, 31, 32, 33, 63, 64, 65,
              100, 127, 128, 129, 1000, 1023, 1024, 1025, 4095, 4096, 4097, 10000]


@pytest.mark.parametrize("netset", ALL_NETSETS)
@pytest.mark.parametrize("algo", ["merge", "quick"])
def test_sort_matches_library_sort(netset, algo):
    fn = oracle.merge_sort if algo == "merge" else oracle.quick_sort
    for n in EDGE_SIZES:
        for dist in hs_inputs.DISTS:
            a = hs_inputs.keys(n, dist, 1000 + n)
            assert np.array_equal(fn(a, netset), np.sort(a)), (n, dist)
    special = [
        np.full(777, 42, np.int32),
        np.arange(1000, 0, -1, dtype=np.int32),
        np.array([2**31 - 1, -2**31] * 300 + [0], np.int32),
        hs_inputs.random_i32(5000, 7) % 3,
    ]
    for a in special:
        a = a.astype(np.int32)
        assert np.array_equal(fn(a, netset), np.sort(a))


@pytest.mark.parametrize("algo", ["merge", "quick"])
def test_all_small_arrays_bruteforce(algo):
    """Every array of length <= 8 over {0,1,2} and every permutation of
    length <= 8, for every Table 3 configuration."""
    segs = []
    for n in range(0, 9):
        segs.extend(_words(n))
        segs.extend(np.array(p, np.int32) for p in itertools.permutations(range(n)))
    flat = np.concatenate(segs).astype(np.int32)
    off = np.zeros(len(segs) + 1, np.int64)
    np.cumsum([s.size for s in segs], out=off[1:])
    want = np.concatenate([np.sort(s) for s in segs]).astype(np.int32)
    for netset in ALL_NETSETS:
        assert np.array_equal(oracle.segsort(flat, off, algo, netset), want), netset


@pytest.mark.parametrize("netset", ALL_NETSETS)
def test_pairs_match_stable_argsort(netset):
    for n in [0, 1, 5, 8, 9, 100, 1000, 4097]:
        k, v = hs_inputs.pair_keys_16bit(n, 55 + n)
        k = (k % 7).astype(np.int32)  # many ties
        ko, vo = oracle.merge_sort_pairs(k, v, netset)
        perm = np.argsort(k, kind="stable")
        assert np.array_equal(ko, k[perm])
        assert np.array_equal(vo, v[perm])


def test_pairs_all_small_words():
    for netset in ["6To8", "3To8", "none", "Odd"]:
        for n in range(0, 9):
            for w in _words(n, 2):
                ko, vo = oracle.merge_sort_pairs(w, np.arange(n, dtype=np.int32), netset)
                perm = np.argsort(w, kind="stable")
                assert np.array_equal(vo, perm.astype(np.int32)), (netset, w)


# ---------------------------------------------------- recursion structure

def closed_form_leaves(n, netset_mask):
    """Leaf histogram of Algorithm 1 from the closed form of halving splits.

    At depth k the subarrays that exist have floor(n/2^k) or ceil(n/2^k) keys,
    and exactly n mod 2^k of the 2^k depth-k positions have the ceiling size.
    A node splits when its size is >= 2 and not in the set; its children have
    ceil(s/2) and floor(s/2) keys.  Walk the depths tracking how many live
    nodes have each of the two sizes."""
    live = {n: 1}
    nets = {}    # network size -> applications
    leaf_keys = 0
    ones = 0
    merges = 0
    depth = 0
    var_k = 0
    if netset_mask & 0x10000:  # VarSortk: leaves are the sizes 2..k, all by the size-k network
        var_k = (netset_mask & ~0x10000).bit_length() - 1
    while live:
        q = n >> depth
        assert set(live) <= {q, q + 1}, (depth, live)  # closed form holds
        nxt = {}
        for s, cnt in live.items():
            leaf_net = (var_k if 2 <= s <= var_k else 0) if var_k else \
                (s if 3 <= s <= 8 and (netset_mask >> s) & 1 else 0)
            if leaf_net:
                nets[leaf_net] = nets.get(leaf_net, 0) + cnt
                leaf_keys += s * cnt
            elif s == 1:
                ones += cnt
            elif s >= 2:
                merges += cnt
                for c in ((s + 1) // 2, s // 2):
                    nxt[c] = nxt.get(c, 0) + cnt
        live = nxt
        depth += 1
    return nets, merges, ones, leaf_keys


@pytest.mark.parametrize("n", [10_000, 25_000, 100_000, 1_000_000, 12345, 1 << 16])
@pytest.mark.parametrize("netset", ["3To5", "6To8", "3To8", "none", "PowerOf2", "Odd",
                                    "VarSort3", "VarSort4", "VarSort5"])
def test_leaf_histogram_closed_form(n, netset):
    a = hs_inputs.random_i32(n, 3)
    out, c = oracle.merge_sort(a, netset, counters=True)
    nets, merges, ones, leaf_keys = closed_form_leaves(n, oracle.NETSETS[netset])
    assert c["net_calls"] == nets
    assert c["merge_calls"] == merges
    leaves = sum(nets.values()) + ones
    assert c["merge_calls"] == leaves - 1           # binary tree
    assert leaf_keys + ones == n
    assert np.array_equal(out, np.sort(a))


def test_varsort_leaves_cover_sizes_two_to_k():
    # n = 10,000 halves down to 4/5 keys: VarSort4 sorts the 4s and splits the
    # 5s into 3 + 2 (both <= 4), VarSort5 stops at the 4/5 level, VarSort3
    # goes one level below; every leaf uses the size-k network.
    for k, name in [(3, "VarSort3"), (4, "VarSort4"), (5, "VarSort5")]:
        _, c = oracle.merge_sort(hs_inputs.random_i32(10_000, 2), name, counters=True)
        assert set(c["net_calls"]) == {k}, name


def test_ten_thousand_has_no_six_to_eight_leaf():
    # Depth-k sizes at n=10,000 run 10000, 5000, ..., 19/20, 9/10, 4/5: never
    # 6, 7 or 8, so 6To8 does exactly the classical Merge calls there.
    _, c = oracle.merge_sort(hs_inputs.random_i32(10_000, 1), "6To8", counters=True)
    assert c["net_calls"] == {} and c["merge_calls"] == 9_999


def test_power_of_two_closed_form():
    n = 1 << 20
    a = hs_inputs.random_i32(n, 9)
    _, c = oracle.merge_sort(a, "6To8", counters=True)
    assert c["net_calls"] == {8: n // 8} and c["merge_calls"] == n // 8 - 1
    _, c = oracle.merge_sort(a, "3To5", counters=True)
    assert c["net_calls"] == {4: n // 4} and c["merge_calls"] == n // 4 - 1
    _, c = oracle.merge_sort(a, "none", counters=True)
    assert c["net_calls"] == {} and c["merge_calls"] == n - 1
    assert c["max_depth"] == 20


def test_quick_sort_structure():
    # Every partition call splits a subarray in two non-empty parts, so with
    # no networks a run of n distinct keys takes exactly n - 1 partitions.
    a = np.random.default_rng(0).permutation(5000).astype(np.int32)
    _, c = oracle.quick_sort(a, "none", counters=True)
    assert c["partition_calls"] == 4999
    # Sorted input: the median of three is the exact median, depth ~ log2 n.
    _, c = oracle.quick_sort(np.arange(1 << 14, dtype=np.int32), "none", counters=True)
    assert c["max_depth"] <= 15


def test_checks():
    a = np.array([3, 1, 2, 2], np.int32)
    assert not oracle.is_sorted(a) and oracle.is_sorted(np.sort(a))
    assert oracle.count_less(a, 2) == 1 and oracle.count_less_equal(a, 2) == 3


# ---------------------------------------------------------------- int64 keys

@pytest.mark.parametrize("netset", ["none", "6To8", "3To5", "VarSort4"])
def test_int64_merge_sort(netset):
    """Algorithm 1 on int64 keys: numpy's sort on every edge size and
    distribution, the extremes of the type, and the same recursion (leaf and
    Merge counts) as the int32 form for the same n."""
    for n in EDGE_SIZES:
        for dist in hs_inputs.DISTS:
            a = hs_inputs.keys_i64(n, dist, 2000 + n)
            assert np.array_equal(oracle.merge_sort_i64(a, netset), np.sort(a)), (n, dist)
    ext = np.array([2**63 - 1, -2**63, 0, -1, 1] * 41, np.int64)
    assert np.array_equal(oracle.merge_sort_i64(ext, netset), np.sort(ext))
    for n in [10_000, 12_345]:
        _, c64 = oracle.merge_sort_i64(hs_inputs.keys_i64(n, "random", 1), netset, counters=True)
        _, c32 = oracle.merge_sort(hs_inputs.random_i32(n, 1), netset, counters=True)
        assert c64["net_calls"] == c32["net_calls"] and c64["merge_calls"] == c32["merge_calls"]


def test_segsort_threads_give_the_same_result(oracle_lib):
    """The threaded driver of the oracle's segmented sort hands disjoint
    ranges of whole segments to host threads: the result equals the
    single-threaded call and numpy's per-segment sort."""
    import hs_inputs as g
    keys, off, _ = g.segmented(3000, 11)
    one = oracle_lib.segsort(keys, off, "merge", "6To8")
    many = oracle_lib.segsort(keys, off, "merge", "6To8", threads=7)
    assert np.array_equal(one, many)
    for s in (0, 1, 1499, 2999):
        assert np.array_equal(many[off[s]:off[s + 1]], np.sort(keys[off[s]:off[s + 1]]))
