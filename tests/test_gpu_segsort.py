"""GPU parity of the batched form (one persistent launch over many arrays)
against the oracle, which sorts each segment with Algorithm 1 on its own.
Sorted keys are unique, so every comparison is bit-exact."""
import itertools
import os

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


def _dev(hs, keys, off):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(keys)).cuda(),
            torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda())


def gpu_segsort(hs, keys, off, plan=None, netset="6To8"):
    tk, to = _dev(hs, keys, off)
    hs.hs_segsort_i32(tk, to, "merge", netset, plan=plan)
    hs.hs_device_check()
    return tk.cpu().numpy()


def test_every_small_word_is_a_segment(hs):
    segs = []
    for n in range(0, 9):
        segs.extend(np.array(t, np.int32) for t in itertools.product(range(3), repeat=n))
        segs.extend(np.array(p, np.int32) * 3 - 7 for p in itertools.permutations(range(n)))
    keys = np.concatenate(segs).astype(np.int32)
    off = np.zeros(len(segs) + 1, np.int64)
    np.cumsum([s.size for s in segs], out=off[1:])
    want = oracle.segsort(keys, off, "merge", "6To8")
    for netset in ["6To8", "3To5", "none", "Odd"]:
        assert np.array_equal(gpu_segsort(hs, keys, off, netset=netset), want), netset


def test_log_uniform_mix_against_oracle(hs):
    """The batched workload's law (sizes log-uniform in [3, 65536], mixed
    random / sorted / nearly sorted), 3,000 segments."""
    keys, off, _ = g.segmented(3000, g.config_seed(3, salt=1))
    want = oracle.segsort(keys, off, "merge", "6To8")
    assert np.array_equal(gpu_segsort(hs, keys, off), want)


@pytest.mark.parametrize("netset", ["6To8", "Odd", "3To5", "3To4", "none"])
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("ctas", [0, 1, 2])
def test_every_plan_gives_the_same_bytes(hs, netset, threads, ctas):
    sizes = np.array([0, 1, 2, 3, 9, 100, 1023, 1024, 1025, 7679, 7680, 7681, 7935, 7936, 7937,
                      8191, 8192, 8193, 15_360, 15_873, 16383, 16384, 16385, 40_000, 65_536, 5, 7,
                      12_345], np.int64)
    keys, off, _ = g.segmented(0, 77, sizes=sizes)
    want = oracle.segsort(keys, off, "merge", "6To8")
    plan = hs.make_plan(netset, threads, ctas)
    assert np.array_equal(gpu_segsort(hs, keys, off, plan=plan), want)


LEAF = {"6To8": 8, "Odd": 7, "3To5": 5, "3To4": 4, "none": 1}


@pytest.mark.parametrize("netset", ["6To8", "Odd", "3To5", "none"])
@pytest.mark.parametrize("threads", [256, 512])
def test_warp_tile_boundary(hs, netset, threads):
    """Segments of up to one warp tile (32 threads x EO keys, EO = 4L-1 at
    256 threads, 2L-1 at 512) are sorted by a single warp; one key more goes
    to a whole CTA.  Many such segments keep every warp of a CTA busy on a
    different one at once."""
    L = LEAF[netset]
    wt = 32 * ((4 if threads == 256 else 2) * L - 1)
    rng = np.random.default_rng(wt + threads)
    edge = [wt - 1, wt, wt + 1, 2, 3, 2 * wt, wt - 31, 33]
    sizes = np.concatenate([edge, rng.integers(0, wt + 1, 600), edge]).astype(np.int64)
    keys, off, _ = g.segmented(0, 5 + wt, sizes=sizes)
    want = oracle.segsort(keys, off, "merge", "6To8")
    plan = hs.make_plan(netset, threads, 0)
    assert np.array_equal(gpu_segsort(hs, keys, off, plan=plan), want)


def test_large_segments_and_many_merge_chunks(hs):
    # One segment long enough for more than 256 merge chunks per level
    # (several split batches), plus neighbours of odd sizes.
    sizes = np.array([3, (1 << 22) + 12_345, 17, 300_001], np.int64)
    keys, off, _ = g.segmented(0, 91, sizes=sizes)
    want = oracle.segsort(keys, off, "merge", "6To8")
    assert np.array_equal(gpu_segsort(hs, keys, off), want)


def test_unaligned_segment_starts(hs):
    sizes = np.array([1, 2, 3, 5, 8190, 16387, 33_001, 4, 70_000], np.int64)
    keys, off, _ = g.segmented(0, 12, sizes=sizes)
    for plan in [hs.make_plan("6To8", 256), hs.make_plan("6To8", 512), hs.make_plan("Odd", 256)]:
        assert np.array_equal(gpu_segsort(hs, keys, off, plan=plan),
                              oracle.segsort(keys, off, "merge", "6To8"))


def test_graph_replay(hs):
    import torch
    keys, off, _ = g.segmented(2000, 5)
    want = oracle.segsort(keys, off, "merge", "6To8")
    tk, to = _dev(hs, keys, off)
    pristine = tk.clone()
    graph = hs.hs_segsort_capture(tk, to, hs.make_plan("6To8", 256))
    for _ in range(3):
        tk.copy_(pristine)
        graph.launch()
        hs.hs_device_check()
        assert np.array_equal(tk.cpu().numpy(), want)
    graph.destroy()


def test_per_array_loop_matches(hs):
    keys, off, _ = g.segmented(300, 6)
    tk, _ = _dev(hs, keys, off)
    hs.hs_sort_i32_many(tk, off, "merge", "6To8")
    hs.hs_device_check()
    assert np.array_equal(tk.cpu().numpy(), oracle.segsort(keys, off, "merge", "6To8"))


def test_autotune_restores_keys_and_caches(hs, tmp_path):
    keys, off, _ = g.segmented(1500, 8)
    tk, to = _dev(hs, keys, off)
    plan, ms = hs.hs_segsort_autotune(tk, to)
    assert ms > 0 and plan.block_threads in (256, 512)
    assert np.array_equal(tk.cpu().numpy(), keys)  # input untouched
    again, ms2 = hs.hs_segsort_autotune(tk, to)  # cache hit: same plan, no timing
    assert again.as_dict() == plan.as_dict() and ms2 == ms
    path = os.path.join(tmp_path, "tune.json")
    hs.hs_tune_cache_save(path)
    hs.hs_tune_cache_load(path)
    text = open(path).read()
    assert '"block_threads"' in text and '"netset"' in text
    assert np.array_equal(gpu_segsort(hs, keys, off, plan=plan),
                          oracle.segsort(keys, off, "merge", "6To8"))
    # With no plan given, a call with the tuned plan's network set takes it;
    # another set keeps the default shape.
    nseg = len(off) - 1
    netsets = {v: k for k, v in hs.NETSETS.items()}
    assert hs.hs_segsort_plan_for(keys.size, nseg, int(plan.netset)).as_dict() == plan.as_dict()
    other = 0xA8 if int(plan.netset) != 0xA8 else 0x1C0
    assert hs.hs_segsort_plan_for(keys.size, nseg, other).as_dict() == \
        {"netset": other, "block_threads": 256, "ctas_per_sm": 0}
    assert np.array_equal(gpu_segsort(hs, keys, off, netset=netsets.get(int(plan.netset), "6To8")),
                          oracle.segsort(keys, off, "merge", "6To8"))
    hs.hs_tune_cache_clear()


def test_malformed_offsets_are_reported(hs):
    import torch
    keys = g.random_i32(1000, 1)
    off = np.array([0, 500, 400, 1000], np.int64)  # second segment has negative length
    tk, to = _dev(hs, keys, off)
    hs.hs_segsort_i32(tk, to)
    with pytest.raises(hs.HsortError) as err:
        hs.hs_device_check()
    assert err.value.status == 1
    hs.hs_device_check()  # cleared


def test_quick_is_unsupported_in_batched_form(hs):
    keys, off, _ = g.segmented(10, 1)
    tk, to = _dev(hs, keys, off)
    with pytest.raises(hs.HsortError) as err:
        hs.hs_segsort_i32(tk, to, "quick")
    assert err.value.status == 2


def test_prefix_of_the_batched_workload(hs):
    """The seeded prefix of the 200,000-segment size sequence that reaches
    2^28 keys: every segment sorted, multiset kept, sampled segments equal
    to the oracle's."""
    import torch
    sizes = g.segment_sizes(200_000, g.config_seed(3))
    k = int(np.searchsorted(np.cumsum(sizes), 1 << 28)) + 1
    keys, off, _ = g.segmented(0, g.config_seed(3), sizes=sizes[:k])
    tk, to = _dev(hs, keys, off)
    hs.hs_segsort_i32(tk, to)
    hs.hs_device_check()
    out = tk.cpu().numpy()
    del tk, to
    d = np.diff(out.astype(np.int64))
    starts = off[1:-1] - 1  # positions where a new segment begins
    d[starts[starts >= 0]] = 0
    assert np.all(d >= 0)
    rng = np.random.default_rng(3)
    for s in rng.integers(0, k, 40).tolist():
        b, e = int(off[s]), int(off[s + 1])
        assert np.array_equal(out[b:e], oracle.merge_sort(keys[b:e], "6To8"))
    from helpers import fingerprint
    assert fingerprint(out) == fingerprint(keys)


def test_full_batched_workload_against_oracle(hs):
    """The whole batched workload of the benchmark: 200,000 segments, sizes
    log-uniform in [3, 65,536] (about 1.31 G keys), mixed distributions, in
    one persistent launch with the default plan: equal element by element
    to the oracle sorting every segment (host threads over disjoint ranges
    of whole segments)."""
    import os
    import torch
    keys, off, _ = g.segmented(200_000, g.config_seed(3))
    tk, to = _dev(hs, keys, off)
    hs.hs_segsort_i32(tk, to)
    hs.hs_device_check()
    out = tk.cpu().numpy()
    del tk, to
    torch.cuda.empty_cache()
    want = oracle.segsort(keys, off, "merge", "6To8", threads=min(16, os.cpu_count() or 1))
    assert np.array_equal(out, want)


@pytest.mark.parametrize("shift", [0, 1, 3])
def test_bulk_staging_at_any_alignment(hs, shift):
    """Large segments staged by bulk copies of their 16-byte aligned
    interiors (three keys at most at each end by the threads) give the
    oracle's result, with the key buffer 16-byte aligned or shifted by one or
    three keys against the workspace (then a tile's output leaves by plain
    stores)."""
    import torch
    sizes = np.array([993, 994, 995, 996, 7935, 7936, 7937, 7938, 8931, 15_875, 16_387, 40_003,
                      65_536, 3, 1, 2, 4, 5, 6, 7, 70_001, 12_345], np.int64)
    keys, off, _ = g.segmented(0, 31 + shift, sizes=sizes)
    want = oracle.segsort(keys, off, "merge", "6To8")
    for plan in [hs.make_plan("6To8", 256), hs.make_plan("Odd", 512), hs.make_plan("3To5", 256)]:
        buf = torch.empty(keys.size + shift, dtype=torch.int32, device="cuda")
        tk = buf[shift:]
        tk.copy_(torch.from_numpy(keys))
        to = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()
        hs.hs_segsort_i32(tk, to, "merge", "6To8", plan=plan)
        hs.hs_device_check()
        assert np.array_equal(tk.cpu().numpy(), want), plan
