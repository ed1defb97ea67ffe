"""GPU checks of the single-array merge path's autotuner (hs_sort_autotune).

Every plan sorts to the same unique output (a sort of int32 keys), so the bar
is bit-exact equality with numpy's sort of the same seeded input.  The tuner
must give the caller's keys back unchanged, cache its winner for the array
size's log2 bucket and leaf size, and a cached plan (tuned or loaded from the
cache file) must steer the launches of later sorts in that bucket."""
import json

import numpy as np
import pytest

import hs_inputs as g
from helpers import hs_module, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return hs_module()


@pytest.fixture(autouse=True)
def empty_cache(hs):
    """Each test starts from the built-in rules and leaves no plan behind."""
    hs.hs_tune_cache_clear()
    yield
    hs.hs_tune_cache_clear()


def plan_of(p):
    return int(p.blocksort_threads), int(p.merge_fanin)


def test_autotune_restores_keys_and_caches_the_winner(hs):
    import torch
    n = (1 << 22) + 4000  # bucket 22, n % 4 == 0: all four candidates apply
    a = g.random_i32(n, 31)
    t = to_dev(a)
    c0 = hs.hs_launch_count()
    plan, ms = hs.hs_sort_autotune(t)
    torch.cuda.synchronize()
    assert hs.hs_launch_count() > c0
    assert np.array_equal(t.cpu().numpy(), a)  # input order restored
    assert plan_of(plan) in {(256, 2), (256, 4), (288, 2), (288, 4)}
    assert ms > 0
    # A second call hits the cache: same answer, nothing launched.
    c1 = hs.hs_launch_count()
    plan2, ms2 = hs.hs_sort_autotune(t)
    assert hs.hs_launch_count() == c1
    assert plan_of(plan2) == plan_of(plan) and ms2 == ms
    # The merge path takes the winner for the whole bucket and leaf size ...
    for m in (1 << 22, (1 << 23) - 4):
        assert plan_of(hs.hs_sort_plan_for(m)) == plan_of(plan)
    # ... but not where four-way levels do not apply, nor for another leaf size.
    assert hs.hs_sort_plan_for((1 << 22) + 1).merge_fanin == 2
    assert hs.hs_sort_plan_for(1 << 22, "3To5").merge_fanin == 2
    hs.hs_sort_i32(t)
    hs.hs_device_check()
    assert np.array_equal(t.cpu().numpy(), np.sort(a))


def test_autotune_unaligned_keys_time_binary_levels_only(hs):
    import torch
    n = (1 << 20) + 12
    a = g.keys(n, "nearly", 5)
    t = to_dev(a, offset=1)  # 4-byte but not 16-byte aligned
    plan, ms = hs.hs_sort_autotune(t, "3To8")
    torch.cuda.synchronize()
    assert plan.merge_fanin == 2 and ms > 0
    assert np.array_equal(t.cpu().numpy(), a)
    hs.hs_sort_i32(t, "merge", "3To8")
    assert np.array_equal(t.cpu().numpy(), np.sort(a))


@pytest.mark.parametrize("n", [2, 1000, 8928, 20000])
def test_autotune_small_arrays(hs, n):
    """Arrays of one tile or a few: the candidates differ little, the keys still
    come back unchanged and the winner sorts correctly."""
    import torch
    a = g.random_i32(n, n)
    t = to_dev(a)
    plan, ms = hs.hs_sort_autotune(t)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), a)
    hs.hs_sort_i32(t)
    assert np.array_equal(t.cpu().numpy(), np.sort(a))


def test_loaded_plan_steers_the_launches(hs, tmp_path):
    """A plan loaded from the cache file replaces the rules for its bucket:
    2^18 keys take 256-thread block-sort tiles (7936 keys, six doublings to
    2^18) and four-way levels (three of them), where the rules take 288-thread
    tiles (five doublings) and binary levels."""
    import torch
    n = 1 << 18
    assert plan_of(hs.hs_sort_plan_for(n)) == (288, 2)  # the rules
    path = tmp_path / "plans.json"
    path.write_text(json.dumps([{
        "kind": "sort", "device": torch.cuda.get_device_name(), "n_bucket": 18, "leaf": 8,
        "blocksort_threads": 256, "merge_fanin": 4, "ms": 1.0}]))
    hs.hs_tune_cache_load(str(path))
    assert plan_of(hs.hs_sort_plan_for(n)) == (256, 4)
    assert plan_of(hs.hs_sort_plan_for(n, "3To5")) != (256, 4)  # another leaf size
    a = g.random_i32(n, 77)
    t = to_dev(a)
    hs.hs_prof_reset()
    hs.hs_prof_enable(True)
    try:
        hs.hs_sort_i32(t)
        torch.cuda.synchronize()
        n_bs, _ = hs.hs_prof_read("blocksort_keys")
        n_mk, _ = hs.hs_prof_read("merge_keys")
        n_m4, _ = hs.hs_prof_read("merge4_keys")
    finally:
        hs.hs_prof_enable(False)
    assert (n_bs, n_mk, n_m4) == (1, 0, 3)
    assert int(hs.lib().hs_keys_tile(hs.netset_mask("6To8"), n)) == 7936
    assert np.array_equal(t.cpu().numpy(), np.sort(a))
    # An option set to a non-automatic value still wins over the cached plan.
    hs.hs_set_option("merge_fanin", 2)
    try:
        assert plan_of(hs.hs_sort_plan_for(n)) == (256, 2)
    finally:
        hs.hs_set_option("merge_fanin", 0)
    # Saved and reloaded, the entry is the same.
    out = tmp_path / "saved.json"
    hs.hs_tune_cache_save(str(out))
    hs.hs_tune_cache_clear()
    assert plan_of(hs.hs_sort_plan_for(n)) == (288, 2)
    hs.hs_tune_cache_load(str(out))
    assert plan_of(hs.hs_sort_plan_for(n)) == (256, 4)
