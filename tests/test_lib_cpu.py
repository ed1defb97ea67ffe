"""The C-ABI library on a machine without a GPU: it loads, exports every
declared symbol, its device networks (host build) sort exhaustively, and its
argument checks fail synchronously before any CUDA call."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hs():
    from paper_2503_05934_gb300 import build
    build.build()
    from paper_2503_05934_gb300 import _lib
    return _lib.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(hs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(hs):
    names = declared_functions()
    assert "hs_sort_i32" in names and "hs_sort_pairs_i32" in names
    for name in names:
        assert hasattr(hs, name), name


def test_binding_covers_header():
    from paper_2503_05934_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_version_and_status_strings(hs):
    assert b"sm_103a" in hs.hs_version()
    for code, name in [(0, b"HS_OK"), (1, b"HS_ERR_INVALID_ARG"), (2, b"HS_ERR_UNSUPPORTED"),
                       (5, b"HS_ERR_TIMEOUT"), (6, b"HS_ERR_OVER_BUDGET")]:
        assert hs.hs_status_str(code) == name


@pytest.mark.parametrize("m", range(2, 9))
def test_device_networks_host_build(hs, m):
    want = {2: 1, 3: 3, 4: 5, 5: 9, 6: 12, 7: 16, 8: 19}
    buf = (ctypes.c_int * 64)()
    assert hs.hs_network_pairs(m, buf, 32) == want[m]
    pairs = [(buf[2 * i], buf[2 * i + 1]) for i in range(want[m])]
    assert all(0 <= i < j < m for i, j in pairs)
    # 0-1 principle
    for bits in range(1 << m):
        a = np.array([(bits >> k) & 1 for k in range(m)], np.int32)
        hs.hs_network_apply(m, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        assert np.all(np.diff(a) >= 0)
    # every permutation of distinct keys, including the int32 extremes
    ext = np.array([2**31 - 1, -2**31, 0, -1, 1, 2**31 - 2, -2**31 + 1, 5][:m], np.int32)
    for p in itertools.permutations(range(m)):
        a = ext[list(p)].copy()
        hs.hs_network_apply(m, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        assert np.array_equal(a, np.sort(ext))


def test_device_networks_differ_from_oracle_construction(hs):
    # Independent constructions: the library uses Bose-Nelson, the oracle
    # pruned Batcher; they agree on sizes but not on every comparator list.
    import oracle
    buf = (ctypes.c_int * 64)()
    differ = 0
    for m in range(3, 9):
        cnt = hs.hs_network_pairs(m, buf, 32)
        lib_pairs = [(buf[2 * i], buf[2 * i + 1]) for i in range(cnt)]
        assert len(lib_pairs) == len(oracle.network(m))
        differ += lib_pairs != oracle.network(m)
    assert differ >= 3


FAKE = 0x100000  # never dereferenced: every case below fails validation first


def test_argument_errors_are_synchronous(hs):
    ws_big = 1 << 40
    # unknown netset bits
    assert hs.hs_sort_i32(FAKE, 100, 0, 0x1, FAKE, ws_big, None) == 1
    assert hs.hs_sort_i32(FAKE, 100, 0, 0x200, FAKE, ws_big, None) == 1
    # unknown algo
    assert hs.hs_sort_i32(FAKE, 100, 7, 0x1C0, FAKE, ws_big, None) == 1
    # NULL keys with n > 0; unaligned keys
    assert hs.hs_sort_i32(None, 100, 0, 0x1C0, FAKE, ws_big, None) == 1
    assert hs.hs_sort_i32(FAKE + 2, 100, 0, 0x1C0, FAKE, ws_big, None) == 1
    assert b"aligned" in hs.hs_last_error()
    # workspace too small for a multi-tile merge sort
    assert hs.hs_sort_i32(FAKE, 1 << 20, 0, 0x1C0, FAKE, 16, None) == 1
    assert b"workspace" in hs.hs_last_error()
    # pairs: quick is unstable -> unsupported; NULL values -> invalid
    assert hs.hs_sort_pairs_i32(FAKE, FAKE, 100, 1, 0x1C0, FAKE, ws_big, None) == 2
    assert hs.hs_sort_pairs_i32(FAKE, None, 100, 0, 0x1C0, FAKE, ws_big, None) == 1
    # n = 0 and n = 1 are no-ops, even without workspace
    assert hs.hs_sort_i32(None, 0, 0, 0x1C0, None, 0, None) == 0
    assert hs.hs_sort_i32(FAKE, 1, 0, 0x1C0, None, 0, None) == 0
    assert hs.hs_last_error() == b""


def test_workspace_sizes(hs):
    for n in [0, 1, 1000, 1 << 20, 1 << 28]:
        ws = hs.hs_sort_workspace_bytes(n, 0, 0)
        assert ws >= 4 * n
        assert hs.hs_sort_workspace_bytes(n, 1, 0) >= 8 * n
        assert hs.hs_sort_host_workspace_bytes(n, 0) >= ws + 4 * n


def test_prof_select_names(hs):
    assert hs.hs_prof_select(b"merge_keys") == 0
    assert hs.hs_prof_select(None) == 0
    assert hs.hs_prof_select(b"no_such_kernel") == 1
    assert b"unknown kernel" in hs.hs_last_error()


def test_bulk_wait_selftest_rejects_bad_poll_limits(hs):
    """Argument errors return before any launch, so they need no GPU."""
    assert hs.hs_bulk_wait_selftest(0, None) == 1
    assert hs.hs_bulk_wait_selftest((1 << 22) + 1, None) == 1


# Every tuning option with its default, a valid alternative and invalid values
# (hs_set_option validates on the host, so no GPU is needed).
OPTIONS = [
    ("blocksort_shape", -1, 4, [-2, 0, 1, 3, 5, 6]),
    ("merge_fanin", 0, 4, [1, 3, 8, -1]),
    ("quick_partition", 3, 2, [1, 4]),
    ("sort_graphs", 1, 0, [2, -1]),
]


@pytest.mark.parametrize("name,default,other,bad", OPTIONS)
def test_option_values_are_validated(hs, name, default, other, bad):
    try:
        assert hs.hs_set_option(name.encode(), other) == 0
        for v in bad:
            assert hs.hs_set_option(name.encode(), v) == 1, (name, v)
    finally:
        assert hs.hs_set_option(name.encode(), default) == 0


def test_unknown_option_is_rejected(hs):
    assert hs.hs_set_option(b"no_such_option", 1) == 1
    for removed in (b"merge_tile", b"merge_kernel", b"merge_samples", b"blocksort_bulk",
                    b"blocksort_threads", b"pairs_blocksort", b"pairs_merge",
                    b"pairs_blocksort_bulk", b"i64_merge", b"segsort_bulk"):
        assert hs.hs_set_option(removed, 1) == 1, removed


def _brute_split(keys, starts, lens, rank):
    """Counts per run among the first `rank` outputs of the stable merge:
    order by (key, run), positions ascending within a run (lexsort)."""
    run_of, vals = [], []
    for i, (s, ln) in enumerate(zip(starts, lens)):
        vals.append(keys[s:s + ln])
        run_of.append(np.full(ln, i, np.int64))
    v = np.concatenate(vals) if vals else np.zeros(0, np.int32)
    r = np.concatenate(run_of) if run_of else np.zeros(0, np.int64)
    order = np.lexsort((np.arange(v.size), r, v.astype(np.int64)))
    return np.bincount(r[order[:rank]], minlength=len(lens))


@pytest.mark.parametrize("k_runs", [2, 4, 8])
def test_merge_split_host_against_brute_force(k_runs):
    """The four-way levels' K-way split (host build) equals the counts of a
    brute-force stable merge at every rank, on runs with heavy duplicates,
    all-equal keys, disjoint ranges, empty and ragged runs, with and without
    the sample array."""
    import paper_2503_05934_gb300 as hs
    rng = np.random.default_rng(7 + k_runs)
    for trial in range(60):
        kind = trial % 4
        lens = [int(x) for x in rng.integers(0, 200, k_runs)]
        if trial % 5 == 0:
            lens[int(rng.integers(0, k_runs))] = 0
        runs = []
        for i, ln in enumerate(lens):
            if kind == 0:
                x = rng.integers(-4, 4, ln)
            elif kind == 1:
                x = rng.integers(-2**31, 2**31, ln)
            elif kind == 2:
                x = np.arange(ln) + 1000 * (k_runs - i)  # later runs hold smaller keys
            else:
                x = np.full(ln, 2**31 - 1)
            runs.append(np.sort(x).astype(np.int32))
        # runs at 32-aligned starts with gaps, so the sample array applies
        starts, keys = [], np.zeros(0, np.int32)
        for r in runs:
            pad = (-keys.size) % 32 + 32 * int(rng.integers(0, 2))
            keys = np.concatenate([keys, rng.integers(-9, 9, pad).astype(np.int32)])
            starts.append(keys.size)
            keys = np.concatenate([keys, r])
        samp = keys[::32].copy()
        total = sum(lens)
        for rank in sorted(set([0, total] + [int(x) for x in rng.integers(0, total + 1, 25)])):
            want = _brute_split(keys, starts, lens, rank)
            assert np.array_equal(hs.hs_merge_split(keys, starts, lens, rank), want)
            assert np.array_equal(hs.hs_merge_split(keys, starts, lens, rank, samp), want)


def test_merge_split_host_rejects_bad_arguments():
    import paper_2503_05934_gb300 as hs
    keys = np.arange(64, dtype=np.int32)
    with pytest.raises(ValueError):
        hs.hs_merge_split(keys, [0, 32, 40], [8, 8, 8], 3)  # 3 runs
    with pytest.raises(ValueError):
        hs.hs_merge_split(keys, [0, 32], [8, 8], 17)  # rank past the total
    with pytest.raises(ValueError):
        hs.hs_merge_split(keys, [0, 33], [8, 8], 3, keys[::32])  # unaligned start with samples


def _plan_for(hs, n, netset=0x1C0, keys=None):
    from paper_2503_05934_gb300 import _lib
    p = _lib.SortPlan()
    assert hs.hs_sort_plan_for(keys, n, netset, ctypes.byref(p)) == 0
    return int(p.blocksort_threads), int(p.merge_fanin)


def test_sort_plan_rules_and_options(hs):
    """The single-array plan from the built-in rules (no cached plan can match
    without a device), and the options' precedence over them."""
    # The 288-thread tile (8928 keys for {6,7,8}) saves a global level for
    # every power of two from 2^14; 2^13 fits either tile.
    assert _plan_for(hs, 1 << 20) == (288, 2)
    assert _plan_for(hs, 9000) == (256, 2)       # 9000 <= 2 * 7936: one level either way
    assert _plan_for(hs, 1 << 27) == (288, 4)    # four-way levels from 2^27 keys
    assert _plan_for(hs, (1 << 27) + 2) == (288, 2)          # n % 4 != 0: binary levels
    assert _plan_for(hs, 1 << 27, keys=FAKE + 4) == (288, 2)  # keys not 16-byte aligned
    try:
        assert hs.hs_set_option(b"blocksort_shape", 2) == 0
        assert hs.hs_set_option(b"merge_fanin", 4) == 0
        assert _plan_for(hs, 1 << 20) == (256, 4)
        assert _plan_for(hs, (1 << 20) + 1) == (256, 2)      # four-way does not apply
        assert hs.hs_set_option(b"merge_fanin", 2) == 0
        assert _plan_for(hs, 1 << 28) == (256, 2)
    finally:
        assert hs.hs_set_option(b"blocksort_shape", -1) == 0
        assert hs.hs_set_option(b"merge_fanin", 0) == 0
    assert _plan_for(hs, 1 << 28) == (288, 4)
    from paper_2503_05934_gb300 import _lib
    p = _lib.SortPlan()
    assert hs.hs_sort_plan_for(None, 100, 0x1, ctypes.byref(p)) == 1
    assert hs.hs_sort_plan_for(None, 100, 0x1C0, None) == 1


def test_sort_autotune_argument_errors(hs):
    from paper_2503_05934_gb300 import _lib
    p, ms = _lib.SortPlan(), ctypes.c_double(-1.0)
    n = 1 << 20
    need = hs.hs_sort_autotune_workspace_bytes(n)
    assert need >= hs.hs_sort_workspace_bytes(n, 0, 0) + 4 * n
    assert hs.hs_sort_autotune(FAKE, n, 0x1C0, FAKE, need, None, None, None) == 1
    assert hs.hs_sort_autotune(FAKE, n, 0x1, FAKE, need, None, ctypes.byref(p), None) == 1
    assert hs.hs_sort_autotune(None, n, 0x1C0, FAKE, need, None, ctypes.byref(p), None) == 1
    assert hs.hs_sort_autotune(FAKE + 2, n, 0x1C0, FAKE, need, None, ctypes.byref(p), None) == 1
    assert hs.hs_sort_autotune(FAKE, n, 0x1C0, FAKE, need - 1, None, ctypes.byref(p), None) == 1
    assert b"workspace" in hs.hs_last_error()
    assert hs.hs_sort_autotune(FAKE, n, 0x1C0, FAKE + 4, need, None, ctypes.byref(p), None) == 1
    # n <= 1: nothing to time, no device needed
    assert hs.hs_sort_autotune(None, 0, 0x1C0, None, 0, None, ctypes.byref(p), ctypes.byref(ms)) == 0
    assert (p.blocksort_threads, p.merge_fanin, ms.value) == (256, 2, 0.0)


def test_tune_cache_json_holds_both_kinds(hs, tmp_path):
    """Sort plans and batched plans share the cache file; a file with one
    invalid entry changes nothing (all or none)."""
    import json
    dev = "cache-test-device-a"
    src = tmp_path / "in.json"
    src.write_text(json.dumps([
        {"kind": "sort", "device": dev, "n_bucket": 24, "leaf": 8,
         "blocksort_threads": 256, "merge_fanin": 4, "ms": 1.25},
        {"device": dev, "n_bucket": 20, "s_bucket": 10, "m_bucket": 10, "netset": 0x1C0,
         "block_threads": 256, "ctas_per_sm": 0, "ms": 0.5},
    ]))
    assert hs.hs_tune_cache_load(str(src).encode()) == 0
    out = tmp_path / "out.json"
    assert hs.hs_tune_cache_save(str(out).encode()) == 0
    entries = [e for e in json.loads(out.read_text()) if e["device"] == dev]
    kinds = sorted(e["kind"] for e in entries)
    assert kinds == ["batched", "sort"]
    (s,) = [e for e in entries if e["kind"] == "sort"]
    assert (s["n_bucket"], s["leaf"], s["blocksort_threads"], s["merge_fanin"]) == (24, 8, 256, 4)
    assert abs(s["ms"] - 1.25) < 1e-9
    # Invalid sort entries: nothing from the file is cached.
    dev_b = "cache-test-device-b"
    for bad in [{"blocksort_threads": 300}, {"merge_fanin": 3}, {"leaf": 9}]:
        good = {"kind": "sort", "device": dev_b, "n_bucket": 20, "leaf": 8,
                "blocksort_threads": 288, "merge_fanin": 2, "ms": 1.0}
        src.write_text(json.dumps([good, dict(good, n_bucket=21, **bad)]))
        assert hs.hs_tune_cache_load(str(src).encode()) == 1
        assert hs.hs_tune_cache_save(str(out).encode()) == 0
        assert not [e for e in json.loads(out.read_text()) if e["device"] == dev_b]
    src.write_text(json.dumps([{"kind": "other", "device": dev_b}]))
    assert hs.hs_tune_cache_load(str(src).encode()) == 1
    assert b"unknown kind" in hs.hs_last_error()


def test_segsort_plan_for_defaults(hs):
    """With no tuned plan for this device (none on a machine without a GPU),
    a NULL batched plan is the network set with the default shape."""
    from paper_2503_05934_gb300 import _lib
    p = _lib.Plan()
    assert hs.hs_segsort_plan_for(100_000, 100, 0x1C0, ctypes.byref(p)) == 0
    assert p.as_dict() == {"netset": 0x1C0, "block_threads": 256, "ctas_per_sm": 0}
    assert hs.hs_segsort_plan_for(100_000, 100, 0xA8, ctypes.byref(p)) == 0
    assert p.netset == 0xA8
    assert hs.hs_segsort_plan_for(100_000, 100, 0x1, ctypes.byref(p)) == 1
    assert hs.hs_segsort_plan_for(100_000, 100, 0x1C0, None) == 1
