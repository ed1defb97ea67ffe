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
    ("merge_tile", 9, 5, [-1, 11]),
    ("merge_kernel", 1, 0, [2]),
    ("merge_samples", 1, 0, [2]),
    ("blocksort_shape", -1, 4, [-2, 6]),
    ("blocksort_bulk", 1, 0, [2, -1]),
    ("pairs_blocksort", 0, 3, [4]),
    ("pairs_merge", 3, 1, [4, -1]),
    ("pairs_blocksort_bulk", 1, 0, [2]),
    ("i64_merge", 1, 0, [2]),
    ("segsort_bulk", 1, 0, [2]),
    ("quick_partition", 3, 2, [1, 4]),
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
