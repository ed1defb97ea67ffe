"""The seeded input generators: determinism and the stated distributions."""
import math

import numpy as np

import hs_inputs as g


def test_splitmix64_reference_values():
    # SplitMix64 with seed 0: published first outputs of the generator
    # (Steele, Lea, Flood 2014; the java.util.SplittableRandom sequence).
    out = g.splitmix64(0, 0, 3)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_chunks_agree():
    a = g.splitmix64(123, 0, 1000)
    b = np.concatenate([g.splitmix64(123, 0, 400), g.splitmix64(123, 400, 600)])
    assert np.array_equal(a, b)


def test_distributions():
    n = 100_000
    r = g.keys(n, "random", 1)
    assert r.dtype == np.int32 and r.size == n
    assert np.array_equal(r, g.keys(n, "random", 1))
    assert r.min() < -(1 << 30) and r.max() > (1 << 30)
    s = g.keys(n, "sorted", 2)
    assert np.all(np.diff(s.astype(np.int64)) >= 0)
    assert s[0] < -(1 << 30) and s[-1] > (1 << 30)
    nearly = g.keys(n, "nearly", 2)
    moved = np.count_nonzero(nearly != s)
    assert 0 < moved <= 2 * (n // 100)
    assert np.array_equal(np.sort(nearly), s)


def test_pair_keys():
    k, v = g.pair_keys_16bit(1 << 18, 5)
    assert np.unique(k).size <= 1 << 16
    assert np.array_equal(v, np.arange(1 << 18, dtype=np.int32))


def test_segment_sizes():
    sz = g.segment_sizes(200_000, 5)
    assert sz.min() >= 3 and sz.max() <= 65536
    mean = (65536 - 3) / math.log(65536 / 3)
    assert abs(sz.mean() / mean - 1) < 0.02
    keys, off, d = g.segmented(500, 6)
    assert off[0] == 0 and off[-1] == keys.size and np.all(np.diff(off) >= 3)
    assert set(np.unique(d)) <= {0, 1, 2}


def test_poisson():
    t = g.poisson_arrivals(20000, 100.0, 3)
    gaps = np.diff(t)
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() * 100.0 - 1) < 0.05


def test_c_forms_match_numpy_definitions():
    for n in [0, 1, 7, 99, 100, 1000, 12345]:
        assert np.array_equal(g.random_i32(n, 3), g.np_random_i32(n, 3))
        assert np.array_equal(g.sorted_i32(n, 4), g.np_sorted_i32(n, 4))
        assert np.array_equal(g.nearly_sorted_i32(n, 5), g.np_nearly_sorted_i32(n, 5))
    sizes = np.array([3, 0, 250, 1000, 7, 4096, 65536, 1, 333], np.int64)
    for seed in [1, 2, 3]:
        a = g.segmented(0, seed, sizes=sizes)
        b = g.np_segmented(0, seed, sizes=sizes)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    a = g.segmented(400, 9)
    b = g.np_segmented(400, 9)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_int64_keys():
    n = 100_000
    r = g.keys_i64(n, "random", 1)
    assert r.dtype == np.int64 and np.array_equal(r, g.keys_i64(n, "random", 1))
    assert r.min() < -(1 << 62) and r.max() > (1 << 62)
    s = g.keys_i64(n, "sorted", 2)
    assert np.all(s[1:] >= s[:-1]) and s[0] < -(1 << 62) and int(s[-1]) - int(s[0]) > (1 << 62)
    nearly = g.keys_i64(n, "nearly", 2)
    assert 0 < np.count_nonzero(nearly != s) <= 2 * (n // 100)
    assert np.array_equal(np.sort(nearly), s)
