"""Shared helpers for the GPU tests (device marshalling and full-size checks)."""
import numpy as np

import oracle


def hs_module():
    from paper_2503_05934_gb300 import build
    build.build()
    import paper_2503_05934_gb300 as hs
    return hs


def to_dev(a: np.ndarray, offset: int = 0):
    """Copies a to the device; offset > 0 shifts the start by that many int32
    slots inside a larger allocation (4-byte but not 16-byte aligned)."""
    import torch
    if offset == 0:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    buf = torch.empty(a.size + offset, dtype=torch.int32, device="cuda")
    view = buf[offset:]
    view.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return view


def fingerprint(a: np.ndarray) -> tuple:
    """Order-independent multiset summary: count, sum, sum of squares
    (mod 2^64), xor and a hashed sum."""
    x = a.astype(np.int64)
    u = a.view(np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = (u * np.uint64(0x9E3779B97F4A7C15)) ^ (u >> np.uint64(7))
        return (a.size, int(x.sum()), int((x.astype(np.uint64) * x.astype(np.uint64)).sum()),
                int(np.bitwise_xor.reduce(u)) if a.size else 0, int(h.sum()))


def check_sorted_permutation(inp: np.ndarray, out: np.ndarray, samples: int = 8, seed: int = 0):
    """Full-size check: out is non-decreasing, has the multiset fingerprint of
    inp, and sampled ranks agree with the oracle's order-statistic counts."""
    assert out.size == inp.size
    assert oracle.is_sorted(out)
    assert fingerprint(out) == fingerprint(inp)
    rng = np.random.default_rng(seed)
    for r in rng.integers(0, inp.size, samples).tolist() + [0, inp.size - 1]:
        v = int(out[r])
        # out[r] is the r-th order statistic: #(< v) <= r < #(<= v)
        assert oracle.count_less(inp, v) <= r < oracle.count_less_equal(inp, v)


def check_stable_pairs_index_values(k_in, k_out, v_out):
    """Complete check of a stable sort whose values are the input indices."""
    n = k_in.size
    assert oracle.is_sorted(k_out)
    assert np.array_equal(np.bincount(v_out, minlength=n), np.ones(n, np.int64))
    assert np.array_equal(k_in[v_out], k_out)
    same = k_out[1:] == k_out[:-1]
    assert np.all(v_out[1:][same] > v_out[:-1][same])
