"""The serving loop: continuous batching under a memory budget.  Each
request's result must be the same bit for bit as the same input sorted alone
(hs_sort_i32) and as the sorted input, whatever it was batched with."""
import numpy as np
import pytest

import hs_inputs as g
from helpers import hs_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return hs_module()


def _requests(n_req, seed, lo=8, hi=1 << 20):
    sizes = g.log_uniform_sizes(n_req, seed, lo, hi)
    dists = g.uniform_int(seed ^ 0x51, n_req, 0, 2)
    return [g.keys(int(s), g.DISTS[int(d)], seed * 7919 + i) for i, (s, d) in
            enumerate(zip(sizes, dists))]


def test_results_alone_equal_results_in_the_mix(hs):
    import torch
    inputs = _requests(300, 11)
    inputs += [np.zeros(0, np.int32), np.array([5], np.int32), g.random_i32(65_536, 1),
               g.random_i32(65_537, 2), g.random_i32(2_000_003, 3)]
    alone = []
    for a in inputs:
        t = torch.from_numpy(a.copy()).cuda()
        if a.size:
            hs.hs_sort_i32(t, "merge", "6To8")
        alone.append(t)
    torch.cuda.synchronize()
    mixed = [torch.from_numpy(a.copy()).cuda() for a in inputs]
    srv = hs.Server(512 << 20)
    try:
        arrivals = np.sort(np.random.default_rng(4).uniform(0, 0.05, len(inputs)))
        ptrs = [t.data_ptr() if t.numel() else 0 for t in mixed]
        lat, makespan = srv.replay(arrivals, ptrs, [t.numel() for t in mixed])
        stats = srv.stats()
    finally:
        srv.destroy()
    assert np.all(lat >= 0) and makespan > 0
    assert stats["batches"] >= 1 and stats["bytes_in_use"] == 0
    for a, x, y in zip(inputs, alone, mixed):
        assert torch.equal(x, y)
        assert np.array_equal(y.cpu().numpy(), np.sort(a))


def test_tight_budget_still_serves_everything(hs):
    import torch
    inputs = _requests(120, 12, 8, 1 << 18)
    mixed = [torch.from_numpy(a.copy()).cuda() for a in inputs]
    srv = hs.Server(8 << 20)  # far smaller than the sum: admission must throttle
    try:
        tickets = [srv.submit(t) for t in mixed]
        results = [srv.wait(tk) for tk in tickets]
        assert srv.stats()["bytes_in_use"] == 0
    finally:
        srv.destroy()
    assert all(st == 0 for st, _ in results)
    for a, y in zip(inputs, mixed):
        assert np.array_equal(y.cpu().numpy(), np.sort(a))


def test_over_budget_and_unsupported_requests(hs):
    import torch
    srv = hs.Server(4 << 20)
    try:
        big = torch.zeros(2 << 20, dtype=torch.int32, device="cuda")  # 8 MiB of keys
        with pytest.raises(hs.HsortError) as err:
            srv.submit(big)
        assert err.value.status == 6
        small = torch.zeros(100, dtype=torch.int32, device="cuda")
        with pytest.raises(hs.HsortError) as err:
            srv.submit(small, algo="quick")
        assert err.value.status == 2
    finally:
        srv.destroy()


def test_destroy_finishes_submitted_work(hs):
    """Shutting the server down with requests still queued (none waited for,
    under a budget that forces admission to throttle) completes every one of
    them before it frees anything."""
    import torch
    inputs = _requests(200, 13, 8, 1 << 19)
    mixed = [torch.from_numpy(a.copy()).cuda() for a in inputs]
    srv = hs.Server(16 << 20)
    for t in mixed:
        srv.submit(t)
    srv.destroy()
    torch.cuda.synchronize()
    for a, y in zip(inputs, mixed):
        assert np.array_equal(y.cpu().numpy(), np.sort(a))
