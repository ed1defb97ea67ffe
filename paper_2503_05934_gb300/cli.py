"""Sorts one synthetic array on the GPU through the library's public calls and
prints the time per sort.

    python -m paper_2503_05934_gb300.cli --what keys --log2n 26 --dist uniform
    python -m paper_2503_05934_gb300.cli --what pairs --log2n 25 --reps 3
    python -m paper_2503_05934_gb300.cli --what int64 --log2n 27
    python -m paper_2503_05934_gb300.cli --what quick --dist nearly --option quick_max_levels=64
    python -m paper_2503_05934_gb300.cli --what batched --segments 20000

Keys are int32 from the seeded generators of ``hs_inputs`` (uniform over the
int32 range, sorted, or nearly sorted); pairs carry keys from 2^16 distinct
values and values = original index; int64 keys are uniform over the int64
range (or sorted / nearly sorted); batched runs sort --segments arrays of
log-uniform sizes in [3, 65536] (mixed distributions), or with --seg-size S
2^log2n keys in arrays of S keys each, in one launch with the default plan.
Every run restores the input from a
pristine device copy (untimed), times the sort with CUDA events on the
sorting stream, and checks that the output is sorted (pairs: and stable).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--what", choices=["keys", "quick", "pairs", "int64", "batched"], default="keys")
    ap.add_argument("--segments", type=int, default=20000)
    ap.add_argument("--seg-size", type=int, default=0,
                    help="batched: every segment this long, 2^log2n keys in all "
                         "(default: --segments log-uniform sizes)")
    ap.add_argument("--log2n", type=int, default=24)
    ap.add_argument("--dist", choices=["uniform", "sorted", "nearly"], default="uniform")
    ap.add_argument("--netset", default="6To8")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--option", action="append", default=[], help="name=value for hs_set_option")
    ap.add_argument("--breakdown", action="store_true",
                    help="also time every launch of one more run, per kernel")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    import hs_inputs
    import paper_2503_05934_gb300 as hs

    for opt in args.option:
        name, value = opt.split("=")
        hs.hs_set_option(name, int(value))
    dev = torch.device("cuda", 0)
    n = 1 << args.log2n
    st = torch.cuda.current_stream(dev)
    if args.what == "pairs":
        k, v = hs_inputs.pair_keys_16bit(n, args.seed)
        src = [torch.from_numpy(k).to(dev), torch.from_numpy(v).to(dev)]
        ws = torch.empty(hs.hs_sort_workspace_bytes(n, True), dtype=torch.uint8, device=dev)

        def run(bufs):
            hs.hs_sort_pairs_i32(bufs[0], bufs[1], "merge", args.netset, ws=ws, stream=st)
    elif args.what == "int64":
        dist = "random" if args.dist == "uniform" else args.dist
        src = [torch.from_numpy(hs_inputs.keys_i64(n, dist, args.seed)).to(dev)]
        ws = torch.empty(hs.hs_sort_i64_workspace_bytes(n), dtype=torch.uint8, device=dev)

        def run(bufs):
            hs.hs_sort_i64(bufs[0], "merge", args.netset, ws=ws, stream=st)
    elif args.what == "batched":
        if args.seg_size > 0:
            sizes = np.full(max(1, n // args.seg_size), args.seg_size, np.int64)
            keys, off, _ = hs_inputs.segmented(0, args.seed, sizes=sizes)
        else:
            keys, off, _ = hs_inputs.segmented(args.segments, args.seed)
        n = keys.size
        src = [torch.from_numpy(keys).to(dev)]
        offs = torch.from_numpy(off).to(dev)

        def run(bufs):
            hs.hs_segsort_i32(bufs[0], offs, "merge", args.netset, stream=st)
    else:
        dist = "random" if args.dist == "uniform" else args.dist
        src = [torch.from_numpy(hs_inputs.keys(n, dist, args.seed)).to(dev)]
        algo = "quick" if args.what == "quick" else "merge"
        ws = torch.empty(hs.hs_sort_workspace_bytes(n, False, algo), dtype=torch.uint8, device=dev)

        def run(bufs):
            hs.hs_sort_i32(bufs[0], algo, args.netset, ws=ws, stream=st)
    work = [torch.empty_like(t) for t in src]
    times = []
    for _ in range(args.reps):
        for w_, s_ in zip(work, src):
            w_.copy_(s_)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        run(work)
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    hs.hs_device_check()
    keys = work[0]
    if args.what == "batched":
        d = keys[1:] >= keys[:-1]
        d[offs[1:-1] - 1] = True  # segment boundaries
        ok = bool(d.all().item())
    else:
        ok = bool((keys[1:] >= keys[:-1]).all().item())
    if args.what == "pairs":
        same = keys[1:] == keys[:-1]
        ok = ok and bool(((work[1][1:] > work[1][:-1]) | ~same).all().item())
    out = {"what": args.what, "n": n, "dist": args.dist, "netset": args.netset, "ms": times,
           "sorted": ok}
    if args.breakdown:
        # One more run with every launch bracketed by events.
        for w_, s_ in zip(work, src):
            w_.copy_(s_)
        hs.hs_prof_reset()
        hs.hs_prof_enable(True)
        run(work)
        torch.cuda.synchronize()
        hs.hs_prof_enable(False)
        out["kernels"] = {}
        for name in ("blocksort_keys", "blocksort_pairs", "merge_partition", "merge_keys", "merge4_keys",
                     "merge_pairs", "qs_plan", "qs_partition", "qs_leaves", "seg_classify",
                     "seg_sort"):
            launches, ms = hs.hs_prof_read(name)
            if launches:
                out["kernels"][name] = {"launches": launches, "ms": ms}
    print(json.dumps(out))
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
