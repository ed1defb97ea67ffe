"""Benchmark: hybrid network-leaf merge sort of 2^28 uniform int32 keys on GB300.

One step = one full sort (block sort with {6,7,8} network leaves + every
global merge level) of n = 2^28 uniform int32 keys resident in HBM.  Prints
ONE JSON line (rank 0).  Multi-GPU runs are independent replicas: each rank
sorts its own array, no collective touches the data path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm (--impl reference) times the plain CPU oracle
(Algorithm 1 with {6,7,8} leaves, single thread) on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hs_inputs  # noqa: E402

METRIC = "int32 keys/s & %HBM roofline; batched vs plain keys/s; serve p50/p99"
UNIT = "keys/s"
FALLBACK_HBM_GBS = 6800.0
SPEC_HBM_GBS = 8000.0
# Sources of each merge-level kernel the roofline may name (the kernel, its
# launch shape and its partition pass): a committed ncu traffic figure applies
# only while these are unchanged.
_CSRC = "paper_2503_05934_gb300/csrc/"
KERNEL_SOURCES = {
    "merge_keys": [_CSRC + f for f in ("hs_merge_tile.cuh", "hs_bulk.cuh",
                                       "hs_merge_prims.cuh", "hs_common.cuh")],
    "merge4_keys": [_CSRC + f for f in ("hs_merge4.cuh", "hs_bulk.cuh",
                                        "hs_merge_prims.cuh", "hs_common.cuh")],
}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--log2n", type=int, default=28)
    p.add_argument("--netset", default="6To8")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--serve-requests", type=int, default=20000)
    p.add_argument("--no-ablation", action="store_true",
                   help="skip the Table 3 network-set ablation at the paper's sizes")
    p.add_argument("--option", action="append", default=[],
                   help="library tuning option name=value (hs_set_option)")
    return p.parse_args()


def workload_config(args, n):
    return {
        "workload": f"hybrid merge sort, n=2^{args.log2n} uniform int32 keys, "
                    f"{args.netset} network leaves",
        "n": n, "dist": "uniform over [INT32_MIN, INT32_MAX]", "algo": "merge",
        "netset": args.netset, "seed": hs_inputs.config_seed(2),
        "l2": (f"inputs larger than L2 ({4 * n / 2**20:.0f} MiB per array vs 129 MB L2)"
               if 4 * n > 129e6 else f"input of {4 * n / 2**20:.1f} MiB may stay in the 129 MB L2"),
        "restore": "in-place sort; the input is restored from a pristine device copy "
                   "before each step, outside the timed events",
        "parallelism": "replicas (one independent array per GPU)",
    }


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, pg, device) -> float:
    """The maximum of a per-rank float over all ranks (the value itself
    without a process group): the slowest rank sets the job's time."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units per second of the whole job: every rank processes its own
    units (replicas), all within the slowest rank's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (every 100 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kernel: str = "merge_keys") -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(n: int, kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary
    (profiles/<kernel>_2p28_uniform.md), scaled to n keys, or None when there
    is none or the kernel sources changed since the capture."""
    try:
        text = open(os.path.join(ROOT, "profiles", f"{kernel}_2p28_uniform.md")).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
    m_bpk = re.search(r"dram_bytes_per_key_per_launch:\s*([0-9.]+)", text)
    if not m_hash or not m_bpk or kernel not in KERNEL_SOURCES or \
            m_hash.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_bpk.group(1)) * n


def sort_passes(n: int, tile: int) -> int:
    p, w = 1, tile
    while w < n:
        w *= 2
        p += 1
    return p


def host_cpu_info() -> dict:
    """The host the CPU baseline ran on: architecture, logical cores, model."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "model": model}


def library_sort_rate(sample: np.ndarray, seconds: float = 2.0) -> float:
    """numpy's library sort on the same sample, one core: context for the
    oracle's rate (a tuned library sort against the paper's algorithms)."""
    done, t_total = 0, 0.0
    while done == 0 or t_total < seconds:
        t0 = time.perf_counter()
        np.sort(sample)
        t_total += time.perf_counter() - t0
        done += sample.size
    return done / t_total


def cpu_oracle_rate(sample: np.ndarray, seconds: float, netset: str):
    import oracle
    done, t_total, reps = 0, 0.0, 0
    while reps == 0 or t_total < seconds:
        t0 = time.perf_counter()
        oracle.merge_sort(sample, netset)
        t_total += time.perf_counter() - t0
        done += sample.size
        reps += 1
    return done / t_total, reps


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = 1 << args.log2n
    sample_n = min(n, 1 << 22)
    a = hs_inputs.random_i32(sample_n, hs_inputs.config_seed(2))
    import oracle
    oracle.lib()
    for _ in range(args.warmup):
        oracle.merge_sort(a, args.netset)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.merge_sort(a, args.netset)
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = sample_n / mean
    sample = (f"first 2^{int(np.log2(sample_n))} keys of the 2^{args.log2n} uniform workload, "
              f"one full oracle sort per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
        "data": "synthetic", "config": workload_config(args, n),
        # what each step actually sorted: a bounded sample of the workload
        # named in config, so keys/s compare per key
        "sample_sorted": {"n": sample_n, "of_n": n, "keys": "first keys of the same seeded array"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    ws_world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws_world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_2503_05934_gb300 import build as hs_build
    hs_build.build()
    import paper_2503_05934_gb300 as hs

    for opt in args.option:
        name, value = opt.split("=")
        hs.hs_set_option(name, int(value))
    n = 1 << args.log2n
    seed = hs_inputs.config_seed(2, salt=rank)
    host = hs_inputs.random_i32(n, seed)
    pristine = torch.from_numpy(host).to(dev)
    work = torch.empty_like(pristine)
    wsb = torch.empty(hs.hs_sort_workspace_bytes(n), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # Everything alive now (torch, numpy, the inputs) stays out of the
    # garbage collector's scans: a collection during a measurement then costs
    # microseconds, not the tens of milliseconds a full scan takes here.
    gc.collect()
    gc.freeze()

    def step_timed():
        work.copy_(pristine)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs.hs_sort_i32(work, "merge", args.netset, ws=wsb, stream=stream)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        step_timed()
    torch.cuda.synchronize(dev)

    # Per-kernel breakdown from a few more (untimed) steps with every launch
    # bracketed by events: it names the dominant kernel and counts the passes
    # over the keys (every block-sort or merge launch reads and writes each
    # key once).
    hs.hs_prof_reset()
    hs.hs_prof_enable(True)
    brk_steps = 3
    for _ in range(brk_steps):
        step_timed()
    torch.cuda.synchronize(dev)
    hs.hs_prof_enable(False)
    kernels = ("blocksort_keys", "merge_partition", "merge_keys", "merge4_keys")
    brk = {k: hs.hs_prof_read(k) for k in kernels}
    breakdown = {k: ms / brk_steps for k, (cnt, ms) in brk.items() if cnt}
    launches_per_sort = {k: cnt // brk_steps for k, (cnt, ms) in brk.items() if cnt}
    dominant = max(breakdown, key=breakdown.get)
    passes_design = sum(launches_per_sort.get(k, 0)
                        for k in ("blocksort_keys", "merge_keys", "merge4_keys"))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # Inside the timed region only the dominant kernel carries timing events
    # (its average launch duration gives the roofline figure).
    hs.hs_prof_reset()
    hs.hs_prof_select(dominant)
    hs.hs_prof_enable(True)
    launches0 = hs.hs_launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    gc.collect()
    gc.disable()
    t_wall0 = time.perf_counter()
    evs = [step_timed() for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    gc.enable()
    if pg:
        pg.barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = hs.hs_launch_count() - launches0
    hs.hs_prof_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    mk_launches, mk_ms = hs.hs_prof_read(dominant)
    hs.hs_prof_select(None)

    # Correctness guard on the last result (cheap: sortedness on the device).
    assert bool((work[1:] >= work[:-1]).all().item()), "benchmark output not sorted"

    total_ms = max_over_ranks(total_ms, pg, dev)
    value = whole_job_rate(ws_world, n * args.steps, total_ms / 1e3)
    peak, peak_kind = measured_peak()
    avg_mk_s = (mk_ms / mk_launches) / 1e3 if mk_launches else None
    # one read + one write of every key per launch (block sort, binary or
    # four-way merge level alike)
    alg_bytes = 8.0 * n
    achieved = alg_bytes / avg_mk_s / 1e9 if avg_mk_s else None
    traffic = profiled_traffic(n, dominant)
    roofline = {
        "kernel": dominant, "bound": "hbm", "achieved": achieved, "peak": peak,
        "peak_kind": peak_kind, "unit": "GB/s",
        "frac": achieved / peak if achieved else None, "traffic": traffic,
        "algorithmic_bytes_per_launch": alg_bytes,
        "launch_ms": avg_mk_s * 1e3 if avg_mk_s else None,
        # ncu DRAM bytes over the live launch time: bandwidth actually drawn
        "traffic_gbs": traffic / avg_mk_s / 1e9 if traffic and avg_mk_s else None,
    }
    p_ref = sort_passes(n, 8192)
    ms_step = total_ms / args.steps
    whole = None
    if passes_design:
        # P_counted = min(P_design, P_ref): passes the design makes, never
        # more than the binary reference with an 8192-key tile.
        b = min(passes_design, p_ref) * 2 * 4 * n
        b_ref = p_ref * 2 * 4 * n
        whole = {"passes": passes_design, "passes_ref": p_ref, "bytes": b,
                 "frac_of_measured": b / (ms_step / 1e3) / (peak * 1e9),
                 "frac_of_8tbs": b / (ms_step / 1e3) / (SPEC_HBM_GBS * 1e9),
                 # the same time against the binary reference's bytes
                 "frac_of_measured_at_passes_ref": b_ref / (ms_step / 1e3) / (peak * 1e9),
                 "launches_per_sort": launches_per_sort,
                 "one_pass_bound_ms": 2 * 4 * n / (peak * 1e9) * 1e3}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
        "data": "synthetic", "config": workload_config(args, n),
        "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "sort_roofline": whole,
        # every launch timed, from 3 extra steps after the timed region
        "kernel_ms_per_step": breakdown,
        "wall_s_timed_region": t_wall,
    }

    del work
    # ---- end to end through the host-buffer C-ABI call (pinned host memory)
    if not args.no_e2e:
        h_pristine = host
        h_buf = torch.empty(n, dtype=torch.int32).pin_memory()
        ws_h = torch.empty(hs.hs_sort_host_workspace_bytes(n), dtype=torch.uint8, device=dev)
        for _ in range(max(1, min(args.warmup, 3))):
            h_buf.numpy()[:] = h_pristine
            hs.hs_sort_i32_host(h_buf, "merge", args.netset, ws=ws_h, stream=stream)
        e2e_steps = max(1, min(args.steps, 20))
        step_s = []
        # The harness's own garbage collection is kept out of the timed calls
        # (as timeit does): a full collection in this long-lived process can
        # take tens of milliseconds.
        gc.collect()
        gc.disable()
        for _ in range(e2e_steps):
            h_buf.numpy()[:] = h_pristine
            if pg:
                pg.barrier()
            t0 = time.perf_counter()
            hs.hs_sort_i32_host(h_buf, "merge", args.netset, ws=ws_h, stream=stream)
            step_s.append(time.perf_counter() - t0)
        gc.enable()
        tot = max_over_ranks(sum(step_s), pg, dev)
        assert bool(np.all(h_buf.numpy()[1:] >= h_buf.numpy()[:-1])), "e2e output not sorted"
        # The host link on this machine: plain copies of the same bytes, each
        # way (context for how much of the end-to-end time is copying).
        d_tmp = torch.empty(n, dtype=torch.int32, device=dev)
        link = {}
        for name, dst, src in (("h2d_gbs", d_tmp, h_buf), ("d2h_gbs", h_buf, d_tmp)):
            best = None
            for _ in range(3):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                dst.copy_(src, non_blocking=True)
                torch.cuda.synchronize(dev)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            link[name] = 4 * n / best / 1e9
        del d_tmp
        copy_ms = 4 * n / (link["h2d_gbs"] * 1e9) * 1e3 + 4 * n / (link["d2h_gbs"] * 1e9) * 1e3
        line["e2e"] = {"value": whole_job_rate(ws_world, n * e2e_steps, tot), "unit": UNIT,
                       "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
                       "steps": e2e_steps, "api": "hs_sort_i32_host (pinned host buffer)",
                       "ms_per_step": tot / e2e_steps * 1e3,
                       # this rank's calls one by one (the host link and host
                       # memory are shared with other jobs on the node)
                       "ms_steps": [round(x * 1e3, 3) for x in step_s],
                       "ms_per_step_median": float(np.median(step_s)) * 1e3,
                       "link": {k: round(v, 1) for k, v in link.items()},
                       # both copies back to back, nothing else: the floor
                       # for a call that must copy in before it can copy out
                       "copies_alone_ms": copy_ms}
        del ws_h, h_buf

    # ---- extra forms (stable pairs), timed the same way
    if not args.no_extras:
        line["extras"] = run_extras(hs, torch, dev, stream, args, rank, pristine, passes_design)

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    if rank == 0 and ws_world == 1 and not args.no_cpu and not args.no_extras:
        line.setdefault("extras", {})["cpu_speedups"] = cpu_speedups()
    if rank == 0 and ws_world == 1 and not args.no_cpu:
        sample_n = min(n, 1 << 22)
        rate, reps = cpu_oracle_rate(host[:sample_n].copy(), args.cpu_seconds, args.netset)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^22 keys of the workload, oracle Algorithm 1 ({args.netset}), "
                      f"{reps} full sorts on one host core",
            "host": host_cpu_info(),
            "library_sort_value": library_sort_rate(host[:sample_n].copy())}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def time_sorts(torch, stream, reps, warmup, restore, sort):
    """Mean CUDA-event milliseconds of `sort` over `reps` runs after `warmup`;
    `restore` (untimed) re-creates the unsorted input before each run."""
    evs = []
    for i in range(warmup + reps):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sort()
        e1.record(stream)
        if i >= warmup:
            evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / len(evs)


def run_extras(hs, torch, dev, stream, args, rank, pristine, passes_design):
    out = {}
    n_keys = pristine.numel()
    peak, peak_kind = measured_peak()
    reps = max(3, args.steps // 4)
    # Both paths on the three distributions of the paper's experiments
    # (uniform, sorted, nearly sorted) at the headline size; the merge path
    # on uniform keys is the headline line itself.
    tile = int(hs.lib().hs_keys_tile(hs.netset_mask(args.netset), n_keys))
    # the merge path's passes over the keys, counted from its launches
    p_counted = min(passes_design, sort_passes(n_keys, 8192)) if passes_design else None
    work = torch.empty_like(pristine)
    wsm = torch.empty(hs.hs_sort_workspace_bytes(n_keys), dtype=torch.uint8, device=dev)
    wsq = torch.empty(hs.hs_sort_workspace_bytes(n_keys, False, "quick"), dtype=torch.uint8,
                      device=dev)
    seed = hs_inputs.config_seed(2, salt=2 + (rank << 8))
    for dist in ["uniform", "sorted", "nearly"]:
        src = pristine if dist == "uniform" else torch.from_numpy(
            hs_inputs.keys(n_keys, dist, seed)).to(dev)
        for algo in (["quick"] if dist == "uniform" else ["merge", "quick"]):
            ws = wsm if algo == "merge" else wsq
            ms = time_sorts(torch, stream, reps, 2, lambda: work.copy_(src),
                            lambda: hs.hs_sort_i32(work, algo, args.netset, ws=ws, stream=stream))
            assert bool((work[1:] >= work[:-1]).all().item()), f"{algo} {dist} output not sorted"
            entry = {"value": n_keys / (ms / 1e3), "unit": "keys/s", "ms_per_sort": ms,
                     "workload": f"2^{args.log2n} {dist} int32, "
                                 + ("hybrid merge sort" if algo == "merge" else
                                    "median-of-three 3-way partitions")
                                 + f", {args.netset} leaves"}
            if algo == "merge" and p_counted:
                entry["frac_of_measured"] = p_counted * 8 * n_keys / (ms / 1e3) / (peak * 1e9)
            elif algo == "quick" and tile:
                # Partition levels of a binary split down to one tile, plus
                # the final block-sort pass: counted at (2 reads + 1 write)
                # per key and level (a count-then-scatter partition), and at
                # the one read + one write the one-pass partition moves.
                levels = sort_passes(n_keys, tile) - 1
                qbytes = 12 * n_keys * levels + 8 * n_keys
                qbytes1 = 8 * n_keys * levels + 8 * n_keys
                entry["roofline_bytes"] = qbytes
                entry["frac_of_measured"] = qbytes / (ms / 1e3) / (peak * 1e9)
                entry["roofline_bytes_one_pass"] = qbytes1
                entry["frac_of_measured_one_pass"] = qbytes1 / (ms / 1e3) / (peak * 1e9)
            out[f"{algo}_2p{args.log2n}_{dist}"] = entry
        del src
    # The single-array autotuner on the headline workload: the plan it picks
    # (block-sort CTA size, merge fan-in) beside the built-in rules' plan.
    # The tuned plan is cleared afterwards so the extras below run on the rules.
    work.copy_(pristine)
    rule = hs.hs_sort_plan_for(n_keys, args.netset, work).as_dict()
    wst = torch.empty(int(hs.lib().hs_sort_autotune_workspace_bytes(n_keys)), dtype=torch.uint8,
                      device=dev)
    t0 = time.perf_counter()
    plan, best_ms = hs.hs_sort_autotune(work, args.netset, ws=wst, stream=stream)
    tune_s = time.perf_counter() - t0
    assert torch.equal(work, pristine), "the autotuner changed the keys"
    out["autotune_2p%d" % args.log2n] = {"plan": plan.as_dict(), "best_ms": best_ms, "rule_plan": rule,
                                         "tuning_s": tune_s,
                                         "candidates": "blocksort_threads 256/288 x merge_fanin 2/4, "
                                                       "one warm-up and two timed sorts each"}
    hs.hs_tune_cache_clear()
    del wst
    del work, wsm, wsq
    # Stable pairs: 2^27 keys from 2^16 distinct values, value = index.
    n = 1 << (args.log2n - 1)
    k, v = hs_inputs.pair_keys_16bit(n, hs_inputs.config_seed(2, salt=1 + (rank << 8)))
    pk, pv = torch.from_numpy(k).to(dev), torch.from_numpy(v).to(dev)
    wk, wv = torch.empty_like(pk), torch.empty_like(pv)
    wsb = torch.empty(hs.hs_sort_workspace_bytes(n, True), dtype=torch.uint8, device=dev)

    def restore_pairs():
        wk.copy_(pk)
        wv.copy_(pv)

    ms = time_sorts(torch, stream, max(3, args.steps // 2), args.warmup, restore_pairs,
                    lambda: hs.hs_sort_pairs_i32(wk, wv, "merge", args.netset, ws=wsb,
                                                 stream=stream))
    ok = bool((wk[1:] >= wk[:-1]).all().item())
    same = wk[1:] == wk[:-1]
    ok = ok and bool(((wv[1:] > wv[:-1]) | ~same).all().item())  # value = index: stable
    assert ok, "pair sort output not sorted or not stable"
    # passes over the pairs: block-sort and merge launches of one more sort
    restore_pairs()
    hs.hs_prof_reset()
    hs.hs_prof_enable(True)
    hs.hs_sort_pairs_i32(wk, wv, "merge", args.netset, ws=wsb, stream=stream)
    torch.cuda.synchronize(dev)
    hs.hs_prof_enable(False)
    p_design = hs.hs_prof_read("blocksort_pairs")[0] + hs.hs_prof_read("merge_pairs")[0]
    pp = min(p_design, sort_passes(n, 8192)) if p_design else None
    out[f"pairs_stable_2p{args.log2n - 1}"] = {
        "value": n / (ms / 1e3), "unit": "pairs/s", "ms_per_sort": ms,
        "passes": p_design, "passes_ref": sort_passes(n, 8192),
        "frac_of_measured": pp * 16 * n / (ms / 1e3) / (peak * 1e9) if pp else None,
        "frac_of_measured_at_passes_ref": sort_passes(n, 8192) * 16 * n / (ms / 1e3) / (peak * 1e9),
        "workload": f"2^{args.log2n - 1} (int32 key from 2^16 values, int32 index) "
                    f"stable merge sort, {args.netset} leaves"}
    del pk, pv, wk, wv, wsb
    # int64 keys: 2^27 (1 GiB), uniform over the int64 range.
    a64 = torch.from_numpy(hs_inputs.keys_i64(n, "random", hs_inputs.config_seed(2, salt=64))).to(dev)
    w64 = torch.empty_like(a64)
    ws64 = torch.empty(hs.hs_sort_i64_workspace_bytes(n), dtype=torch.uint8, device=dev)
    ms = time_sorts(torch, stream, max(3, args.steps // 4), 2, lambda: w64.copy_(a64),
                    lambda: hs.hs_sort_i64(w64, "merge", args.netset, ws=ws64, stream=stream))
    assert bool((w64[1:] >= w64[:-1]).all().item()), "int64 sort output not sorted"
    p64 = sort_passes(n, int(hs.lib().hs_i64_tile(hs.netset_mask(args.netset), n)))
    out[f"merge_int64_2p{args.log2n - 1}"] = {
        "value": n / (ms / 1e3), "unit": "keys/s", "ms_per_sort": ms, "passes": p64,
        "frac_of_measured": min(p64, sort_passes(n, 8192)) * 16 * n / (ms / 1e3) / (peak * 1e9),
        "workload": f"2^{args.log2n - 1} uniform int64 keys, hybrid merge sort, {args.netset} leaves"}
    del a64, w64, ws64
    if not args.no_ablation:
        out["netset_ablation"] = run_netset_ablation(hs, torch, dev, stream)
    if not args.no_batched:
        out["batched_segsort"] = run_batched(hs, torch, dev, stream, args)
    if not args.no_serve:
        out["serve"] = run_serving(hs, torch, dev, args)
    return out


ABLATION_SIZES = (10_000, 25_000, 100_000, 1_000_000)
ABLATION_SETS = ("none", "3", "3To4", "3To5", "6To8", "3To8", "PowerOf2", "Even", "Odd",
                 "VarSort3", "VarSort4", "VarSort5")


def run_netset_ablation(hs, torch, dev, stream):
    """Every Table 3 network set at the paper's sizes and distributions, for
    both paths (the GPU counterpart of the paper's speedup figures): mean
    microseconds per sort and the speedup over the classical set ("none")."""
    out = {}
    for n in ABLATION_SIZES:
        ws = torch.empty(max(hs.hs_sort_workspace_bytes(n, False, a) for a in ("merge", "quick")),
                         dtype=torch.uint8, device=dev)
        for dist in ("random", "sorted", "nearly"):
            src = torch.from_numpy(hs_inputs.keys(n, dist, hs_inputs.config_seed(1, salt=n))).to(dev)
            work = torch.empty_like(src)
            for algo in ("merge", "quick"):
                us = {}
                for netset in ABLATION_SETS:
                    ms = time_sorts(torch, stream, 10, 3, lambda: work.copy_(src),
                                    lambda: hs.hs_sort_i32(work, algo, netset, ws=ws, stream=stream))
                    us[netset] = round(ms * 1e3, 2)
                assert bool((work[1:] >= work[:-1]).all().item())
                out[f"{algo}/{dist}/{n}"] = {
                    "us": us, "speedup_vs_none": {k: round(us["none"] / v, 3) for k, v in us.items()}}
    return out


# The paper's speedups of the hybrid sorts over the classical ones (Eq. 1),
# single-threaded on a Ryzen 5 1600AF, as printed in its text (its figures are
# not available): context for the oracle's speedups on this machine's host.
PAPER_CPU_SPEEDUPS = {
    "merge/random/6To8": "about 2x at n = 10,000, about 1.5x up to 1,000,000",
    "merge/sorted/3To8": "slightly above 2x from 10,000 to 1,000,000",
    "merge/nearly/3To8": "above 1.5x at every size",
    "quick/random/3To8": "about 1.25x at 10,000; others negligible",
    "quick/sorted/6To8": "about 1.5x from 25,000 to 1,000,000",
    "quick/nearly/3To8": "about 1.3x from 10,000",
}


def cpu_speedups(seconds_cap: float = 20.0):
    """The oracle's speedup of each hybrid over its classical form (Eq. 1:
    T_classical / T_hybrid) on one host core, at the paper's sizes and
    distributions, beside the paper's own figures."""
    import oracle
    oracle.lib()
    t_start = time.perf_counter()
    out = {}
    for algo in ("merge", "quick"):
        sort = oracle.merge_sort if algo == "merge" else oracle.quick_sort
        for dist in ("random", "sorted", "nearly"):
            for n in ABLATION_SIZES:
                a = hs_inputs.keys(n, dist, hs_inputs.config_seed(1, salt=n))
                t = {}
                for netset in ("none", "3To5", "6To8", "3To8"):
                    reps = 3 if n >= 1_000_000 else 7
                    best = float("inf")
                    for _ in range(reps):
                        t0 = time.perf_counter()
                        sort(a, netset)
                        best = min(best, time.perf_counter() - t0)
                    t[netset] = best
                out[f"{algo}/{dist}/{n}"] = {k: round(t["none"] / v, 3) for k, v in t.items()
                                             if k != "none"}
                if time.perf_counter() - t_start > seconds_cap:
                    out["truncated"] = f"stopped after {seconds_cap:.0f} s"
                    return {"speedup_vs_classical": out, "paper": PAPER_CPU_SPEEDUPS,
                            "cores": 1, "kind": "oracle"}
    return {"speedup_vs_classical": out, "paper": PAPER_CPU_SPEEDUPS, "cores": 1, "kind": "oracle",
            "timing": "best of 3 (1,000,000 keys) or 7 runs per sort, one host core"}


def run_batched(hs, torch, dev, stream, args):
    """200,000 independent arrays, sizes log-uniform in [3, 65536], mixed
    distributions: one persistent launch replayed from a CUDA graph with the
    autotuned plan, against one hs_sort_i32 call per array on one stream."""
    keys, off, _ = hs_inputs.segmented(200_000, hs_inputs.config_seed(3))
    n = keys.size
    pristine = torch.from_numpy(keys).to(dev)
    del keys
    work = torch.empty_like(pristine)
    offs = torch.from_numpy(off).to(dev)
    work.copy_(pristine)
    plan, tune_ms = hs.hs_segsort_autotune(work, offs, stream=stream)
    graph = hs.hs_segsort_capture(work, offs, plan)
    launches0 = hs.hs_launch_count()
    ms = time_sorts(torch, stream, max(3, args.steps // 4), 2, lambda: work.copy_(pristine),
                    lambda: graph.launch(stream))
    launches = hs.hs_launch_count() - launches0
    hs.hs_device_check(stream)
    batched = work.clone()
    d = batched[1:] >= batched[:-1]
    d[offs[1:-1] - 1] = True  # segment boundaries
    assert bool(d.all().item()), "batched output not sorted per segment"
    # Per-array plain launches: one hs_sort_i32 per segment, FIFO on one stream.
    work.copy_(pristine)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hs.hs_sort_i32_many(work, off, "merge", "6To8", stream=stream)
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0
    assert torch.equal(work, batched), "per-array result differs from batched result"
    graph.destroy()
    # The seeded prefix of the same size sequence that first reaches 2^28
    # keys (the total the workload's description names), same plan.
    kp = int(np.searchsorted(off, 1 << 28))
    np_keys = int(off[kp])
    pw, po = work[:np_keys], offs[:kp + 1]
    pgraph = hs.hs_segsort_capture(pw, po, plan)
    pms = time_sorts(torch, stream, max(3, args.steps // 4), 2,
                     lambda: pw.copy_(pristine[:np_keys]), lambda: pgraph.launch(stream))
    pgraph.destroy()
    assert torch.equal(pw, batched[:np_keys]), "prefix result differs from the full batch"
    del work, pristine, batched, offs, d, pw, po
    # Roofline bytes: one read and one write per key per pass, 1 + the merge
    # levels above the plan's tile for each segment (two-way merges).
    pd = plan.as_dict()
    leaf = max((k for k in range(3, 9) if (pd["netset"] >> k) & 1), default=1)
    tile = 256 * (4 * leaf - 1) if pd["block_threads"] == 256 else 512 * (2 * leaf - 1)
    sizes = np.diff(off)
    levels = np.where(sizes > tile, np.ceil(np.log2(np.maximum(sizes, 1) / tile)), 0)
    rbytes = float(np.sum(8.0 * sizes * (1 + levels)))
    peak, _ = measured_peak()
    return {"value": n / (ms / 1e3), "unit": "keys/s", "ms_per_batch": ms,
            "roofline_bytes": rbytes, "frac_of_measured": rbytes / (ms / 1e3) / (peak * 1e9),
            "plain_value": n / plain_s, "plain_s": plain_s,
            "speedup_vs_plain": plain_s / (ms / 1e3), "keys": int(n), "segments": 200_000,
            "plan": plan.as_dict(), "autotune_best_ms": tune_ms,
            "gpu_launches_per_batch": launches / (max(3, args.steps // 4) + 2),
            "prefix_2p28": {"segments": kp, "keys": np_keys, "ms_per_batch": pms,
                            "value": np_keys / (pms / 1e3), "unit": "keys/s"},
            "workload": "200,000 int32 arrays, sizes log-uniform in [3, 65536], "
                        "1/3 random, 1/3 sorted, 1/3 nearly sorted; CUDA-graph replay of "
                        "one persistent launch; plain = one hs_sort_i32 per array"}


def run_serving(hs, torch, dev, args):
    """Poisson arrivals of sort requests (sizes log-uniform in [8, 4194304],
    mixed distributions) into the continuous-batching server under an 8 GiB
    budget; p50/p99 latency at 0.5/0.8/0.95 of its measured capacity; then
    serial plain launches (one hs_sort_i32 at a time, FIFO) and the server
    both driven live by one arrival schedule at 0.8 of the serial capacity."""
    import numpy as np
    nreq = args.serve_requests
    seed = hs_inputs.config_seed(4)
    sizes = hs_inputs.log_uniform_sizes(nreq, seed, 8, 4194304)
    dists = hs_inputs.uniform_int(seed ^ 0x51, nreq, 0, 2)
    pool_n = 1 << 23
    pools = [torch.from_numpy(hs_inputs.keys(pool_n, d, seed + i)).to(dev)
             for i, d in enumerate(hs_inputs.DISTS)]
    starts = hs_inputs.uniform_int(seed ^ 0x52, nreq, 0, pool_n - 4194304)
    off = np.zeros(nreq + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    total = int(off[-1])
    arena = torch.empty(total, dtype=torch.int32, device=dev)
    for i in range(nreq):
        s0, n_i = int(starts[i]), int(sizes[i])
        arena[int(off[i]):int(off[i]) + n_i].copy_(pools[int(dists[i])][s0:s0 + n_i])
    del pools
    pristine = arena.clone()
    base = arena.data_ptr()
    ptrs = (base + 4 * off[:-1]).astype(np.uint64)
    srv = hs.Server(8 << 30)
    out = {"requests": nreq, "keys": total, "budget_bytes": 8 << 30,
           "workload": "Poisson arrivals, sizes log-uniform in [8, 4194304], mixed "
                       "random/sorted/nearly sorted, 8 GiB budget"}
    try:
        srv.replay(np.zeros(min(nreq, 500)), ptrs[:500], sizes[:500])  # warm-up
        arena.copy_(pristine)
        torch.cuda.synchronize(dev)
        lat, mk = srv.replay(np.zeros(nreq), ptrs, sizes)
        cap_req_s = nreq / mk
        out["capacity"] = {"keys_per_s": total / mk, "requests_per_s": cap_req_s,
                           "makespan_s": mk}
        for frac in (0.5, 0.8, 0.95):
            arena.copy_(pristine)
            torch.cuda.synchronize(dev)
            arr = hs_inputs.poisson_arrivals(nreq, frac * cap_req_s, seed ^ int(frac * 100))
            lat, mk = srv.replay(arr, ptrs, sizes)
            out[f"load_{int(frac * 100)}"] = {
                "rate_req_per_s": frac * cap_req_s, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e3, "sustained_keys_per_s": total / mk}
        out["server_stats"] = srv.stats()
    finally:
        srv.destroy()
    # Serial plain launches: one hs_sort_i32 call at a time, FIFO, each
    # synchronised before the next starts (the plain-launch serving loop).
    arena.copy_(pristine)
    ws = torch.empty(hs.hs_sort_workspace_bytes(4194304), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    L = hs.lib()
    mask = hs.netset_mask("6To8")
    ws_p, ws_b, st_p = ws.data_ptr(), ws.numel(), stream.cuda_stream

    def serial_replay(arrivals):
        """Live: request i starts at max(its arrival, the previous finish),
        runs alone and is waited for; returns (latencies, service times)."""
        lat_, svc = np.zeros(nreq), np.zeros(nreq)
        t_start = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t_start < arrivals[i]:
                pass
            t0 = time.perf_counter()
            hs._lib.check(L.hs_sort_i32(int(ptrs[i]), int(sizes[i]), 0, mask, ws_p, ws_b, st_p))
            stream.synchronize()
            t1 = time.perf_counter()
            svc[i] = t1 - t0
            lat_[i] = (t1 - t_start) - arrivals[i]
        return lat_, svc

    _, service = serial_replay(np.zeros(nreq))  # back to back: capacity
    serial_cap_req_s = nreq / service.sum()
    out["serial_plain"] = {"keys_per_s": total / service.sum(), "requests_per_s": serial_cap_req_s,
                           "mean_service_ms": float(service.mean()) * 1e3,
                           "driver": "Python loop of C-ABI calls, each waited for"}
    # One common offered rate both can sustain: 0.8 of the serial capacity.
    rate = 0.8 * serial_cap_req_s
    arr = hs_inputs.poisson_arrivals(nreq, rate, seed ^ 81)
    arena.copy_(pristine)
    torch.cuda.synchronize(dev)
    lat, _ = serial_replay(arr)
    out["serial_plain"]["at_common_rate"] = {
        "rate_req_per_s": rate, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
        "p99_ms": float(np.percentile(lat, 99)) * 1e3}
    srv = hs.Server(8 << 30)
    try:
        arena.copy_(pristine)
        torch.cuda.synchronize(dev)
        lat, mk = srv.replay(arr, ptrs, sizes)
        out["server_at_common_rate"] = {
            "rate_req_per_s": rate, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
            "p99_ms": float(np.percentile(lat, 99)) * 1e3, "sustained_keys_per_s": total / mk}
    finally:
        srv.destroy()
    del arena, pristine, ws
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
