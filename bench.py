"""Benchmark: factorizations/s on the single large query
g = (11,13,17,19,23,29), n = 3000 (|Z| = 72,082,790; 1.73 GB of int32 rows).

One step = the whole hot path over that query: fs_count (uint64 result, on a
second stream beside the enumeration) and fs_enumerate (all rows into a device
buffer), i.e. precompute, planner, slice walks, consumers, finalisation.
`value` = |Z| per step / device time per step (inputs resident, results left
on the device); `e2e` = the same through the synchronous C ABI (fs_count, and
fs_enumerate_host streaming the rows into pinned host memory) inside the timed
region.  The dominant kernel's roofline is the enumerate write walk against
the measured HBM copy bandwidth; inside the timed steps only that kernel is
bracketed by CUDA events, and the per-kernel breakdown and the launch count come
from the same number of identical steps run right after them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs the same query on its
own GPU (independent replicas: weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "single large query g=(11,13,17,19,23,29), n=3000: fs_count + fs_enumerate (int32 rows)"
METRIC = "factorizations/s (count & enumerate)"
FALLBACK_HBM_GBS = 6800.0


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def bench_config(Z: int, row_bytes: int) -> dict:
    """The `config` object both arms print for the bench workload."""
    return {"workload": WORKLOAD, "factorizations_per_step": Z, "output_bytes": Z * row_bytes,
            "l2": "flushed between steps (256 MB write)"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# the translation unit that defines each profiled kernel
KERNEL_SOURCE = {"pair_enum": "enum_fixed.cu", "pair_count": "pair.cu", "quad_count": "pair.cu"}


def strip_c_comments(src: str) -> str:
    """C/C++ source without comments (string and character literals kept) and
    with every run of whitespace reduced to one space."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_sha(kernel: str = "pair_enum") -> str:
    """Hash of the kernel's translation unit and every file it includes
    (quoted #include lines, followed recursively), comments and whitespace
    aside: a change anywhere in the code the kernel is compiled from changes
    it; host-only files and comments do not."""
    csrc = os.path.join(ROOT, "paper_2405_07989_gb300", "csrc")
    seen, todo = [], [os.path.join(csrc, KERNEL_SOURCE[kernel])]
    while todo:
        path = os.path.normpath(todo.pop())
        if path in seen:
            continue
        seen.append(path)
        with open(path) as f:
            for line in f:
                if line.startswith("#include \""):
                    todo.append(os.path.join(os.path.dirname(path), line.split('"')[1]))
    h = hashlib.sha256()
    for path in sorted(seen):
        with open(path) as f:
            h.update(os.path.relpath(path, ROOT).encode())
            h.update(strip_c_comments(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    e = rec.get(kernel)
    if not e or e.get("source_sha") != kernel_source_sha(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def recorded_instructions(kernel: str):
    """Warp instructions per pipe of one launch of `kernel` on the heavy count
    query, from a committed ncu summary, if it was taken on the current kernel
    sources; else None."""
    p = os.path.join(ROOT, "profiles", "count_inst.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    e = rec.get(kernel)
    if not e or e.get("source_sha") != kernel_source_sha(kernel):
        return None
    return e


def numa_placement(index: int) -> dict:
    """The host's NUMA nodes and the GPU's node (from sysfs), for the pinned
    buffer's placement; empty where sysfs does not say."""
    out = {}
    base = "/sys/devices/system/node"
    if os.path.isdir(base):
        out["host_nodes"] = sorted(x for x in os.listdir(base) if x.startswith("node") and x[4:].isdigit())
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().lower()
        for cand in (bus, bus[-12:]):
            p = f"/sys/bus/pci/devices/{cand}/numa_node"
            if cand and os.path.exists(p):
                out["gpu_node"] = int(open(p).read().strip())
                break
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest x over all ranks (the job takes as long as its slowest
    replica); x itself when there is one rank."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: int, ws: int, ms: float) -> float:
    """Whole-job throughput of ws independent replicas that each process
    units_per_rank units, given the max-over-ranks time in ms."""
    return ws * units_per_rank / (ms / 1000.0)


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def _oracle_task(args):
    n, wg, lo, hi = args
    import oracle
    rows, _ = oracle.enumerate_range(n, wg, lo, hi)
    return int(rows.shape[0])


def cpu_oracle_run(pool, n, wg, budget_s: float = 30.0):
    """The oracle's bounded stream (save consumer) over the whole query, cut
    by the leading coordinate a_1 into independent slices run on all host
    cores.  Returns (factorizations, seconds, slices_done, slices_total)."""
    d = len(wg)
    top = n // wg[0]
    tasks = []
    for x in range(top + 1):
        lo = [x] + [0] * (d - 1)
        hi = [x + 1] + [0] * (d - 1) if x < top else None
        tasks.append((n, wg, lo, hi))
    # heaviest slices (small a_1) first
    t0 = time.perf_counter()
    total = 0
    done = 0
    for c in pool.imap_unordered(_oracle_task, tasks, chunksize=1):
        total += c
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return total, dt, done, len(tasks)


def cpu_single_thread(n, wg, budget_s: float = 4.0):
    """The oracle's bounded stream on one host thread over leading-coordinate
    slices, lightest first, until the budget is spent: (factorizations,
    seconds, slices).  And the exact count by the oracle's DP (not the
    method: a coefficient of prod 1 / (1 - x^g_i)), timed alone."""
    import oracle
    d = len(wg)
    top = n // wg[0]
    t0 = time.perf_counter()
    total = done = 0
    for x in range(top, -1, -1):
        lo = [x] + [0] * (d - 1)
        hi = [x + 1] + [0] * (d - 1) if x < top else None
        rows, _ = oracle.enumerate_range(n, wg, lo, hi)
        total += int(rows.shape[0])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.count_dp(n, wg)
    dp_s = time.perf_counter() - t1
    return total, dt, done, dp_s


def make_pool():
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2405_07989_gb300 import workloads
    n, g = workloads.CONFIG2
    wg = sorted(g, reverse=True)
    pool, cores = make_pool()
    try:
        for _ in range(args.warmup):
            cpu_oracle_run(pool, n, wg)
        times, tot = [], 0
        for _ in range(args.steps):
            c, dt, done, ntask = cpu_oracle_run(pool, n, wg)
            times.append(dt)
            tot = c
    finally:
        pool.close()
        pool.join()
    ms = 1000.0 * sum(times) / len(times)
    value = tot / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "factorizations/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": bench_config(tot, 4 * len(g)),
        "cpu_baseline": {"value": value, "unit": "factorizations/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"whole query per step: oracle bounded streams (Algorithm 3.1,"
                                   f" save consumer) over {ntask} leading-coordinate slices"},
        "e2e": {"value": value, "unit": "factorizations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    ws, rank, local = dist_setup()
    pool = cores = None
    if ws == 1 and not args.no_cpu_baseline:
        pool, cores = make_pool()  # before the first GPU call
    import torch
    import torch.distributed as dist
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2405_07989_gb300 as fs
    from paper_2405_07989_gb300 import workloads
    fs.lib()

    n, g = workloads.CONFIG2
    d = len(g)
    Z = fs.fs_count(n, g)
    row_bytes = d * 4
    out = torch.empty(Z * d, dtype=torch.int32, device=dev)
    dc = torch.zeros(2, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the count and the enumeration are independent: the count runs on a
    # second stream (each stream has its own library scratch) beside the
    # enumeration's kernels; the step ends when both have finished
    s_count = torch.cuda.Stream(dev)

    def step():
        s_count.wait_stream(stream)
        fs.fs_count_async(n, g, dc[0:1], stream=s_count.cuda_stream)
        fs.fs_enumerate_async(n, g, out, Z, dc[1:2])
        stream.wait_stream(s_count)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert int(dc[0]) == Z and int(dc[1]) == Z, (int(dc[0]), int(dc[1]), Z)
    # host time to enqueue one step (the GPU idles between short kernels when
    # this exceeds their device time)
    t0 = time.perf_counter()
    for _ in range(5):
        step()
    host_ms = (time.perf_counter() - t0) / 5 * 1000.0
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (untimed) ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    fs.fs_profile_read()
    # inside the timed steps only the write walk is bracketed by events (its
    # duration for the roofline); every other kernel runs without
    fs.fs_profile_only("pair_enum")
    fs.fs_profile_enable(True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    fs.fs_profile_enable(False)
    fs.fs_profile_only(None)
    prof = fs.fs_profile_read()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(sum(ms_steps) / len(ms_steps), ws, dev)
    assert int(dc[0]) == Z and int(dc[1]) == Z
    value = replica_value(Z, ws, ms)
    # every kernel of a step, timed and counted in the same number of identical
    # steps right after the timed ones (events on every kernel lengthen a step)
    fs.fs_profile_enable(True)
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        step()
    torch.cuda.synchronize()
    fs.fs_profile_enable(False)
    prof_all = fs.fs_profile_read()
    launches_per_step = sum(v[0] for v in prof_all.values()) // args.steps

    # ---- roofline of the dominant kernel (enumerate write walk) ----
    peaks, peak_src = measured_peaks()
    enum_launches, enum_ms = prof.get("pair_enum", (0, 0.0))
    enum_avg = enum_ms / max(enum_launches, 1)
    alg_bytes = Z * row_bytes
    achieved = alg_bytes / (enum_avg / 1000.0) / 1e9
    peak = float(peaks["hbm_gbs"])
    roofline = {"bound": "hbm", "kernel": "pair_enum", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                "traffic": recorded_traffic("pair_enum"),
                "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": enum_avg}
    breakdown = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
                 for k, v in prof_all.items()}

    # ---- end to end through the synchronous C ABI: the count, and the rows
    # streamed into pinned host memory (fs_enumerate_host: each window's walk
    # overlaps the device-to-host copy of the previous one) ----
    host = torch.empty(Z * d, dtype=torch.int32, pin_memory=True)
    with fs.Cursor(n, g) as cur:
        S_enum = cur.slices()
    e2e_steps = max(2, min(args.steps, 5))
    c2 = fs.fs_enumerate_host(n, g, host, Z)  # warm-up (staging buffers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c1 = fs.fs_count(n, g)
        c2 = fs.fs_enumerate_host(n, g, host, Z)
        assert c1 == Z and c2 == Z
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws, dev)
    assert torch.equal(host.view(-1, d)[:4].to(dev), out.view(-1, d)[:4])
    # the link's own ceiling: one plain device-to-host copy of the same bytes
    # into the same pinned buffer, event-timed
    host.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    link = []
    for _ in range(7):
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record()
        host.copy_(out, non_blocking=True)
        l1.record()
        torch.cuda.synchronize()
        link.append(Z * row_bytes / (l0.elapsed_time(l1) / 1000.0) / 1e9)
    link.sort()
    link_gbs = link[-1]
    e2e = {"value": replica_value(Z, ws, e2e_s * 1000.0), "unit": "factorizations/s",
           "h2d_bytes_per_step": 2 * d * 4,
           # rows, three counter reads (128 B each) and the slice offsets
           "d2h_bytes_per_step": Z * row_bytes + 3 * 128 + 8 * (S_enum + 1),
           "ms_per_step": e2e_s * 1000.0,
           "path": "fs_count + fs_enumerate_host into pinned host memory",
           "d2h_link_ceiling_gbs": link_gbs,
           "d2h_link_median_gbs": link[len(link) // 2],
           "link_frac": (Z * row_bytes / e2e_s / 1e9) / link_gbs,
           "link_note": ("plain cudaMemcpyAsync of the same bytes into the same pinned buffer, "
                         "best and median of 7"),
           "numa": numa_placement(local)}

    # ---- extras: the integer-bound count walk on the heavy count-only query ----
    extras = None
    if not args.no_extras:
        extras = heavy_count_extras(fs, workloads, dev)
        # the integer-bound count kernel's roofline beside the dominant kernel's
        roofline["count"] = extras["count_roofline"]
        roofline["count_quad"] = extras["count_quad_roofline"]
        extras["batched"] = batch_extras(fs, workloads, dev)
        extras["serving"] = serving_extras(fs, workloads, args.serve_rate, args.serve_requests)
        # capacity: the same requests all at once (no arrival pacing)
        extras["serving_saturated"] = serving_extras(fs, workloads, 1e9, args.serve_requests)
        # the same without the histograms (count and length range only)
        extras["serving_saturated_no_hist"] = serving_extras(fs, workloads, 1e9, args.serve_requests,
                                                             hist=False)
        extras["table1_context"] = table1_extras(fs, dev)
        extras["methods"] = method_extras(fs, workloads, dev)

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1) ----
    cpu = None
    if pool is not None:
        wg = sorted(g, reverse=True)
        c, dt, done, ntask = cpu_oracle_run(pool, n, wg)
        pool.close()
        pool.join()
        c1, dt1, done1, dp_s = cpu_single_thread(n, wg)
        cpu = {"value": c / dt, "unit": "factorizations/s", "cores": cores, "kind": "oracle",
               "sample": (f"{done}/{ntask} leading-coordinate slices of the same query "
                          f"({c} factorizations): oracle bounded streams, Algorithm 3.1, save "
                          f"consumer, one slice per process ({cores} spawn processes)"),
               "single_thread": {"value": c1 / dt1, "unit": "factorizations/s", "cores": 1,
                                 "sample": f"{done1} leading-coordinate slices ({c1} factorizations)"},
               "dp_count_seconds": dp_s,
               "dp_note": "exact |Z| by the oracle's DP, one thread: not the method"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "factorizations/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": bench_config(Z, row_bytes),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "gpu_launches_per_step": launches_per_step,
            "clocks": clk, "breakdown": breakdown, "host_enqueue_ms_per_step": host_ms,
            "extras": extras,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


# Integer operations of the PAIR count's closed form at one visited leaf:
# quotient by the lcm (multiply-high, shift), remainder (multiply-subtract),
# the class bit's index, its load, its extraction (shift, mask), and the add.
COUNT_OPS_PER_LEAF = 8


def visited_leaves(fs, n, gens) -> int:
    """The leaves the PAIR count walk resolves, exactly: a leaf (a prefix of
    the first d-2 generators in descending order, residual r = n - phi) is
    visited iff G = gcd of the last two generators divides r (common-divisor
    skipping), i.e. iff phi + t G = n for some t >= 0.  So their number is the
    factorization count of n over the first d-2 generators and G."""
    w = sorted(gens, reverse=True)
    if len(w) < 3:
        return 0
    return fs.fs_count(n, w[:-2] + [math.gcd(w[-1], w[-2])])


# Integer operations of the trailing-four count at one leaf: the table entry's
# address, its load, and the add.
QUAD_OPS_PER_LEAF = 3


def quad_leaves(fs, n, gens) -> int:
    """The leaves of the trailing-four (QUAD) count walk, exactly: prefixes of
    the first d-4 generators (descending) with phi <= n, i.e. the
    factorizations of n over those generators and a slack generator 1."""
    w = sorted(gens, reverse=True)
    return fs.fs_count(n, w[:-4] + [1]) if len(w) >= 5 else 0


def count_roofline(fs, n, g, walk_ms, rates, key="pair_count"):
    """A count walk against the probed 32-bit add rate (128 lanes per clock
    per SM: the ALU and FMA pipes together).  `frac` is its integer-pipe
    issue: the ALU- and FMA-pipe warp instructions of one launch, counted by
    ncu on the same kernel sources at this size (profiles/count_inst.json),
    x 32 lanes / the walk's event-timed duration here.  `useful_frac` counts
    only the closed form's operations per leaf it resolves (PAIR: the visited
    leaves, COUNT_OPS_PER_LEAF each; QUAD: every leaf, QUAD_OPS_PER_LEAF)."""
    if key == "pair_count":
        units, ops, kernel = visited_leaves(fs, n, g), COUNT_OPS_PER_LEAF, "k_pair_count"
    else:
        units, ops, kernel = quad_leaves(fs, n, g), QUAD_OPS_PER_LEAF, "k_triple_walk (QUAD)"
    peak = rates["add"]
    useful = units * ops / (walk_ms / 1000.0)
    rec = recorded_instructions(key)
    out = {"bound": "alu", "kernel": kernel, "workload": f"g={tuple(g)}, n={n}",
           "unit": "int32 lane-ops/s", "peak": peak, "peak_source": "probed add rate (fs_probe_int_rate)",
           "avg_launch_ms": walk_ms, "leaves_resolved": units,
           "useful_ops_per_leaf": ops, "useful_frac": useful / peak,
           "achieved": None, "frac": None}
    if rec and rec.get("n") == n and list(rec.get("gens", [])) == list(g):
        ints = rec["alu_warp_inst"] + rec["fma_warp_inst"]
        ach = ints * 32 / (walk_ms / 1000.0)
        out.update({"achieved": ach, "frac": ach / peak, "int_warp_inst_per_launch": ints,
                    "warp_inst_per_launch": rec["warp_inst"],
                    "warp_inst_per_leaf": rec["warp_inst"] / units if units else None,
                    "inst_source": "ncu counters of the same kernel sources, profiles/count_inst.json"})
    return out


def heavy_count_extras(fs, workloads, dev):
    """Count and length statistics of the count-only heavy query (8 generators
    from seed 0, n = 40000, 7.66e12 factorizations), event-timed, with the
    count walk's integer roofline against the probed add rate; the counts of
    the same draw at seeds 1 and 2 beside it."""
    import torch
    n, g = workloads.config3(0)
    rates = {name: fs.fs_probe_int_rate(k, 2048) for k, name in ((0, "add"), (1, "lop3"),
                                                                  (2, "mad"))}
    pair = fs.make_config(method=fs.METHOD_PAIR)
    _, _, leaves = fs.fs_plan(n, g, 1, pair)
    dc = torch.zeros(1, dtype=torch.int64, device=dev)

    def timed_count(cfg, walk, n=n, g=g):
        fs.fs_count_async(n, g, dc, cfg)
        torch.cuda.synchronize()
        fs.fs_profile_read()
        fs.fs_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fs.fs_count_async(n, g, dc, cfg)
        e1.record()
        torch.cuda.synchronize()
        fs.fs_profile_enable(False)
        prof = fs.fs_profile_read()
        ms = e0.elapsed_time(e1)
        return int(dc[0].item()), ms, prof.get(walk, (1, ms))[1], prof

    Z, ms, walk_ms, _ = timed_count(pair, "pair_count")
    Z3, ms3, walk3, prof3 = timed_count(fs.make_config(method=fs.METHOD_TRIPLE), "triple_count")
    Z4, ms4, walk4, prof4 = timed_count(None, "quad_count")
    assert Z3 == Z and Z4 == Z
    roof = count_roofline(fs, n, g, walk_ms, rates)
    roof_quad = count_roofline(fs, n, g, walk4, rates, key="quad_count")
    hist = torch.zeros(n // min(g) + 1, dtype=torch.int64, device=dev)
    fs.fs_length_stats(n, g, hist)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cnt, mn, mx = fs.fs_length_stats(n, g, hist)
    len_s = time.perf_counter() - t0
    assert cnt == Z
    t0 = time.perf_counter()
    assert fs.fs_length_stats(n, g, None) == (cnt, mn, mx)
    len_minmax_s = time.perf_counter() - t0
    # the same draw at seeds 1 and 2: every walk, the same count
    seeds = {}
    for seed in (1, 2):
        ns, gs = workloads.config3(seed)
        _, _, lv = fs.fs_plan(ns, gs, 1, pair)
        zs, mss, wms, _ = timed_count(pair, "pair_count", ns, gs)
        z3, ms3s, _, _ = timed_count(fs.make_config(method=fs.METHOD_TRIPLE), "triple_count", ns, gs)
        z4, ms4s, _, _ = timed_count(None, "quad_count", ns, gs)
        assert z3 == zs and z4 == zs
        vs = visited_leaves(fs, ns, gs)
        seeds[str(seed)] = {"gens": list(gs), "n": ns, "factorizations": zs, "leaves": lv,
                            "leaves_visited": vs,
                            "count_ms": mss, "count_leaves_per_s": lv / (wms / 1000.0),
                            "count_useful_frac": vs * COUNT_OPS_PER_LEAF / (wms / 1000.0) / rates["add"],
                            "count_triple_ms": ms3s, "count_quad_ms": ms4s}
    return {
        "workload": f"count-only heavy query g={tuple(g)}, n={n}",
        "factorizations": Z, "leaves": leaves, "leaves_visited": roof["leaves_resolved"],
        "count_ms": ms, "count_walk_ms": walk_ms,
        "count_factorizations_per_s": Z / (ms / 1000.0), "count_leaves_per_s": leaves / (walk_ms / 1000.0),
        "count_triple_ms": ms3, "count_triple_walk_ms": walk3,
        "count_triple_factorizations_per_s": Z / (ms3 / 1000.0),
        "count_triple_breakdown_ms": {k: v[1] for k, v in prof3.items()},
        "count_quad_ms": ms4, "count_quad_walk_ms": walk4,
        "count_quad_factorizations_per_s": Z / (ms4 / 1000.0),
        "count_quad_breakdown_ms": {k: v[1] for k, v in prof4.items()},
        "count_roofline": roof,
        "count_quad_roofline": roof_quad,
        "int_rates": rates,
        "length_stats_s": len_s, "length_min_max": [mn, mx],
        "length_factorizations_per_s": Z / len_s,
        "length_stats_vs_count": len_s / (walk_ms / 1000.0),
        "length_min_max_only_s": len_minmax_s,
        "other_seeds": seeds,
    }


# The largest Table 1 cell per d, with the paper's best CUDA time (seconds,
# RTX 3080 + Ryzen 3900X, whole-second resolution): context, not a target.
TABLE1_CONTEXT = [(3, (13, 37, 38), 500000, 52), (4, (13, 37, 38, 40), 45000, 132),
                  (5, (13, 37, 38, 40, 41), 9000, 131), (6, (13, 37, 38, 40, 41, 42), 3000, 335),
                  (7, (13, 37, 38, 40, 41, 42, 43), 2000, 760)]


def table1_extras(fs, dev):
    """Materialise Z(n) for the largest Table 1 input of each d through the
    synchronous C ABI (count, then enumerate into device memory), wall-clock
    timed, beside the paper's own runtime for the same input."""
    import torch
    out = []
    for d, g, n, paper_s in TABLE1_CONTEXT:
        Z = fs.fs_count(n, g)
        buf = torch.empty(max(Z, 1) * d, dtype=torch.int32, device=dev)
        fs.fs_enumerate(n, g, buf, Z)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = fs.fs_count(n, g)
        c2 = fs.fs_enumerate(n, g, buf, Z)
        dt = time.perf_counter() - t0
        assert c == Z and c2 == Z
        out.append({"d": d, "n": n, "factorizations": Z, "seconds": dt,
                    "paper_seconds_rtx3080": paper_s})
        del buf
    return out


def method_extras(fs, workloads, dev):
    """The single large query through the other walks, event-timed on the
    device: the paper's Algorithm 3.1 step by step (PLAIN) for count and
    enumerate, the PAIR count, and the predicate consumer (fs_any) with a
    predicate no factorization satisfies (a full walk) and one the first
    leaves satisfy (early exit)."""
    import torch
    n, g = workloads.CONFIG2
    d = len(g)
    Z = fs.fs_count(n, g)
    out = torch.empty(Z * d, dtype=torch.int32, device=dev)
    dc = torch.zeros(1, dtype=torch.int64, device=dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    plain = fs.make_config(method=fs.METHOD_PLAIN)
    pair = fs.make_config(method=fs.METHOD_PAIR)
    res = {"workload": f"g={tuple(g)}, n={n}: {Z} factorizations"}
    res["plain_count_ms"] = timed(lambda: fs.fs_count_async(n, g, dc, plain))
    assert int(dc[0]) == Z
    res["plain_enumerate_ms"] = timed(lambda: fs.fs_enumerate_async(n, g, out, Z, dc, cfg=plain), 2)
    assert int(dc[0]) == Z
    res["pair_count_ms"] = timed(lambda: fs.fs_count_async(n, g, dc, pair))
    assert int(dc[0]) == Z
    res["quad_count_ms"] = timed(lambda: fs.fs_count_async(n, g, dc))
    # sum of a_i = -1 never holds: every leaf is visited
    t0 = time.perf_counter()
    assert not fs.fs_any(n, g, [1] * d, -1)
    res["any_false_ms"] = (time.perf_counter() - t0) * 1000.0
    t0 = time.perf_counter()
    assert fs.fs_any(n, g, [0] * d, 0)
    res["any_true_ms"] = (time.perf_counter() - t0) * 1000.0
    res["plain_enumerate_factorizations_per_s"] = Z / (res["plain_enumerate_ms"] / 1000.0)
    return res


def batch_extras(fs, workloads, dev):
    """The batched workload (4096 seeded queries, d in [3, 8], generators in
    [5, 100], n in [100, 5000]): one persistent launch per batch, autotuned,
    against one single-query call per query, at equal exact counts."""
    import torch
    qs = workloads.config4(0)
    out = {"workload": "4096 batched queries, d in [3,8], distinct gens in [5,100], n in [100,5000] (seed 0)"}
    reps = 5
    counts = None
    for mode, name in ((fs.BATCH_COUNT, "count"), (fs.BATCH_LENGTHS, "lengths")):
        best, tune_ms = fs.fs_batch_autotune(qs, mode)
        with fs.Batch(qs, mode, best) as b:
            b.launch()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.launch()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res = b.results()
        if counts is None:
            counts = [r[0] for r in res]
        assert [r[0] for r in res] == counts
        out[f"persistent_{name}_ms"] = ms
        out[f"persistent_{name}_queries_per_s"] = len(qs) / (ms / 1000.0)
        out[f"autotuned_{name}"] = {"block_threads": best.block_threads,
                                    "blocks_per_sm": best.blocks_per_sm, "items": best.slices}
    out["factorizations"] = sum(counts)
    dcs = torch.zeros(len(qs), dtype=torch.int64, device=dev)
    for i, (n, g) in enumerate(qs):  # warm-up of the per-query path
        fs.fs_count_async(n, g, dcs[i:i + 1])
    torch.cuda.synchronize()
    dcs.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i, (n, g) in enumerate(qs):
        fs.fs_count_async(n, g, dcs[i:i + 1])
    e1.record()
    torch.cuda.synchronize()
    per_ms = e0.elapsed_time(e1)
    assert [int(x) for x in dcs.tolist()] == counts  # equal exact results
    out["per_query_count_ms"] = per_ms
    out["per_query_queries_per_s"] = len(qs) / (per_ms / 1000.0)
    out["persistent_speedup_count"] = per_ms / out["persistent_count_ms"]
    return out


def serving_stages(rs):
    """Per-stage durations (seconds) of served responses: queue (submit to
    launch), batch (batch launch to its results), direct_job (a count / length
    request run as a job from the start, t_start = t_job: launch to results),
    job_wait and job (an enumerate or histogram after its batch), answer (results
    to the response, requests without a job after the batch)."""
    ran = [r for r in rs if r["t_start"] > 0]
    direct_t = {r["ticket"] for r in ran if r["t_job"] > 0 and r["t_start"] == r["t_job"]}
    direct = [r for r in ran if r["ticket"] in direct_t]
    batched = [r for r in ran if r["ticket"] not in direct_t]
    jobs = [r for r in batched if r["t_job"] > 0]
    return {"queue": [r["t_start"] - r["t_submit"] for r in ran],
            "batch": [r["t_counted"] - r["t_start"] for r in batched],
            "direct_job": [r["t_counted"] - r["t_start"] for r in direct],
            "job_wait": [r["t_job"] - r["t_counted"] for r in jobs],
            "job": [r["t_done"] - r["t_job"] for r in jobs],
            "answer": [r["t_done"] - r["t_counted"] for r in ran
                       if r["t_job"] == 0 or r["ticket"] in direct_t]}


def serving_extras(fs, workloads, rate: float, nreq: int, hist: bool = True):
    """The serving workload: Poisson arrivals of queries drawn like the batched
    ones with n up to 20000, 80 % count / 15 % length statistics (with the
    length histogram) / 5 % enumerate (int16 rows), through the
    continuous-batching request loop; a client thread releases rows and
    histograms as soon as they are polled.  Per stage: queue (submit to batch
    launch), batch (launch to results), job wait and job (enumerate rows or
    histogram), answer (results to completion for requests without a job)."""
    import threading
    reqs = workloads.config5(0, nreq, rate, 20000)
    budget = 32 << 30
    scfg = dict(mem_budget_bytes=budget, table_bytes=1 << 30, max_batch=512, slots=3,
                window_us=200, job_streams=4)
    srv = fs.Server(**scfg)

    def job_of(r):
        return r["status"] == fs.FS_OK and r["rows"] != 0

    try:
        warm = [srv.submit(op, n, g, hist=hist and op == fs.REQ_LENGTHS) for (_, op, n, g) in reqs[:16]]
        seen = 0
        while seen < len(warm):
            for r in srv.poll(64, wait_ms=50):
                seen += 1
                if job_of(r):
                    srv.release(r["ticket"])
        done = {}

        def poller():
            while len(done) < nreq:
                for r in srv.poll(1024, wait_ms=20):
                    done[r["ticket"]] = r
                    if job_of(r):
                        srv.release(r["ticket"])

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for (ta, op, n, g) in reqs:
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            srv.submit(op, n, g, elem_bytes=2, hist=hist and op == fs.REQ_LENGTHS)
        th.join()
    finally:
        srv.close()
    rs = list(done.values())
    lat = np.array([r["t_done"] - r["t_submit"] for r in rs]) * 1000.0
    span = max(r["t_done"] for r in rs) - min(r["t_submit"] for r in rs)

    def pct(v):
        v = np.asarray(v) * 1000.0
        return {"n": int(v.size), "p50_ms": float(np.percentile(v, 50)),
                "p99_ms": float(np.percentile(v, 99))} if v.size else {"n": 0}

    by_op = {}
    for op, name in ((fs.REQ_COUNT, "count"), (fs.REQ_LENGTHS, "lengths"),
                     (fs.REQ_ENUMERATE, "enumerate")):
        by_op[name] = pct([r["t_done"] - r["t_submit"] for r in rs if r["op"] == op])
    stages = {k: pct(v) for k, v in serving_stages(rs).items()}
    status = {}
    for r in rs:
        status[fs.status_name(r["status"])] = status.get(fs.status_name(r["status"]), 0) + 1
    return {
        "workload": (f"{nreq} requests, Poisson arrivals at {rate:g}/s, d in [3,8], gens in "
                     f"[5,100], n in [100,20000], 80/15/5 % count/lengths{'+histogram' if hist else ''}"
                     f"/enumerate (int16), seed 0"),
        "server": scfg,
        "queries_per_s": nreq / span, "span_s": span,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "by_op": by_op, "stages": stages, "status": status,
        "histograms": sum(1 for r in rs if r["op"] == fs.REQ_LENGTHS and job_of(r)),
        "factorizations_served": int(sum(r["count"] for r in rs if r["status"] == fs.FS_OK)),
        # the size distribution of the requests' sets |Z| beside the latencies
        "set_size": {q: float(np.percentile([r["count"] for r in rs], p))
                     for q, p in (("p50", 50), ("p90", 90), ("p99", 99), ("max", 100))},
    }


def run_profile_case(args):
    """Small cases of the same kernels for ncu captures, a few calls each:
    "enum": the single-large-query generators at a smaller n (output still
    larger than L2); "count" / "count_triple" / "count_quad": the heavy
    count-only query's generators at --profile-n through the PAIR walk or the
    trailing-three / trailing-four tables; "lengths": the same generators'
    count, length range and histogram (PAIR walk); "batch5": the first
    --profile-n queries of the serving workload in one batch (--profile-mode);
    "batch": the first --profile-n
    queries of the batched workload, count mode."""
    import torch
    import paper_2405_07989_gb300 as fs
    from paper_2405_07989_gb300 import workloads
    if args.profile_case in ("batch", "batch5"):
        if args.profile_case == "batch":
            qs = workloads.config4(0, nq=args.profile_n)
        else:
            qs = [(n, g) for (_, op, n, g) in workloads.config5(0, args.profile_n, 1000.0, 20000)]
        mode = fs.BATCH_LENGTHS if args.profile_mode == "lengths" else fs.BATCH_COUNT
        with fs.Batch(qs, mode) as b:
            for _ in range(args.steps):
                b.launch()
            res = b.results()
        print(json.dumps({"profile_case": {"queries": len(qs), "calls": args.steps,
                                           "factorizations": sum(r[0] for r in res)}}))
        return 0
    walk = {"auto": fs.WALK_AUTO, "packed": fs.WALK_PACKED, "lanes": fs.WALK_LANES}[args.profile_walk]
    if args.profile_case == "lengths":
        n, g = workloads.config3(0, n=args.profile_n)
        hist = torch.zeros(n // min(g) + 1, dtype=torch.int64, device="cuda")
        for _ in range(args.steps):
            res = fs.fs_length_stats(n, g, hist, fs.make_config(walk=walk))
        print(json.dumps({"profile_case": {"n": n, "gens": list(g), "count": res[0],
                                           "min_max": list(res[1:]), "calls": args.steps}}))
        return 0
    if args.profile_case in ("count", "count_triple", "count_quad"):
        n, g = workloads.config3(0, n=args.profile_n)
        dc = torch.zeros(1, dtype=torch.int64, device="cuda")
        cfg = fs.make_config(method={"count": fs.METHOD_PAIR, "count_triple": fs.METHOD_TRIPLE,
                                     "count_quad": fs.METHOD_QUAD}[args.profile_case], walk=walk)
        for _ in range(args.steps):
            fs.fs_count_async(n, g, dc, cfg)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": {"n": n, "gens": list(g), "count": int(dc[0]),
                                           "calls": args.steps}}))
        return 0
    _, g = workloads.CONFIG2
    n = args.profile_n
    d = len(g)
    Z = fs.fs_count(n, g)
    out = torch.empty(Z * d, dtype=torch.int32, device="cuda")
    dc = torch.zeros(2, dtype=torch.int64, device="cuda")
    for _ in range(args.steps):
        fs.fs_count_async(n, g, dc[0:1])
        fs.fs_enumerate_async(n, g, out, Z, dc[1:2])
    torch.cuda.synchronize()
    assert int(dc[0]) == Z and int(dc[1]) == Z
    print(json.dumps({"profile_case": {"n": n, "gens": list(g), "rows": Z,
                                       "bytes": Z * d * 4, "calls": args.steps}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the heavy count-only query measurements")
    ap.add_argument("--profile-case",
                    choices=["enum", "count", "count_triple", "count_quad", "lengths", "batch",
                             "batch5"],
                    default=None,
                    help="run only a small case of the same kernels (for ncu)")
    ap.add_argument("--profile-n", type=int, default=2000)
    ap.add_argument("--profile-walk", choices=["auto", "packed", "lanes"], default="auto",
                    help="profile cases: how the order-free walks take a sibling group")
    ap.add_argument("--profile-mode", choices=["count", "lengths"], default="count",
                    help="batch profile cases: count only, or count and length range")
    ap.add_argument("--serve-rate", type=float, default=1000.0,
                    help="serving extras: Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
