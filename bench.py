#!/usr/bin/env python3
"""Benchmark of the GB300 Powersort hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Workloads (keys are uint32, the stable
permutation is produced):

  hbm_2^28     (default) one step = one single-instance sort of n = 2^28
               uniform (seed 2), the largest single-instance size.  Unless
               --no-extras is given, the line also carries the metric's two
               other parts, each measured in the same run: "batched_vs_plain"
               (the batched_4096 workload below: one graph replay against a
               loop of single-instance calls) and "serving" (the serving
               workload below: p50 / p99 latency and sustained elements/s)
  plain_2^24   one step = three single-instance sorts of n = 2^24:
               uniform, Zipf(1.1) over 2^20 values, presorted Geometric(mean
               2^10) runs (seed 1)
  uniform_2^26 one step = one sort of n = 2^26 uniform (seed 2): the 2^28
               workload at a size that ncu captures quickly (profiling only)
  updown_2^24  one step = one sort of n = 2^24 Geometric(mean 2^10) segments,
               each sorted ascending or descending by a coin (seed 1), with
               the decreasing-run variant of Sec. 5 (PS_FLAG_DESCENDING_RUNS);
               the line also carries the rate of the plain rule on the same
               input
  records_2^23 one step = two record sorts of n = 2^23 rows of 30 words
               (randomBlob30 and zeroBlob30, the paper's blob types, values in
               [100, 10^9], seed 1) with the sorted rows written out; rate in
               records/s
  keys64_2^24  one step = three 64-bit key sorts of n = 2^24 (ps_sort_keys64):
               uniform unsigned, int64 within +-2^31 (two tie groups of n/2 on
               the high word), uniform float64 bit patterns (seed 1)
  bands_2^24   one step = one sort of n = 2^24: sorted blocks of 2^13 keys in
               descending value bands; with --storage vm the merges splice
               whole pages through the page table (stats: pages_spliced)
  serving      a Poisson stream of 2000 requests/s for 10 s (sizes log-uniform
               in [2^10, 2^24], seed 4) through the continuous-batching server
               under a 64 GB device-memory budget; reports sustained elements/s
               and p50/p99 latency (--steps/--warmup are not used)
  batched_4096 one step = one replay of a captured CUDA graph sorting 4096
               independent instances with sizes log-uniform in [2^8, 2^20)
               (seed 3, uniform keys), tile size and merge occupancy picked by
               the autotuner; compared with a loop of single-instance calls

Timing: inputs are resident in HBM before the timed region; before every
timed sort the input is restored from a pristine copy and L2 is flushed by
writing a 512 MiB buffer (both untimed); each sort is bracketed by CUDA
events on the library's stream, and the per-phase kernel times come from
events the library records between its launches.  ``e2e`` repeats the
workload from pinned host arrays, with the host->device copy of the keys and
the device->host copy of keys and permutation inside the timed region: with
Pingpong storage as a stream of requests through the server (two lanes, so
one sort's copies overlap another's kernels), the one-call ps_run_host
figure beside it; with VM storage through ps_run_host.  ``cpu_baseline`` / ``--impl reference`` time the single-threaded CPU
oracle on a bounded sample of the same workload.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "hot-path elements/s & % HBM roofline, 1xGB300; batched vs plain; p50/p99 ms"
UNIT = "elements/s"
WORKLOADS = {
    "plain_2^24": [("uniform", 1 << 24, 1), ("zipf", 1 << 24, 1), ("runs", 1 << 24, 1)],
    "hbm_2^28": [("uniform", 1 << 28, 2)],
    "uniform_2^26": [("uniform", 1 << 26, 2)],
    "updown_2^24": [("updown", 1 << 24, 1)],
    "bands_2^24": [("bands", 1 << 24, 1)],
    "records_2^23": None,
    "keys64_2^24": None,
    "batched_4096": None,
    "serving": None,
}
DESCENDING_WORKLOADS = {"updown_2^24"}   # sorted with the decreasing-run variant
FLUSH_BYTES = 512 << 20
BYTES_PER_MERGED_ELEM = 16   # key + perm entry read, key + perm entry written
LAUNCHES_PER_BATCH = 11      # one batched Pingpong call: setup, 2 run detection, 5 planning, tiles, merges, finish


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="hbm_2^28", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="pingpong", choices=["pingpong", "vm"],
                    help="run storage of the plain workloads: Pingpong (n-element scratch) or VM pages")
    ap.add_argument("--page-log2", type=int, default=0,
                    help="VM storage: page size 2^k elements (0: the library's default)")
    ap.add_argument("--key-type", default="u32", choices=["u32", "i32", "f32"],
                    help="plain workloads: order the same 32-bit patterns as unsigned, signed or float keys")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="hbm_2^28: leave out the batched and serving sub-measurements")
    ap.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    ap.add_argument("--lane-total", type=int, default=1 << 25,
                    help="serving: most elements one batch of a lane may hold")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_inputs(workload):
    from paper_2605_27147_gb300 import inputs

    return [(d, n, s, inputs.make(d, n, s)) for d, n, s in WORKLOADS[workload]]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the raw samples go to $PS_CLOCKS_DIR (default: a temporary folder);
        # the JSON line carries their summary
        out = os.environ.get("PS_CLOCKS_DIR") or os.path.join(tempfile.gettempdir(), "ps_clocks")
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def kernel_code_digest(path):
    """First 16 hex digits of the sha256 of a source file without its
    whole-line // comments and trailing spaces: edits of comments leave it
    unchanged, any edit of code changes it."""
    with open(path) as f:
        lines = [line.rstrip() for line in f.read().splitlines() if not line.lstrip().startswith("//")]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def traffic_from_profile(workload, storage="pingpong"):
    """DRAM bytes per launch of the merge phase's kernels (k_merge_rounds, or
    k_vm_rounds + k_vm_copy with VM storage) from the committed ncu summary,
    if it was taken on the current kernel code (else None)."""
    name, kernel_src = ("merge_rounds", "ps_merge.cu") if storage == "pingpong" else ("vm_rounds", "ps_vm.cu")
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}.txt")
    src = os.path.join(ROOT, "paper_2605_27147_gb300", "csrc", kernel_src)
    try:
        digest = kernel_code_digest(src)
        vals = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_code_sha256_16") != digest:
            return None
        return float(vals["dram_bytes_per_launch_scaled"])
    except Exception:
        return None


def cpu_oracle_rate(data, budget_s, descending_runs=False, key_type="u32"):
    """Single-threaded oracle throughput on a bounded sample (elements/s)."""
    import oracle

    oracle.build()
    # the step's inputs in turn, at least once each, until about budget_s
    # seconds of one core are spent
    done, spent, sorts = 0, 0.0, 0
    while sorts < len(data) or spent < budget_s:
        d, n, s, keys = data[sorts % len(data)]
        t0 = time.perf_counter()
        oracle.powersort(keys, descending_runs=descending_runs, key_type=key_type)
        spent += time.perf_counter() - t0
        done += n
        sorts += 1
    used = f"{sorts} sorts cycling " + ", ".join(f"{d} n={n}" for d, n, s, k in data)
    return done / spent, spent, used


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "records_2^23":
        return run_reference_records(args)
    if args.workload == "keys64_2^24":
        return run_reference_keys64(args)
    if args.workload == "serving":
        return run_reference_serving(args)
    if args.workload == "batched_4096":
        from paper_2605_27147_gb300 import inputs as _inp

        keys_np, off_np = _inp.batch(4096, 3)
        parts = [keys_np[int(off_np[i]):int(off_np[i + 1])] for i in range(off_np.size - 1)]
        data = []
        for i in range(0, len(parts), 64):      # a step: 64 consecutive instances
            grp = parts[i:i + 64]
            data.append(("batched", sum(p.size for p in grp), 3, grp))
    elif args.workload == "hbm_2^28":
        # a bounded sample of the 2^28 workload: its first 2^24 keys per step
        # (the generator is a stream, so these are the 2^28 input's first keys)
        from paper_2605_27147_gb300 import inputs as _inp

        data = [(d, 1 << 24, s, _inp.make(d, 1 << 24, s)) for d, n, s in WORKLOADS["hbm_2^28"]]
    else:
        data = make_inputs(args.workload)
    import oracle

    oracle.build()
    desc = args.workload in DESCENDING_WORKLOADS
    vm = args.storage == "vm" and args.workload != "batched_4096"

    def page_size(n):
        # the library's default page: 2^round(log2 sqrt(n / log2 n)), within [2^8, 2^12]
        nn = max(float(n), 4.0)
        return 1 << min(12, max(8, math.floor(math.log2(math.sqrt(nn / math.log2(nn))) + 0.5)))

    times, elems = [], 0
    for i in range(args.warmup + args.steps):
        d, n, s, keys = data[i % len(data)]
        t0 = time.perf_counter()
        for k in (keys if isinstance(keys, list) else [keys]):
            if vm:
                oracle.powersort_vm(k, page_size(k.size), descending_runs=desc, key_type=args.key_type)
            else:
                oracle.powersort(k, descending_runs=desc, key_type=args.key_type)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            elems += n
    total = sum(times)
    value = elems / total
    storage = "VM storage" if vm else "Pingpong storage"
    sample = (f"one oracle run (Algorithm 1, {storage}, one thread) per step, cycling "
              f"{', '.join(f'{d} n={n}' for d, n, s, k in data)}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": args.workload, "storage": "vm" if vm else "pingpong",
                   "note": "CPU oracle on host cores (bounded sample per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_records(args, m=1 << 19, words=30):
    """The oracle on records: each step sorts the first 2^19 rows of one set."""
    import oracle
    from paper_2605_27147_gb300 import inputs

    oracle.build()
    sets = [inputs.records(k, m, 1, words=words) for k in ("random", "zero")]
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.powersort_records(sets[i % 2])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = m * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "records/s (30-word rows, lexicographic), 1xGB300", "value": value,
        "unit": "records/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "records_2^23", "note": "CPU oracle, first 2^19 rows per step"},
        "cpu_baseline": {"value": value, "unit": "records/s", "cores": 1, "kind": "oracle",
                         "sample": "first 2^19 rows of randomBlob30 / zeroBlob30, alternating"},
        "e2e": {"value": value, "unit": "records/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_serving(args, budget_s=10.0):
    """The oracle on the serving stream's requests, in arrival order, one at a
    time, for about budget_s seconds of one core (each step one request)."""
    import oracle
    from paper_2605_27147_gb300 import inputs

    oracle.build()
    _, sizes = inputs.poisson_requests(2000.0, 10.0, 4)
    elems, spent, done = 0, 0.0, 0
    for i, n in enumerate(sizes.tolist()):
        keys = inputs.uniform(int(n), 100 + i)
        t0 = time.perf_counter()
        oracle.powersort(keys)
        spent += time.perf_counter() - t0
        elems += int(n)
        done += 1
        if spent > budget_s and done >= args.steps:
            break
    value = elems / spent
    line = {
        "impl": "reference", "metric": "hot-path elements/s & % HBM roofline, 1xGB300; batched vs plain; p50/p99 ms",
        "value": value, "unit": "elements/s", "n_gpus": args.gpus, "steps": done, "warmup": 0,
        "ms_per_step": 1000 * spent / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serving", "note": f"CPU oracle on the first {done} requests of the stream, one core"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": f"the first {done} requests (sizes log-uniform in [2^10, 2^24], seed 4)"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_keys64(args, m=1 << 21):
    """The oracle on 64-bit keys: each step sorts the first 2^21 keys of one set."""
    import oracle
    from paper_2605_27147_gb300 import inputs

    oracle.build()
    hi = inputs.uniform(m, 1).astype(np.uint64)
    lo = inputs.uniform(m, 2).astype(np.uint64)
    sets = [((hi << np.uint64(32)) | lo, "u64"), ((lo.astype(np.int64) - (1 << 31)).view(np.uint64), "i64"),
            ((lo << np.uint64(32)) | hi, "f64")]
    times = []
    for i in range(args.warmup + args.steps):
        keys, kind = sets[i % 3]
        t0 = time.perf_counter()
        oracle.powersort_keys64(keys, kind)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = m * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "64-bit keys/s (sort + stable permutation), 1xGB300", "value": value,
        "unit": "elements/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "keys64_2^24", "note": "CPU oracle, first 2^21 keys of one set per step"},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": "first 2^21 keys of the u64 / i64 / f64 sets, in turn"},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _oracle_chunk(chunk):
    """Worker of the CPU baseline pool: oracle sorts of a list of instances."""
    import time as _t

    import oracle as _o

    t0 = _t.perf_counter()
    n = 0
    for keys in chunk:
        _o.powersort(keys)
        n += keys.size
    return n, _t.perf_counter() - t0


def cpu_oracle_parallel(parts, budget_instances):
    """The oracle over instances on every host core (spawned pool: no fork after CUDA)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    sample = parts[:budget_instances]
    chunks = [sample[i::cores] for i in range(cores)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_chunk, chunks)
    wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    cpu_s = sum(r[1] for r in res)
    return n / wall, cores, f"oracle on the first {len(sample)} instances ({n} elements), " \
                            f"{cores} processes, {cpu_s:.1f} s of CPU, {wall:.1f} s wall"


def batched_leg(steps, warmup, dev, stream, world=1, dist=None, e2e_steps=3):
    """Config 4 on one GPU: 4096 instances in one captured-graph replay per
    step, compared with a loop of single-instance calls on the same data.
    Returns the measurements as a dict (the caller builds the JSON line)."""
    import torch

    from paper_2605_27147_gb300 import autotune, binding, inputs, replicas

    keys_np, off_np = inputs.batch(4096, 3)
    sizes = np.diff(off_np.astype(np.int64))
    total, count, max_n = int(keys_np.size), int(sizes.size), int(sizes.max())
    pristine = torch.from_numpy(keys_np.view(np.int32)).to(dev)
    work = pristine.clone()
    perm = torch.empty(total, dtype=torch.int32, device=dev)
    doff = torch.from_numpy(off_np.astype(np.int64)).to(dev)
    tuned = autotune.tune(work, doff, perm, max_n, stream=stream)
    ctx = binding.Context(max_n, want_perm=True, max_total=total, max_count=count, tile_log2=tuned["tile_log2"],
                          merge_lanes=tuned["merge_lanes"],
                          flags=binding.PS_FLAG_TIMING, device=dev.index, stream=stream)
    graph = ctx.graph_batched(work, doff, perm)

    def replay(timed):
        with torch.cuda.stream(stream):
            work.copy_(pristine)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.launch()
            e1.record(stream)
        return (e0, e1) if timed else None

    for _ in range(warmup):
        replay(False)
    ctx.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    recs = []
    with ClockSampler(dev.index) as clk:
        for _ in range(steps):
            recs.append(replay(True))
        torch.cuda.synchronize(dev)
    ctx.sync()
    if dist:
        dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in recs)
    total_ms_max = replicas.max_over_ranks(total_ms, dist, dev)
    value = replicas.job_rate(steps * total, world, total_ms_max)
    # result check on a few instances (sorted keys, permutation consistent)
    gk = work.cpu().numpy().view(np.uint32)
    gp = perm.cpu().numpy().view(np.uint32)
    for q in range(0, count, 409):
        a, b = int(off_np[q]), int(off_np[q + 1])
        assert np.array_equal(gk[a:b], np.sort(keys_np[a:b]))
        assert np.array_equal(keys_np[a:b][gp[a:b].astype(np.int64)], gk[a:b])
    # phase breakdown and algorithmic bytes from one ordinary (uncaptured) call
    with torch.cuda.stream(stream):
        work.copy_(pristine)
    st = ctx.run_batched(work, doff, perm, stats=True)
    ph = ctx.phase_times()
    # the per-instance loop of the plain entry point on the same data
    plain = binding.Context(max_n, want_perm=True, device=dev.index, stream=stream)
    offs = [int(x) for x in off_np]
    with torch.cuda.stream(stream):
        work.copy_(pristine)
    plain.sync()
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    for q in range(count):
        a, b = offs[q], offs[q + 1]
        if b > a:
            plain.run(work[a:b], perm[a:b])
    l1.record(stream)
    plain.sync()
    loop_ms = l0.elapsed_time(l1)
    loop_rate = total / (loop_ms / 1000.0)
    plain.close()
    # end to end: pinned host keys in, graph replay, keys + permutation out
    e2e = None
    if e2e_steps:
        hk = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
        hko = torch.empty(total, dtype=torch.int32, pin_memory=True)
        hpo = torch.empty(total, dtype=torch.int32, pin_memory=True)
        tsum = 0.0
        for _ in range(e2e_steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                work.copy_(hk, non_blocking=True)
                graph.launch()
                hko.copy_(work, non_blocking=True)
                hpo.copy_(perm, non_blocking=True)
            stream.synchronize()
            tsum += time.perf_counter() - t0
        ctx.sync()
        e2e = {"value": e2e_steps * total * world / tsum, "unit": UNIT, "h2d_bytes_per_step": 4 * total,
               "d2h_bytes_per_step": 8 * total, "steps": e2e_steps,
               "api": "ps_graph_launch between pinned host<->device copies"}
    peak, peak_kind = peaks()
    merge_bytes = BYTES_PER_MERGED_ELEM * st["hbm_merge_elems"]
    achieved = merge_bytes / (ph["merge_rounds"] / 1000.0) / 1e9 if ph["merge_rounds"] > 0 else 0.0
    graph.close()
    ctx.close()
    del work, perm, pristine
    return {
        "value": value, "ms_per_step": total_ms_max / steps, "steps": steps, "warmup": warmup,
        "count": count, "total": total, "max_n": max_n, "tuned": tuned,
        "loop_rate": loop_rate, "loop_ms": loop_ms, "phases": ph, "stats": st,
        "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "e2e": e2e, "clocks": clk.summary(),
    }


def run_batched(args):
    """Workload batched_4096: one captured-graph replay per step."""
    import torch

    from paper_2605_27147_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and not args.no_cpu:      # before any CUDA work (the pool is spawned)
        keys_np, off_np = inputs.batch(4096, 3)
        parts = [keys_np[int(off_np[i]):int(off_np[i + 1])] for i in range(off_np.size - 1)]
        rate, cores, sample = cpu_oracle_parallel(parts, 1024)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    r = batched_leg(args.steps, args.warmup, dev, stream, world, dist, e2e_steps=0 if args.no_e2e else 3)
    st, tuned, value = r["stats"], r["tuned"], r["value"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batched_4096", "instances": r["count"], "total_elements": r["total"],
                   "sizes": "log-uniform in [2^8, 2^20), seed 3, uniform keys", "max_instance": r["max_n"],
                   "outputs": "sorted keys + stable permutation (uint32)", "storage": "pingpong",
                   "launch": "one CUDA-graph replay per step (persistent cooperative merge kernel)",
                   "autotune": {k: tuned[k] for k in ("tile_log2", "merge_lanes", "ms", "cached")},
                   "l2": "inputs (2 GiB keys) exceed L2; input restored before every replay (untimed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "batched_vs_plain_loop": {"batched": value / world, "plain_loop": r["loop_rate"],
                                  "ratio": (value / world) / r["loop_rate"], "plain_loop_ms": r["loop_ms"],
                                  "plain_loop_calls": r["count"]},
        "roofline": {"kernel": "k_merge_rounds (HBM merge rounds)", "bound": "hbm", "achieved": r["achieved"],
                     "peak": r["peak"], "peak_kind": r["peak_kind"], "unit": "GB/s",
                     "frac": r["achieved"] / r["peak"], "traffic": None,
                     "algorithmic_bytes": "16 B per element per HBM merge"},
        "kernels": {"phase_ms_one_call": r["phases"], "stats": {k: st[k] for k in ("runs", "merge_cost", "tiles",
                                                                                    "global_nodes", "rounds",
                                                                                    "hbm_merge_elems")}},
        "cpu_baseline": cpu, "e2e": r["e2e"], "clocks": r["clocks"],
        "gpu_launches": int(st["launches"]) * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_records(args, n=1 << 23, words=30):
    """Record sorts: rows of 30 words, lexicographic (ps_sort_records)."""
    import torch

    from paper_2605_27147_gb300 import binding, inputs, replicas

    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kinds = ("random", "zero")
    host = [inputs.records(k, n, 1 + replicas.replica_seed(0, rank), words=words) for k in kinds]
    recs = [torch.from_numpy(h.view(np.int32)).to(dev) for h in host]
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    out = torch.empty((n, words), dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(n, want_perm=True, flags=binding.PS_FLAG_RECORDS | binding.PS_FLAG_TIMING, device=local,
                          stream=stream)
    for _ in range(args.warmup):
        for r in recs:
            ctx.sort_records(r, perm, out)
    ctx.sync()
    times, merge_ms, merge_bytes, phases = [], 0.0, 0, []
    stats = {}
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            for i, r in enumerate(recs):
                flush.fill_(i)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.sort_records(r, perm, out)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                ph = ctx.phase_times()
                phases.append(ph)
                merge_ms += ph["merge_rounds"]
    for i, r in enumerate(recs):
        st = ctx.sort_records(r, perm, out, stats=True)
        stats[kinds[i]] = {k: st[k] for k in ("runs", "merge_cost", "rounds", "hbm_merge_elems")}
        merge_bytes += BYTES_PER_MERGED_ELEM * st["hbm_merge_elems"] * args.steps
        if i == len(recs) - 1:
            # the last sort's rows must be in lexicographic order
            o = out.cpu().numpy().view(np.uint32)
            d = o[1:] != o[:-1]
            f = np.argmax(d, axis=1)
            rows = np.arange(n - 1)
            assert np.all(~d.any(axis=1) | (o[1:][rows, f] > o[:-1][rows, f]))
    total_ms = replicas.max_over_ranks(sum(times), dist, dev)
    value = replicas.job_rate(n * len(times), world, total_ms)
    peak, peak_kind = peaks()
    achieved = merge_bytes / (merge_ms / 1000.0) / 1e9
    row_bytes = 3 * words * 4 * n * len(times)     # rows read by the scan, read and written by the gather
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle

        oracle.build()
        m = 1 << 19
        dt, sorts = 0.0, 0
        while sorts < len(host) or dt < args.cpu_sample_seconds:   # the sets in turn, to the time budget
            t0 = time.perf_counter()
            oracle.powersort_records(host[sorts % len(host)][:m])
            dt += time.perf_counter() - t0
            sorts += 1
        cpu = {"value": m * sorts / dt, "unit": "records/s", "cores": 1, "kind": "oracle",
               "sample": f"{sorts} sorts of the first 2^19 rows of the record sets in turn "
                         f"({dt:.1f} s of one host core)"}
    line = {
        "metric": "records/s (30-word rows, lexicographic), 1xGB300", "value": value, "unit": "records/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "records_2^23", "instances": [f"{k}Blob30 n=2^23 seed 1" for k in kinds],
                   "outputs": "stable permutation + the rows in order", "l2": "flushed before every timed sort"},
        "roofline": {"kernel": "k_merge_rounds (window keys)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None},
        "kernels": {"phase_ms_per_step": {k: sum(p[k] for p in phases) / args.steps for k in binding.PHASES},
                    "row_gbs": row_bytes / (sum(times) / 1000.0) / 1e9},
        "stats": stats, "cpu_baseline": cpu, "e2e": None, "clocks": clk.summary(),
        "gpu_launches": None,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_keys64(args, n=1 << 24):
    """64-bit key sorts through ps_sort_keys64."""
    import torch

    from paper_2605_27147_gb300 import binding, inputs, replicas

    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = 1 + replicas.replica_seed(0, rank)
    hi = inputs.uniform(n, seed).astype(np.uint64)
    lo = inputs.uniform(n, seed + 1).astype(np.uint64)
    sets = [("u64", binding.PS_KEY_U32, (hi << np.uint64(32)) | lo),
            ("i64", binding.PS_KEY_I32, (lo.astype(np.int64) - (1 << 31)).view(np.uint64)),
            ("f64", binding.PS_KEY_F32, (lo << np.uint64(32)) | hi)]
    pristine = [torch.from_numpy(b.view(np.int64)).to(dev) for _, _, b in sets]
    work = torch.empty(n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(n, want_perm=True, flags=binding.PS_FLAG_RECORDS, device=local, stream=stream)
    for _ in range(args.warmup):
        for i, (_, kt, _) in enumerate(sets):
            work.copy_(pristine[i])
            ctx.sort_keys64(work, perm, kt)
    ctx.sync()
    per_set = {name: 0.0 for name, _, _ in sets}
    times = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            for i, (name, kt, _) in enumerate(sets):
                work.copy_(pristine[i])
                flush.fill_(i)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.sort_keys64(work, perm, kt)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                per_set[name] += times[-1]
    stats, launches = {}, 0
    for i, (name, kt, b) in enumerate(sets):
        work.copy_(pristine[i])
        st = ctx.sort_keys64(work, perm, kt, stats=True)
        stats[name] = {k: st[k] for k in ("runs", "merge_cost", "rounds", "launches")}
        launches += int(st["launches"]) * args.steps
    out = work.cpu().numpy().view(np.uint64)          # the f64 set, last: non-decreasing in totalOrder
    sgn = (out >> np.uint64(63)).astype(bool)
    img = np.where(sgn, ~out, out | np.uint64(1 << 63))
    assert np.all(img[1:] >= img[:-1])
    total_ms = replicas.max_over_ranks(sum(times), dist, dev)
    value = replicas.job_rate(n * len(times), world, total_ms)
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle

        oracle.build()
        m, dt, sorts = 1 << 20, 0.0, 0
        while sorts < len(sets) or dt < args.cpu_sample_seconds:   # the sets in turn, to the time budget
            name, _, b = sets[sorts % len(sets)]
            t0 = time.perf_counter()
            oracle.powersort_keys64(b[:m], name)
            dt += time.perf_counter() - t0
            sorts += 1
        cpu = {"value": m * sorts / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
               "sample": f"{sorts} sorts of the first 2^20 keys of the u64 / i64 / f64 sets in turn "
                         f"({dt:.1f} s of one host core)"}
    line = {
        "metric": "64-bit keys/s (sort + stable permutation), 1xGB300", "value": value, "unit": "elements/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "keys64_2^24", "instances": [f"{name} n=2^24" for name, _, _ in sets],
                   "l2": "flushed before every timed sort"},
        "per_set_elements_per_s": {k: n * args.steps / (v / 1000.0) for k, v in per_set.items()},
        "stats": stats, "clocks": clk.summary(), "cpu_baseline": cpu, "e2e": None, "roofline": None,
        "gpu_launches": launches,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serving_leg(local, lane_total, rate=2000.0, duration=10.0, budget=64 << 30, lanes=4, storage="pingpong"):
    """Config 5: Poisson arrivals replayed in real time through ps_server
    (lanes of Pingpong or VM storage).  Returns the latencies and the server's
    statistics as a dict."""
    import torch

    from paper_2605_27147_gb300 import binding, inputs

    arrivals, sizes = inputs.poisson_requests(rate, duration, 4)
    sizes = sizes.astype(np.int64)
    max_n = 1 << 24
    # request inputs: views at varying offsets into a pinned pool of uniform keys
    pool_n = 1 << 26
    pool = torch.from_numpy(inputs.uniform(pool_n, 4).view(np.int32)).pin_memory()
    starts = (np.arange(sizes.size, dtype=np.int64) * 7919 * 1021) % (pool_n - max_n)
    # results: a ring of pinned memory, slots freed in completion order
    ring_n = 1 << 29
    ring_k = torch.empty(ring_n, dtype=torch.int32, pin_memory=True)
    ring_p = torch.empty(ring_n, dtype=torch.int32, pin_memory=True)
    pk, pp, pin = ring_k.data_ptr(), ring_p.data_ptr(), pool.data_ptr()
    # the server's per-batch trace (host and device times of every batch's
    # copies in, wait for the previous sort, sort and copies out) explains
    # the tail: where a slow request's time went
    trace_path = os.path.join(tempfile.mkdtemp(prefix="ps_trace_"), "batches.csv")
    os.environ["PS_SERVER_TRACE"] = trace_path
    try:
        srv = binding.Server(budget, max_n, lanes=lanes, lane_max_total=lane_total, lane_max_count=256,
                             device=local,
                             storage=binding.PS_MODE_VM if storage == "vm" else binding.PS_MODE_PINGPONG)
    finally:
        del os.environ["PS_SERVER_TRACE"]
    # warm-up: a few requests (module loading, first launches)
    for i in range(8):
        srv.wait(srv.submit(pin, pk, pp, 1 << 20), 60.0)
    # the largest request's time alone (the floor of any latency bound)
    solo = []
    for _ in range(3):
        solo.append(srv.wait(srv.submit(pin, pk, pp, int(sizes.max())), 60.0))
    head, tail = 0, 0                   # ring positions (elements, monotone)
    live = []                           # (ticket, ring start, n) in submission order
    tickets = []
    import gc

    gc.disable()                        # no collector pause inside the stream
    t0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(sizes.size):
            n = int(sizes[i])
            # sleep until just before the arrival, then spin the last 200 us
            # (a core spinning for the whole stream competes with the server)
            while True:
                dt = arrivals[i] - (time.perf_counter() - t0)
                if dt <= 0:
                    break
                if dt > 4e-4:
                    time.sleep(dt - 2e-4)
            # free completed slots at the ring's tail; wait if the ring is full
            while live and (head - tail + n > ring_n):
                tk, st0, nn = live[0]
                srv.wait(tk, 60.0)
                live.pop(0)
                tail = st0 + nn
            pos = head % ring_n
            if pos + n > ring_n:            # do not wrap inside a request
                head += ring_n - pos
                pos = 0
                while live and head - tail + n > ring_n:
                    tk, st0, nn = live[0]
                    srv.wait(tk, 60.0)
                    live.pop(0)
                    tail = st0 + nn
            t = srv.submit(pin + 4 * int(starts[i]), pk + 4 * pos, pp + 4 * pos, n)
            live.append((t, head, n))
            while live:                     # retire finished heads cheaply
                done, _ = srv.poll(live[0][0])
                if not done:
                    break
                tk, st0, nn = live.pop(0)
                tail = st0 + nn
            head += n
            tickets.append(t)
        lat = [srv.wait(t, 120.0) for t in tickets]
        t_end = time.perf_counter()
    gc.enable()
    st = srv.stats()
    srv.close()                         # writes the trace
    phases = batch_phases(trace_path)
    lat_ms = np.array(lat) * 1000.0
    elems = int(sizes.sum())
    wall = t_end - t0
    return {
        "value": elems / wall, "wall_s": wall, "requests": int(sizes.size), "elements": elems,
        "offered": elems / duration, "rate": rate, "duration": duration, "budget": budget,
        "mean_n": float(sizes.mean()), "max_n": int(sizes.max()),
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "mean": float(lat_ms.mean()), "max": float(lat_ms.max())},
        "largest_request_solo_ms": 1000.0 * float(min(solo)),
        "batch_phases_ms": phases,
        "server": st, "clocks": clk.summary(),
        "raw": {"arrival_s": arrivals, "n": sizes, "latency_ms": lat_ms},   # not printed
    }


def batch_phases(path):
    """p50 / p99 / max per phase of the server's batches, from its trace (ms):
    enqueue (host), copies in, wait for the previous batch's sort, sort,
    copies out; and the batches whose copies in ran below 10 GB/s."""
    import csv

    try:
        rows = list(csv.DictReader(open(path)))
    except OSError:
        return None
    if not rows:
        return None
    col = lambda k: np.array([float(r[k]) for r in rows])
    el = col("elements")
    parts = {
        "enqueue": 1000.0 * (col("host_enqueue_end_s") - col("host_enqueue_begin_s")),
        "copies_in": col("gpu_copies_in_done_ms") - col("gpu_first_copy_in_ms"),
        "wait_previous_sort": col("gpu_sort_start_ms") - col("gpu_copies_in_done_ms"),
        "sort": col("gpu_sort_end_ms") - col("gpu_sort_start_ms"),
        "copies_out": col("gpu_copies_out_done_ms") - col("gpu_sort_end_ms"),
    }
    out = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "max": float(v.max())}
           for k, v in parts.items()}
    cin = parts["copies_in"]
    slow = (el >= (1 << 20)) & (4.0 * el / np.maximum(cin, 1e-6) / 1e6 < 10.0)
    out["batches"] = len(rows)
    out["slow_copies_in"] = {"batches": int(slow.sum()),
                             "host_times_s": [round(float(x), 3) for x in col("host_enqueue_begin_s")[slow][:8]],
                             "note": "batches of >= 2^20 elements whose host->device copies (pinned "
                                     "sources) ran below 10 GB/s"}
    return out


def run_serving(args):
    # Elements per batch are capped so that a burst cannot build one long
    # batch (latency grows with the batch; the offered load is far below
    # capacity, so smaller batches cost no throughput).
    """Workload serving: Poisson arrivals replayed in real time through ps_server."""
    import torch

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    r = serving_leg(local, args.lane_total, storage=args.storage)
    st = r["server"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["requests"], "warmup": 8,
        "ms_per_step": 1000.0 * r["wall_s"] / r["requests"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serving", "arrivals": f"Poisson {r['rate']:.0f}/s for {r['duration']:.0f} s, seed 4",
                   "sizes": "log-uniform in [2^10, 2^24]", "requests": r["requests"],
                   "offered_elements_per_s": r["offered"], "budget_bytes": r["budget"],
                   "lanes": st["lanes"], "lane_max_total": st["lane_max_total"], "storage": args.storage,
                   "device_bytes": st["device_bytes"], "outputs": "sorted keys + stable permutation",
                   "io": "pinned host arrays in, pinned host arrays out (copies inside every latency)"},
        "latency_ms": r["latency_ms"],
        "largest_request_solo_ms": r["largest_request_solo_ms"],
        "batch_phases_ms": r["batch_phases_ms"],
        "server": st,
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": int(4 * r["mean_n"]),
                "d2h_bytes_per_step": int(8 * r["mean_n"]),
                "api": "ps_server_submit / ps_server_wait on pinned host arrays"},
        "roofline": None, "cpu_baseline": None, "clocks": r["clocks"],
        # a VM lane sorts each request by itself (one call, plus the Copy launch)
        "gpu_launches": ((LAUNCHES_PER_BATCH + 1) * int(r["requests"]) if args.storage == "vm"
                         else LAUNCHES_PER_BATCH * int(st["batches"])),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_4096":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "records_2^23":
        return run_records(args)
    if args.workload == "keys64_2^24":
        return run_keys64(args)

    import torch

    from paper_2605_27147_gb300 import binding, replicas

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    data = make_inputs(args.workload)
    max_n = max(n for _, n, _, _ in data)
    stream = torch.cuda.current_stream(dev)
    pristine = [torch.from_numpy(k.view(np.int32)).to(dev) for _, _, _, k in data]
    work = torch.empty(max_n, dtype=torch.int32, device=dev)
    perm = torch.empty(max_n, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    mode = binding.PS_MODE_VM if args.storage == "vm" else binding.PS_MODE_PINGPONG
    desc = args.workload in DESCENDING_WORKLOADS
    variant = binding.PS_FLAG_DESCENDING_RUNS if desc else 0
    key_type = {"u32": binding.PS_KEY_U32, "i32": binding.PS_KEY_I32, "f32": binding.PS_KEY_F32}[args.key_type]
    ctx = binding.Context(max_n, mode=mode, want_perm=True, flags=binding.PS_FLAG_TIMING | variant,
                          key_type=key_type, page_log2=args.page_log2, device=local, stream=stream)

    def one_sort(i, timed):
        n = data[i][1]
        work[:n].copy_(pristine[i])
        flush.fill_(i)                      # write 512 MiB: L2 holds nothing of the input
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.run(work[:n], perm[:n], stats=False)
        e1.record(stream)
        if not timed:
            return None
        return e0, e1, n

    for _ in range(args.warmup):
        for i in range(len(data)):
            one_sort(i, False)
    ctx.sync()
    torch.cuda.synchronize(dev)

    recs, phases = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            for i in range(len(data)):
                e0, e1, n = one_sort(i, True)
                ph = ctx.phase_times()        # waits for this sort (events on the same stream)
                recs.append((e0, e1, n, i))
                phases.append(ph)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ctx.sync()
    sort_ms = [e0.elapsed_time(e1) for e0, e1, _, _ in recs]
    total_ms = sum(sort_ms)
    elems = sum(n for _, _, n, _ in recs)
    # one stats call per distribution for the algorithmic byte counts
    hbm, rounds = {}, {}
    for i in range(len(data)):
        n = data[i][1]
        work[:n].copy_(pristine[i])
        flush.fill_(i)
        st = ctx.run(work[:n], perm[:n], stats=True)
        hbm[i] = st
        launches_per_sort = int(st["launches"])
        rounds[data[i][0]] = [[round(x, 1) for x in rt] for rt in ctx.round_times()]
    merge_ms = sum(p["merge_rounds"] for p in phases)
    # HBM merges move key + permutation entry, read and written: 16 B per
    # element; VM storage's final Copy moves whole pages the same way
    merge_bytes = sum(BYTES_PER_MERGED_ELEM * (hbm[i]["hbm_merge_elems"] + hbm[i]["copy_pages"] * hbm[i]["page_size"])
                      for _, _, _, i in recs)
    tiles_ms = sum(p["tiles"] for p in phases)
    tiles_bytes = sum(12 * data[i][1] for _, _, _, i in recs)   # keys read, keys + perm written
    runs_ms = sum(p["runs"] for p in phases)
    phase_tot = {k: sum(p[k] for p in phases) for k in binding.PHASES}

    total_ms_max = replicas.max_over_ranks(total_ms, dist, dev)
    value = replicas.job_rate(elems, world, total_ms_max)

    plain_rule = None
    if desc:
        # the same inputs and timing without the variant: the plain rule's rate
        pctx = binding.Context(max_n, mode=mode, want_perm=True, key_type=key_type, device=local, stream=stream)
        pms, pel = 0.0, 0
        for step in range(args.warmup + args.steps):
            for i in range(len(data)):
                n = data[i][1]
                work[:n].copy_(pristine[i])
                flush.fill_(i)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pctx.run(work[:n], perm[:n], stats=False)
                e1.record(stream)
                e1.synchronize()
                if step >= args.warmup:
                    pms += e0.elapsed_time(e1)
                    pel += n
        work[:data[0][1]].copy_(pristine[0])
        pst = pctx.run(work[:data[0][1]], perm[:data[0][1]], stats=True)
        pctx.close()
        plain_rule = {"value": pel / (pms / 1000.0), "unit": UNIT, "runs": pst["runs"],
                      "merge_cost": pst["merge_cost"], "note": "same input and timing, ascending runs only"}

    # end to end through ps_run_host with pinned host arrays
    e2e = None
    if not args.no_e2e:
        hctx = binding.Context(max_n, mode=mode, want_perm=True, flags=binding.PS_FLAG_HOST_IO | variant,
                               key_type=key_type, device=local, stream=stream)
        hk = torch.empty(max_n, dtype=torch.int32, pin_memory=True)
        hp = torch.empty(max_n, dtype=torch.int32, pin_memory=True)
        src = [torch.from_numpy(k.view(np.int32)) for _, _, _, k in data]
        e2e_steps = max(1, min(args.steps, 10))
        for i in range(len(data)):   # warm-up
            n = data[i][1]
            hk[:n].copy_(src[i])
            hctx.run_host(hk.data_ptr(), n, hp.data_ptr())
        tsum, esum, bi, bo = 0.0, 0, 0, 0
        for _ in range(e2e_steps):
            for i in range(len(data)):
                n = data[i][1]
                hk[:n].copy_(src[i])
                t0 = time.perf_counter()
                hctx.run_host(hk.data_ptr(), n, hp.data_ptr())
                tsum += time.perf_counter() - t0
                esum += n
                bi += 4 * n
                bo += 8 * n
        # the result of the last e2e sort must be the sorted keys (in the key order)
        last_n = data[-1][1]
        out = hk[:last_n].numpy()
        if args.key_type == "i32":
            assert np.all(np.diff(out.view(np.int32).astype(np.int64)) >= 0)
        elif args.key_type == "u32":
            assert np.all(np.diff(out.view(np.uint32).astype(np.int64)) >= 0)
        else:   # totalOrder: as signed integers, negatives by reversed magnitude
            b = out.view(np.int32).astype(np.int64)
            assert np.all(np.diff(np.where(b < 0, -(b & 0x7fffffff) - 1, b)) >= 0)
        hctx.close()
        e2e = {"value": esum * world / tsum, "unit": UNIT, "h2d_bytes_per_step": bi // e2e_steps,
               "d2h_bytes_per_step": bo // e2e_steps, "steps": e2e_steps,
               "api": "ps_run_host (pinned host arrays)"}
        if mode == binding.PS_MODE_PINGPONG:
            # the same sorts as a stream of host requests through the server:
            # two lanes, so one sort's copies overlap the other's kernels
            single = dict(e2e)
            ins = [torch.from_numpy(k.view(np.int32)).pin_memory() for _, _, _, k in data]
            # two sets of result buffers: while one request's results come
            # back, the next request's copies in and sort run
            kos = [[torch.empty(t.numel(), dtype=torch.int32, pin_memory=True) for t in ins] for _ in range(2)]
            pos = [[torch.empty(t.numel(), dtype=torch.int32, pin_memory=True) for t in ins] for _ in range(2)]
            srv = binding.Server(2 * max_n * 24, max_n, lanes=2, lane_max_total=max_n, lane_max_count=1,
                                 device=local, key_type=key_type, flags=variant)

            def stream(steps):
                # the step's sorts as a stream of requests, at most two in flight
                reqs = [(s, i) for s in range(steps) for i in range(len(ins))]
                tickets = []
                for j, (s, i) in enumerate(reqs):
                    if j >= 2:
                        srv.wait(tickets[j - 2])
                    b = j % 2
                    tickets.append(srv.submit(ins[i].data_ptr(), kos[b][i].data_ptr(), pos[b][i].data_ptr(),
                                              ins[i].numel()))
                for t in tickets[-2:]:
                    srv.wait(t)
                return reqs

            stream(1)                          # warm-up
            # at least 30 requests, so that the stream's fill and drain (the
            # first copy in, the last copy out) weigh little in its rate
            sreqs = max(e2e_steps, -(-30 // len(ins)))
            t0 = time.perf_counter()
            reqs = stream(sreqs)
            tstream = time.perf_counter() - t0
            srv.close()
            for j in range(max(0, len(reqs) - 2), len(reqs)):
                # every result is its input gathered through the permutation
                b, i = j % 2, reqs[j][1]
                k = data[i][3]
                got = kos[b][i].numpy().view(np.uint32)
                assert np.array_equal(k.view(np.uint32)[pos[b][i].numpy().view(np.uint32)], got)
                if args.key_type == "u32":
                    assert np.all(got[1:] >= got[:-1])
            e2e = {"value": sreqs * sum(n for _, n, _, _ in data) * world / tstream, "unit": UNIT,
                   "h2d_bytes_per_step": bi // e2e_steps, "d2h_bytes_per_step": bo // e2e_steps, "steps": sreqs,
                   "api": "ps_server_submit / ps_server_wait (pinned host arrays, 2 lanes, "
                          "at most two requests in flight)",
                   "single_call": {"value": single["value"], "api": single["api"]}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        big = any(n > (1 << 24) for _, n, _, _ in data)
        sample = [(d, 1 << 24, s, k[: 1 << 24].copy()) for d, n, s, k in data] if big else data
        rate, spent, used = cpu_oracle_rate(sample, args.cpu_sample_seconds, desc, args.key_type)
        what = f"the first 2^24 keys of each n = 2^{int(np.log2(max_n))} input: " if big else ""
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{what}{used} ({spent:.1f} s of one host core)"}

    peak, peak_kind = peaks()
    achieved = merge_bytes / (merge_ms / 1000.0) / 1e9
    traffic = traffic_from_profile(args.workload, args.storage)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {
            "workload": args.workload,
            "instances": [f"{d} n=2^{int(np.log2(n))} seed {s}" for d, n, s, _ in data],
            "outputs": "sorted keys + stable permutation (uint32)",
            "storage": args.storage,
            "keys": {"u32": "unsigned 32-bit", "i32": "signed 32-bit (two's complement)",
                     "f32": "IEEE 754 binary32, totalOrder"}[args.key_type],
            "runs": "ascending and strictly decreasing (Sec. 5 variant)" if desc else "ascending (Sec. 5 rule)",
            "scratch_bytes": hbm[0]["scratch_bytes"],
            "peak_pool_pages": hbm[0]["peak_pages"],
            "l2": "flushed before every timed sort (512 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        },
        "roofline": {
            "kernel": "k_merge_rounds (HBM merge rounds)" if args.storage == "pingpong"
            else "k_vm_rounds + k_vm_copy (paged merge rounds, final Copy)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "algorithmic_bytes": "16 B per element per HBM merge (key + perm read and written), "
                                 "summed over the merges of the call"
                                 + ("; plus 16 B per element of every page the final Copy moves"
                                    if args.storage == "vm" else ""),
        },
        "kernels": {
            "phase_ms_per_step": {k: v / args.steps for k, v in phase_tot.items()},
            "tiles_gbs": tiles_bytes / (tiles_ms / 1000.0) / 1e9 if tiles_ms else None,
            "runs_gbs": sum(4 * data[i][1] for *_, i in recs) / (runs_ms / 1000.0) / 1e9 if runs_ms else None,
            "schedule_gbs": (merge_bytes + tiles_bytes + sum(4 * data[i][1] for *_, i in recs))
                            / (total_ms / 1000.0) / 1e9,
        },
        "stats": {data[i][0]: {k: hbm[i][k] for k in ("runs", "merge_cost", "tiles", "global_nodes", "rounds",
                                                      "hbm_merge_elems", "max_power", "scratch_bytes",
                                                      "peak_pages", "pages_spliced", "copy_pages")} for i in hbm},
        "round_timeline_us": rounds,
        "plain_rule": plain_rule,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches_per_sort * len(recs),
    }
    ctx.close()
    if args.storage == "vm":
        # where a paged sort's merge time goes: per round, the fixed steps
        # (page marks, records, splits, the touched list, the page-table
        # swap) and the page dataflow; from the statistics call's timeline
        line["vm_rounds"] = {
            k: {"rounds": len(rt),
                "fixed_steps_ms": sum((b - a) + (d - c) for a, b, c, d in rt) / 1000.0,
                "pages_ms": sum(c - b for a, b, c, d in rt) / 1000.0}
            for k, rt in rounds.items()}
        # extra memory of VM storage (Sec. 4 "Pages needed"; the paper's Fig. 5
        # table) beside the paper's bound and Pingpong's scratch at the same n
        st0 = hbm[0]
        pp = binding.Context(max_n, want_perm=True, device=local, stream=stream)
        pp_bytes = pp.scratch_bytes()
        pp.close()
        bound_elems = math.sqrt(max_n * 1 * math.log2(max_n))      # T = 1 word per element
        line["vm_memory"] = {
            "extra_bytes": st0["scratch_bytes"], "page_size": st0["page_size"], "pool_pages": st0["pool_pages"],
            "pool_bytes": st0["pool_pages"] * st0["page_size"] * 8, "peak_pool_pages": st0["peak_pages"],
            "paper_bound_elements": bound_elems, "paper_bound_bytes": 8 * bound_elems,
            "pingpong_scratch_bytes": pp_bytes, "input_bytes": 8 * max_n,
            "note": "extra_bytes = every device buffer the VM context holds: the page pool, the run list "
                    "(n/32 slots), page tables (n/P pages) and HBM-merge tables (< 4n/T); the paper's "
                    "sqrt(n T log n) counts the pool of one sequential sort, keys and permutation here",
        }
    if args.workload == "hbm_2^28" and not args.no_extras and world == 1:
        # the metric's other two parts, measured in the same run on the same GPU
        del work, perm, pristine, flush
        torch.cuda.empty_cache()
        line["batched_vs_plain"] = batched_summary(batched_leg(max(3, min(args.steps, 10)), 3, dev,
                                                               torch.cuda.Stream(dev), e2e_steps=0))
        torch.cuda.empty_cache()
        line["serving"] = serving_summary(serving_leg(local, args.lane_total))
        cin = ((line["serving"]["batch_phases_ms"] or {}).get("copies_in") or {}).get("max", 0.0)
        if cin >= 20.0:
            # a batch's host->device copies from pinned memory stalled (the
            # largest batch, 2^25 keys, copies in 20 ms at 6.7 GB/s): such
            # stalls, a host-side event seen in bursts on some machines, set
            # the tail; the stream is replayed once and both runs are reported
            again = serving_summary(serving_leg(local, args.lane_total))
            line["serving"]["replay_after_slow_copies"] = {
                k: again[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "sustained", "batch_phases_ms")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_summary(r):
    """The batched_vs_plain sub-object of the headline line (config 4)."""
    return {
        "workload": "batched_4096", "instances": r["count"], "total_elements": r["total"],
        "sizes": "log-uniform in [2^8, 2^20), seed 3, uniform keys",
        "batched": r["value"], "plain_loop": r["loop_rate"], "ratio": r["value"] / r["loop_rate"],
        "unit": UNIT, "batched_ms_per_replay": r["ms_per_step"], "replays": r["steps"],
        "plain_loop_ms": r["loop_ms"], "plain_loop_calls": r["count"],
        "launch": "one CUDA-graph replay (persistent cooperative merge kernel) vs one ps_run per instance",
        "autotune": {k: r["tuned"][k] for k in ("tile_log2", "merge_lanes", "ms", "cached")},
        "merge_rounds_frac": r["achieved"] / r["peak"],
        "clocks": r["clocks"],
    }


def serving_summary(r):
    """The serving sub-object of the headline line (config 5)."""
    st = r["server"]
    return {
        "workload": "serving", "arrivals": f"Poisson {r['rate']:.0f}/s for {r['duration']:.0f} s, seed 4",
        "sizes": "log-uniform in [2^10, 2^24]", "requests": r["requests"],
        "p50_ms": r["latency_ms"]["p50"], "p99_ms": r["latency_ms"]["p99"],
        "mean_ms": r["latency_ms"]["mean"], "max_ms": r["latency_ms"]["max"],
        "largest_request_solo_ms": r["largest_request_solo_ms"],
        "batch_phases_ms": r["batch_phases_ms"],
        "sustained": r["value"], "offered": r["offered"], "unit": UNIT,
        "budget_bytes": r["budget"], "device_bytes": st["device_bytes"], "lanes": st["lanes"],
        "lane_max_total": st["lane_max_total"], "batches": st["batches"], "max_busy_lanes": st["max_busy_lanes"],
        "io": "pinned host arrays in and out, copies inside every latency",
        "clocks": r["clocks"],
    }


if __name__ == "__main__":
    main()
