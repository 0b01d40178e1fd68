#!/usr/bin/env python
"""Benchmark: connected induced k-subgraphs classified per second.

One step = one pass of the whole counting path over one graph already in HBM:
graph ingest (pair-state matrix, G* neighbour lists), the two enumeration
launches and the histogram flush, through the C ABI acc_motif_count.  The
default workload is the directed Chung-Lu graph n=20000, m=100000 (Pareto
exponent 2.2, degrees capped at 500, 10% reciprocal arcs) at k=4; its line
is the headline, and the default run adds "sub_records" for every other
workload of the benchmark set, each timed under its own clock samples: k=3
on the Erdos-Renyi graph, k=5 on the regulatory-shaped graph, the 4008-graph
batch (graphs/s, beside one graph per launch) and the request server at 200
(saturated) and 50 (unsaturated) requests/s (latency percentiles,
subgraphs/s, beside the same requests counted one at a time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--headline-only]

N>1 runs one independent replica per GPU (rank), each counting its own copy
of the workload ("replicas only": the count has no exchange step), and
reports the units all ranks processed over the slowest rank's time.
``--impl reference`` times the CPU oracle on this host's cores over the same
workload (every ESU root in every step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "connected induced k-subgraphs classified/sec (k=3,4,5) and graphs/sec batched, bit-exact"
UNIT = "subgraphs/s"

WORKLOADS = {
    "chung_lu_n20000_m100000_k4": (synth.chung_lu_k4, 4),
    "er_n1000_m5000_k3": (synth.er_k3, 3),
    "regulatory_n5000_m15000_k5": (synth.regulatory_k5, 5),
}
DEFAULT_WORKLOAD = "chung_lu_n20000_m100000_k4"
BATCH_WORKLOAD = "batch_k4"
SIGNIFICANCE_WORKLOAD = "significance_k4"
SERVING_WORKLOAD = "serving"

# Algorithmic integer operations per classified subgraph when every leaf is
# visited (the leaf-enumerating form): k-1 pair states, each an address, a
# load and a 2-bit extract (4 ops) placed into the code (2 ops), then one
# table load and one histogram increment: 6(k-1) + 2.
def ops_per_subgraph(k: int) -> int:
    return 6 * (k - 1) + 2


# The counting form's unit of work is one neighbour entry scanned by the last
# two levels: the entry's load and its test against the root (2 ops), its
# k-2 pair states to the prefix (4 ops each: address, load, shift, mask),
# then one table load and one histogram increment: 4(k-2) + 4.
def ops_per_scanned_entry(k: int) -> int:
    return 4 * (k - 2) + 4


L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

REASON_BITS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
    0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting",
}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu),
               "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", str(self.period)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 3:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[2], 16) if parts[2].startswith("0x") else int(parts[2])
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b:
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; replicas)
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def reduce_max(dist, value: float, device=None) -> float:
    """Maximum of value over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_all_ranks: float, max_seconds: float) -> float:
    return units_all_ranks / max_seconds if max_seconds > 0 else float("nan")


# ---------------------------------------------------------------------------
# profiles: ncu DRAM traffic of the enumeration kernel, if captured for this source
# ---------------------------------------------------------------------------

def kernel_source_digest() -> str:
    h = hashlib.sha256()
    for f in ("enum.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1203_3415_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_counters(workload: str, mode: str):
    """(dram bytes per enumeration stage, ncu counters) from
    profiles/enum_<workload>_traffic.txt, when it was taken on the current
    kernel source in this mode; else (None, None)."""
    path = os.path.join(ROOT, "profiles", f"enum_{workload}_traffic.txt")
    if not os.path.exists(path):
        return None, None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            key, _, val = line.partition(":")
            kv[key.strip()] = val.strip()
    if kv.get("source_digest") != kernel_source_digest() or kv.get("mode", "count") != mode:
        return None, None
    try:
        traffic = float(kv["dram_bytes_per_stage"])
    except (KeyError, ValueError):
        traffic = None
    counters = {}
    for key in ("issue_active_pct", "lts_throughput_pct", "l1tex_throughput_pct", "warps_active_pct"):
        if key in kv:
            counters[key] = [float(x) for x in kv[key].split(",")]
    if counters:
        counters["phases"] = ["phase 1", "phase 2"]
        counters["source"] = "ncu --set full capture in profiles/, % of peak sustained"
    return traffic, (counters or None)



def golden_counts(workload: str):
    path = os.path.join(ROOT, "tests", "golden", workload + ".txt")
    if not os.path.exists(path):
        return None
    from tests.golden.golden_io import read_counts
    return read_counts(path)


# ---------------------------------------------------------------------------
# the CPU oracle timed on this host (cpu_baseline leg and reference arm)
# ---------------------------------------------------------------------------

def time_oracle(g, k: int, roots):
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    oracle.table(k)
    t = time.perf_counter()
    c = oracle.count(g.n, g.src, g.dst, k, threads=threads, roots=roots)
    dt = time.perf_counter() - t
    return int(c.sum()), dt, threads


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    make, k = WORKLOADS[args.workload]
    g = make()
    roots = (0, g.n if args.reference_roots <= 0 else min(g.n, args.reference_roots))
    times, units = [], 0
    threads = 1
    for i in range(args.warmup + args.steps):
        units, dt, threads = time_oracle(g, k, roots)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = units * len(times) / total
    sample = (f"the whole workload, all {g.n} ESU roots ({units} subgraphs per step)" if roots[1] == g.n else
              f"ESU roots {roots[0]}..{roots[1] - 1} of {g.n} ({units} subgraphs per step)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "k": k, "n": g.n, "m": g.m, "subgraphs_per_step": units},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

class GpuEnv:
    """Torch, the process group, the device and the library of one rank."""

    def __init__(self):
        import torch
        self.torch = torch
        self.world, self.rank, self.local = dist_env()
        torch.cuda.set_device(self.local)
        self.dist = dist_init(self.world, "nccl")
        self.dev = torch.device("cuda", self.local)
        from paper_1203_3415_gb300 import build as lib_build
        if self.rank == 0 or self.world == 1:
            lib_build.build()
        if self.dist is not None:
            self.dist.barrier()
        import paper_1203_3415_gb300 as acc
        self.acc = acc

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def issue_peak_gops(env):
    """Integer issue peak: SMs x 4 schedulers x 32 lanes per clock, at the
    measured maximum SM clock; (Gop/s, source)."""
    props = env.torch.cuda.get_device_properties(env.dev)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    src = "recipe nominal max SM clock 2070 MHz"
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            sm_max = float(json.load(f).get("sm_max_mhz", sm_max))
        src = "SM clock from MEASURED_PEAKS.json"
    return props.multi_processor_count * 4 * 32 * sm_max * 1e6 / 1e9, src


def table_build_ms(env, k, stream):
    """Device time of one build of the code -> class table for k (canonical
    labelling of all 2^(k(k-1)) codes and the class ranks), median of three
    builds after one untimed build, through the allocation-free entry point
    (so no allocation sits between the events)."""
    torch, acc, dev = env.torch, env.acc, env.dev
    table = torch.empty(1 << (k * (k - 1)), dtype=torch.int16, device=dev)
    codes = torch.empty(acc.NUM_CLASSES[k], dtype=torch.int32, device=dev)
    times = []
    for i in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = acc.acc_motif_build_table_static(k, stream.cuda_stream, table.data_ptr(), codes.data_ptr())
        e1.record(stream)
        if rc < 0:
            raise RuntimeError(f"table build failed: {acc.acc_strerror(rc)}")
        torch.cuda.synchronize(dev)
        if i:
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def measure_single(env, workload, steps, warmup, mode="count", schedule="", cpu_baseline=True, adjacency="auto"):
    """One graph counted per step through acc_motif_count, inputs resident in
    HBM, L2 flushed between steps; then the same through the host-buffer
    entry point.  Returns the bench line (without the run-wide keys)."""
    torch, acc, dev, dist = env.torch, env.acc, env.dev, env.dist
    make, k = WORKLOADS[workload]
    g = make()
    rowptr_np, col_np = g.csr()
    rowptr = torch.from_numpy(rowptr_np).to(dev)
    col = torch.from_numpy(col_np).to(dev)
    counts = torch.zeros(acc.NUM_CLASSES[k], dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    counter = acc.Counter(env.local)
    counter.set_mode({"count": acc.ACC_MODE_COUNT, "enumerate": acc.ACC_MODE_ENUMERATE,
                      "formula": acc.ACC_MODE_FORMULA, "auto": acc.ACC_MODE_AUTO}[mode])
    # the path the automatic mode takes (formula for k = 3 on the dense block)
    eff = mode if mode != "auto" else ("formula" if k == 3 and adjacency in ("auto", "dense") else "count")
    counter.prepare(k)
    counter.set_adjacency({"auto": acc.ACC_ADJ_AUTO, "dense": acc.ACC_ADJ_DENSE, "hash": acc.ACC_ADJ_HASH,
                           "sparse": acc.ACC_ADJ_SPARSE}[adjacency])
    if schedule:
        light, target = (int(x) for x in schedule.split(","))
        counter.set_schedule(light, target)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(warmup):
        flush.fill_(1)
        counter.count(rowptr, col, g.n, k, counts=counts, status=status, stream=stream)
    torch.cuda.synchronize(dev)
    if int(status.item()) != 0:
        raise RuntimeError(f"count failed: {acc.acc_strerror(int(status.item()))}")
    stats = counter.last_stats()
    n_k = int(counts.sum().item())
    gold = golden_counts(workload)
    parity = None
    if gold is not None:
        parity = bool(np.array_equal(counts.cpu().numpy(), gold[1]))

    # timed region: K steps, each bracketed by events on the launching stream;
    # L2 flushed (256 MiB write) between steps, outside the events.  Repeated
    # counts replay the library's launch graph of the whole sequence.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(env.local) if env.rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        counter.count(rowptr, col, g.n, k, counts=counts, status=status, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [s.elapsed_time(e) for s, e in ev]
    if int(status.item()) != 0 or int(counts.sum().item()) != n_k:
        raise RuntimeError("timed steps disagree with the warm-up result")
    # stage breakdown from a separate pass with per-stage events (kernels
    # launched one by one)
    counter.set_timing(True)
    build_ms, enum_ms, p1_ms, p2_ms = [], [], [], []
    for i in range(max(3, min(steps, 20))):
        flush.fill_(i & 0xFF)
        counter.count(rowptr, col, g.n, k, counts=counts, status=status, stream=stream)
        b, e, e1, e2 = counter.last_timing()
        build_ms.append(b)
        enum_ms.append(e)
        p1_ms.append(e1)
        p2_ms.append(e2)
    torch.cuda.synchronize(dev)
    counter.set_timing(False)
    local_s = sum(step_ms) / 1000.0
    if int(status.item()) != 0 or int(counts.sum().item()) != n_k:
        raise RuntimeError("timed steps disagree with the warm-up result")

    max_s = reduce_max(dist, local_s, dev)
    units = reduce_sum(dist, float(n_k) * steps, dev)
    value = whole_job_rate(units, max_s)

    # end to end through the public host-buffer entry point: pinned host
    # arrays in, int64 counts out, copies inside the timed region
    h_rowptr = torch.from_numpy(rowptr_np).pin_memory()
    h_col = torch.from_numpy(col_np).pin_memory()
    h_counts = torch.zeros(acc.NUM_CLASSES[k], dtype=torch.int64).pin_memory()
    e2e_steps = max(3, min(steps, 20))
    # two untimed calls: the second captures the launch graph the timed calls replay
    for _ in range(2):
        counter.count_host(h_rowptr, h_col, g.n, k, counts=h_counts)
    e2e_t = 0.0
    for _ in range(e2e_steps):
        flush.fill_(3)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        counter.count_host(h_rowptr, h_col, g.n, k, counts=h_counts)
        e2e_t += time.perf_counter() - t0
    if int(h_counts.sum().item()) != n_k:
        raise RuntimeError("host-buffer count differs from the device count")
    e2e_max = reduce_max(dist, e2e_t, dev)
    e2e_units = reduce_sum(dist, float(n_k) * e2e_steps, dev)
    counter.close()
    table_ms = table_build_ms(env, k, stream)
    if env.rank != 0:
        return None

    peak_gops, peak_src = issue_peak_gops(env)
    enum_s = statistics.mean(enum_ms) / 1000.0
    leaf_achieved = ops_per_subgraph(k) * n_k / enum_s / 1e9
    if eff == "count":
        units, per_unit = int(stats["scanned_entries"]), ops_per_scanned_entry(k)
        unit_name = "neighbour entries scanned by the last two levels"
    elif eff == "formula" and k == 3:
        units, per_unit = n_k, ops_per_subgraph(k)
        unit_name = "classified subgraphs (leaf-equivalent: the formula path visits none)"
    else:
        units, per_unit = n_k, ops_per_subgraph(k)
        unit_name = "classified subgraphs"
    achieved = per_unit * units / enum_s / 1e9
    # the profiles were taken with the default probe structure
    traffic, counters = profiled_counters(workload, eff) if adjacency == "auto" else (None, None)

    # CPU baseline: the oracle on this host's cores, the whole workload
    cpu = None
    if env.world == 1 and cpu_baseline:
        units_cpu, dt, threads = time_oracle(g, k, (0, g.n))
        cpu = {"value": units_cpu / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"the whole workload, all {g.n} ESU roots ({units_cpu} subgraphs), one pass, "
                         f"{dt:.2f} s"}
    return {
        "value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": 1000.0 * max_s / steps,
        "config": {"workload": workload, "k": k, "n": g.n, "m": g.m, "subgraphs_per_step": n_k,
                   "mode": mode if mode == eff else f"{mode} ({eff} path)", "adjacency": adjacency,
                   "l2": "flushed between timed steps (256 MiB device write)",
                   "parallelism": f"replicas{env.world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": traffic,
                     "kernel": "k_formula3" if eff == "formula" and k == 3 else f"k_enum<{k}> (phase 1 + phase 2)",
                     "work_unit": unit_name, "units_per_launch": units, "ops_per_unit": per_unit,
                     "peak_source": peak_src,
                     # what a kernel visiting every leaf would have to sustain for this rate
                     "leaf_equivalent": {"ops_per_subgraph": ops_per_subgraph(k), "achieved": leaf_achieved,
                                         "frac": leaf_achieved / peak_gops},
                     # measured issue-slot and cache throughput of the same kernel (ncu)
                     "ncu_counters": counters},
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_rate(e2e_units, e2e_max), "unit": UNIT,
                "h2d_bytes_per_step": int(rowptr_np.nbytes + col_np.nbytes),
                "d2h_bytes_per_step": int(acc.NUM_CLASSES[k] * 8)},
        "gpu_launches": int(stats["launches"]) * steps,
        "clocks": clocks,
        "stages_ms": {"how": "separate pass, per-stage events, kernels launched one by one",
                      "build": statistics.mean(build_ms), "enumerate": statistics.mean(enum_ms),
                      "enumerate_phase1": statistics.mean(p1_ms), "enumerate_phase2": statistics.mean(p2_ms),
                      "step_median": statistics.median(step_ms)},
        "parity_vs_stored_oracle_counts": parity,
        # once per k per device, outside the timed steps
        "table_build_ms": table_ms,
        "work": {"chunks": stats["chunks"], "undirected_edges": stats["undirected_edges"],
                 "max_degree": stats["max_degree"], "blocks": stats["blocks"]},
    }


def bench_line(env, rec, steps, warmup):
    """The contract's JSON line around one measurement record."""
    line = {"metric": METRIC, "value": rec["value"], "unit": rec["unit"], "n_gpus": env.world, "steps": steps,
            "warmup": warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic"}
    line.update({k: v for k, v in rec.items() if k not in line})
    return line


def run_ours(args):
    env = GpuEnv()
    rec = measure_single(env, args.workload, args.steps, args.warmup, args.mode, args.schedule,
                         not args.no_cpu_baseline, adjacency=args.adjacency)
    subs = None
    if args.workload == DEFAULT_WORKLOAD and not args.headline_only:
        # every other workload of the benchmark set, each under its own
        # clock samples, in the same run
        subs = {}
        for w in ("er_n1000_m5000_k3", "regulatory_n5000_m15000_k5"):
            r = measure_single(env, w, args.steps, args.warmup, args.mode, "", not args.no_cpu_baseline)
            if r is not None:
                subs[w] = r
        r = measure_batch(env, max(3, min(args.steps, 10)), args.warmup, not args.no_cpu_baseline, cpu_budget_s=5.0)
        if r is not None:
            subs[BATCH_WORKLOAD] = r
        alone = {}
        for rate in (200.0, 50.0):
            r = measure_serving(env, args.sub_serve_seconds, rate, args.slots, args.mem_budget_gb, args.serve_policy,
                                args.serve_aging_s, alone)
            if r is not None:
                subs[f"{SERVING_WORKLOAD}_{int(rate)}_per_s"] = r
    if env.rank == 0:
        line = bench_line(env, rec, args.steps, args.warmup)
        if subs is not None:
            line["sub_records"] = subs
        print(json.dumps(line), flush=True)
    env.close()
    return 0


def batch_graphs():
    graphs = []
    for b in range(synth.BATCH_BASES):
        base = synth.batch_base(b)
        graphs.append(base)
        graphs.extend(synth.batch_randomisation(base, b, i) for i in range(synth.BATCH_RANDOMISATIONS))
    return graphs


def batch_cpu_baseline(graphs, budget_s):
    """The oracle counting graphs of the batch (taken round-robin over the
    bases, so the sample has the batch's size mix) until about budget_s
    seconds; graphs/s."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    oracle.table(4)
    R1 = synth.BATCH_RANDOMISATIONS + 1
    order = [b * R1 + i for i in range(R1) for b in range(synth.BATCH_BASES)]
    t0 = time.perf_counter()
    done = 0
    while done < len(order) and time.perf_counter() - t0 < budget_s:
        g = graphs[order[done]]
        oracle.count(g.n, g.src, g.dst, 4, threads=threads)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "graphs/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} of the {len(graphs)} graphs (round-robin over the {synth.BATCH_BASES} bases), "
                      f"ESU count each, {dt:.1f} s"}


def measure_batch(env, steps, warmup, cpu_baseline=True, cpu_budget_s=10.0):
    """Batched k=4 workload: 8 Chung-Lu bases x (1 + 500 randomisations) =
    4008 graphs counted by one prepared batch, replayed from a captured CUDA
    graph; compared with one acc_motif_count launch sequence per graph."""
    torch, acc, dev, dist = env.torch, env.acc, env.dev, env.dist
    graphs = batch_graphs()
    B, R1 = len(graphs), synth.BATCH_RANDOMISATIONS + 1
    tens = []
    for g in graphs:
        r, c = g.csr()
        tens.append((torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev), g.n))
    counter = acc.Counter(env.local)
    stream = torch.cuda.Stream(dev)
    counts = torch.zeros((B, 199), dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        counter.prepare_batch(tens, 4, stream=stream)
        # the schedule is tuned once per prepared batch, outside the timed region
        sched = counter.autotune_batch(stream=stream)
        for _ in range(warmup):
            counter.run_batch(counts=counts, status=status, stream=stream)
    torch.cuda.synchronize(dev)
    if int(status.item()) != 0:
        raise RuntimeError(f"batch failed: {acc.acc_strerror(int(status.item()))}")
    eager = counts.clone()
    stats = counter.last_stats()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        counter.run_batch(counts=counts, status=status, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(env.local) if env.rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            graph.replay()
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    local_s = sum(s.elapsed_time(e) for s, e in ev) / 1000.0
    if not torch.equal(counts, eager) or int(status.item()) != 0:
        raise RuntimeError("graph replay differs from the eager batch")
    total = int(counts.sum().item())
    max_s = reduce_max(dist, local_s, dev)
    value = whole_job_rate(reduce_sum(dist, float(B) * steps, dev), max_s)
    sub_rate = whole_job_rate(reduce_sum(dist, float(total) * steps, dev), max_s)
    # the enumeration stage alone (per-stage events, launched one by one)
    counter.set_timing(True)
    enum_ms = []
    with torch.cuda.stream(stream):
        for i in range(3):
            flush.fill_(i & 0xFF)
            counter.run_batch(counts=counts, status=status, stream=stream)
            enum_ms.append(counter.last_timing()[1])
    counter.set_timing(False)
    # Z-scores of each base against its randomisations
    z = counter.zscores(counts, synth.BATCH_BASES, R1, 4)
    torch.cuda.synchronize(dev)
    # one acc_motif_count launch sequence per graph, same GPU, same graphs
    single = torch.zeros(199, dtype=torch.int64, device=dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for r, c, n in tens[:8]:
            counter.count(r, c, n, 4, counts=single, status=status, stream=stream)
        flush.fill_(7)
        t0.record(stream)
        for r, c, n in tens:
            counter.count(r, c, n, 4, counts=single, status=status, stream=stream)
        t1.record(stream)
    torch.cuda.synchronize(dev)
    single_rate = B / (t0.elapsed_time(t1) / 1000.0)
    counter.close()
    if env.rank != 0:
        return None
    gold = os.path.join(ROOT, "tests", "golden", "batch_k4.txt")
    parity = None
    if os.path.exists(gold):
        rows = [ln.split() for ln in open(gold) if ln.strip() and not ln.startswith("#")]
        host = counts.cpu().numpy()
        zh = z.cpu().numpy()
        parity = all(
            hashlib.sha256(np.ascontiguousarray(host[b * R1:(b + 1) * R1], dtype="<i8").tobytes()).hexdigest()
            == rows[b][4]
            and all(float(x).hex() == w or (np.isnan(x) and w == "nan") for x, w in zip(zh[b], rows[b][6:]))
            for b in range(len(rows)))
    peak_gops, peak_src = issue_peak_gops(env)
    enum_s = statistics.mean(enum_ms) / 1000.0
    scanned = int(stats["scanned_entries"])
    achieved = ops_per_scanned_entry(4) * scanned / enum_s / 1e9
    cpu = batch_cpu_baseline(graphs, cpu_budget_s) if (env.world == 1 and cpu_baseline) else None
    return {
        "value": value, "unit": "graphs/s", "steps": steps, "warmup": warmup, "ms_per_step": 1000.0 * max_s / steps,
        "config": {"workload": BATCH_WORKLOAD, "k": 4, "graphs": B, "bases": synth.BATCH_BASES,
                   "randomisations_per_base": synth.BATCH_RANDOMISATIONS, "subgraphs_per_step": total,
                   "l2": "flushed between timed steps (256 MiB device write)",
                   "launch": "prepared batch replayed from a captured CUDA graph",
                   "schedule": {"light": sched[0], "target": sched[1], "autotuned": True},
                   "parallelism": f"replicas{env.world}"},
        "subgraphs_per_s": sub_rate,
        "one_graph_per_launch": {"value": single_rate, "unit": "graphs/s",
                                 "how": "acc_motif_count per graph, same stream, same GPU"},
        "batched_over_single": value / single_rate,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": None, "kernel": "k_enum<4> (phase 1 + phase 2)",
                     "work_unit": "neighbour entries scanned by the last two levels", "units_per_launch": scanned,
                     "ops_per_unit": ops_per_scanned_entry(4), "peak_source": peak_src,
                     "enumerate_ms": statistics.mean(enum_ms)},
        "cpu_baseline": cpu,
        "zscores_finite": int(np.isfinite(z.cpu().numpy()).sum()),
        "gpu_launches": int(stats["launches"]) * steps,
        "clocks": clocks,
        "parity_vs_stored_oracle_counts": parity,
    }


def run_batch_bench(args):
    env = GpuEnv()
    steps = max(1, args.steps)
    rec = measure_batch(env, steps, args.warmup, not args.no_cpu_baseline)
    if env.rank == 0:
        print(json.dumps(bench_line(env, rec, steps, args.warmup)), flush=True)
    env.close()
    return 0


def run_significance_bench(args):
    """The significance step on the device for the batched k=4 workload: each
    step randomises 8 Chung-Lu bases x 500 copies (3m double-edge swap
    attempts each), counts the 4008 graphs as one batch and scores every base
    against its copies; the three calls are replayed from one CUDA graph."""
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    from paper_1203_3415_gb300 import build as lib_build
    if rank == 0 or world == 1:
        lib_build.build()
    if dist is not None:
        dist.barrier()
    import paper_1203_3415_gb300 as acc

    bases = [synth.batch_base(b) for b in range(synth.BATCH_BASES)]
    graphs = []
    for g in bases:
        r, c = g.csr()
        graphs.append((torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev), g.n))
    R = synth.BATCH_RANDOMISATIONS
    G, B = len(graphs), len(graphs) * (R + 1)
    seeds = [1_000_000 * (b + 1) for b in range(G)]
    counter = acc.Counter(local)
    stream = torch.cuda.Stream(dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    counts = torch.zeros((B, 199), dtype=torch.int64, device=dev)
    z = torch.zeros((G, 199), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    m_total = sum(int(c.numel()) for _, c, _ in graphs)
    out = torch.empty(R * m_total, dtype=torch.int32, device=dev)
    accepted = torch.empty((G, R), dtype=torch.int64, device=dev)

    rmode = acc.ACC_RAND_MUTUAL if args.rand_mode == "mutual" else acc.ACC_RAND_SWAP

    def step():
        counter.randomise(graphs, R, seeds, 3, mode=rmode, out=out, accepted=accepted, status=status, stream=stream)
        counter.run_batch(counts=counts, status=status, stream=stream)
        acc._check(acc.acc_motif_zscores(counts.data_ptr(), G, R + 1, 4, stream.cuda_stream, z.data_ptr()),
                   "acc_motif_zscores")

    with torch.cuda.stream(stream):
        counter.randomise(graphs, R, seeds, 3, mode=rmode, out=out, accepted=accepted, status=status, stream=stream)
        batch = []
        for g, cps in zip(graphs, acc.Counter.copies(graphs, R, out)):
            batch.append(g)
            batch.extend(cps)
        counter.prepare_batch(batch, 4, stream=stream)
        sched = counter.autotune_batch(stream=stream)
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    if int(status.item()) != 0:
        raise RuntimeError(f"significance step failed: {acc.acc_strerror(int(status.item()))}")
    eager = counts.clone()
    # the randomisation alone, eager, for its share of the step
    rt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    with torch.cuda.stream(stream):
        for a, b in rt:
            flush.fill_(3)
            a.record(stream)
            counter.randomise(graphs, R, seeds, 3, mode=rmode, out=out, accepted=accepted, status=status,
                              stream=stream)
            b.record(stream)
    torch.cuda.synchronize(dev)
    rand_ms = min(a.elapsed_time(b) for a, b in rt)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    steps = max(1, args.steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            graph.replay()
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    local_s = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    if not torch.equal(counts, eager) or int(status.item()) != 0:
        raise RuntimeError("graph replay differs from the eager significance step")
    total = int(counts.sum().item())
    attempts = 3 * R * m_total
    acc_swaps = int(accepted.sum().item())
    max_s = reduce_max(dist, local_s, dev)
    value = whole_job_rate(reduce_sum(dist, float(B) * steps, dev), max_s)
    if rank != 0:
        counter.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0
    gold = os.path.join(ROOT, "tests", "golden", "batch_k4.txt")
    parity = None
    if os.path.exists(gold) and rmode == acc.ACC_RAND_SWAP:  # stored for the double-edge swaps
        import hashlib
        rows = [ln.split() for ln in open(gold) if ln.strip() and not ln.startswith("#")]
        host = counts.cpu().numpy()
        zh = z.cpu().numpy()
        parity = all(
            hashlib.sha256(np.ascontiguousarray(host[b * (R + 1):(b + 1) * (R + 1)], dtype="<i8").tobytes())
            .hexdigest() == rows[b][4]
            and all(float(x).hex() == w or (np.isnan(x) and w == "nan") for x, w in zip(zh[b], rows[b][6:]))
            for b in range(len(rows)))
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = significance_cpu_baseline(bases)
    line = {
        "metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * max_s / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": SIGNIFICANCE_WORKLOAD, "k": 4, "graphs": B, "bases": G,
                   "randomisations_per_base": R, "swap_attempts_per_copy": "3m",
                   "randomisation": "mutual arcs kept" if rmode == acc.ACC_RAND_MUTUAL else "double-edge swaps",
                   "subgraphs_per_step": total,
                   "l2": "flushed between timed steps (256 MiB device write)",
                   "launch": "randomise + batched count + Z-scores replayed from one captured CUDA graph",
                   "schedule": {"light": sched[0], "target": sched[1], "autotuned": True},
                   "parallelism": f"replicas{world}"},
        "randomise_ms": rand_ms,
        "swap_attempts_per_s": attempts / (rand_ms / 1000.0),
        "accepted_swaps": acc_swaps,
        "swap_attempts": attempts,
        "subgraphs_per_s": total * steps / max_s,
        "gpu_launches": (2 + counter.last_stats()["launches"] + 1) * steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "parity_vs_stored_oracle_counts_and_z": parity,
    }
    print(json.dumps(line), flush=True)
    counter.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def significance_cpu_baseline(bases, budget_s=10.0):
    """The oracle's copy and count of randomised copies of the smallest base,
    one after another until about budget_s seconds."""
    import oracle
    oracle.build()
    b = min(range(len(bases)), key=lambda i: bases[i].n)
    g = bases[b]
    rowptr, col = g.csr()
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(rowptr))
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s:
        dst, _ = oracle.swap_randomise(g.n, rowptr, col, 3 * g.m, 1_000_000 * (b + 1) + done)
        oracle.count(g.n, src, dst, 4, threads=threads)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "graphs/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} randomised copies of base {b} (n={g.n}, m={g.m}): swaps and ESU count each"}


def serving_alone_times(env, graphs, tens, combos):
    """GPU seconds and subgraphs of each (graph, k) in combos counted alone
    through acc_motif_count on the whole GPU, one after another (CUDA events
    on the launching stream; the workspace is first grown for the largest
    graph, outside the timed counts)."""
    torch, acc = env.torch, env.acc
    counter = acc.Counter(env.local)
    stream = torch.cuda.current_stream(env.dev)
    big = max(range(len(graphs)), key=lambda i: graphs[i].n)
    for k in (3, 4, 5):
        counter.prepare(k)
    counter.count(tens[big][0], tens[big][1], graphs[big].n, 3)
    out = {}
    counts = torch.zeros(9364, dtype=torch.int64, device=env.dev)
    for gi, k in sorted(combos):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c = counter.count(tens[gi][0], tens[gi][1], graphs[gi].n, k, counts=counts[:acc.NUM_CLASSES[k]],
                          stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(env.dev)
        out[(gi, k)] = (e0.elapsed_time(e1) / 1000.0, int(c.sum().item()))
    counter.close()
    return out


def measure_serving(env, window_s, rate, slots, mem_budget_gb, policy, aging_s, alone=None):
    """Serving workload: 64 resident directed Chung-Lu graphs (n log-uniform
    in [100, 50000], mean out-degree 4-10), a Poisson stream of requests at
    `rate` per second with k in {3: 50%, 4: 35%, 5: 15%}, replayed in real
    time against the request server; latency = completion - scheduled
    arrival."""
    torch, acc, dev, dist = env.torch, env.acc, env.dev, env.dist
    specs = synth.serving_pool_specs()
    graphs = [synth.serving_graph(sp) for sp in specs]
    reqs = synth.serving_requests(duration_s=window_s, rate=rate)
    srv = acc.Server(env.local, slots=slots, mem_budget_bytes=int(mem_budget_gb * (1 << 30)))
    srv.set_policy(acc.ACC_SERVE_FIFO if policy == "fifo" else acc.ACC_SERVE_SHORTEST, aging_s)
    tens = []
    for g in graphs:
        r, c = g.csr()
        tens.append((torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev)))
    ids = [srv.add_graph(r, c, g.n) for (r, c), g in zip(tens, graphs)]
    srv.reserve()
    # warm-up: one request per k on the smallest graph
    for k in (3, 4, 5):
        srv.submit(ids[int(np.argmin([g.n for g in graphs]))], k)
    srv.drain()
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(env.local) if env.rank == 0 else None
    if sampler:
        sampler.start()
    t0 = time.perf_counter()
    rids, arrivals = [], []
    busy, t_last, was_busy = 0.0, 0.0, False
    i = 0
    while i < len(reqs):
        now = time.perf_counter() - t0
        if was_busy:
            busy += now - t_last
        t_last = now
        while i < len(reqs) and reqs[i][0] <= now:
            t_arr, gid, k = reqs[i]
            rids.append(srv.submit(ids[gid], k))
            arrivals.append((t_arr, now, gid, k))
            i += 1
        running, _ = srv.progress()
        was_busy = running > 0
        if i < len(reqs):
            wait = reqs[i][0] - (time.perf_counter() - t0)
            if wait > 0.0005:
                time.sleep(min(wait, 0.001))
    while True:
        now = time.perf_counter() - t0
        if was_busy:
            busy += now - t_last
        t_last = now
        running, queued = srv.progress()
        was_busy = running > 0
        if running == 0 and queued == 0:
            break
    srv.drain()
    t_end = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    lat, units, by_k = [], 0, {3: [], 4: [], 5: []}
    failed = 0
    for rid, (t_arr, t_sub, gid, k) in zip(rids, arrivals):
        st, counts, l = srv.poll(rid)
        if st != acc.ACC_REQ_DONE:
            failed += 1
            continue
        total_l = l + (t_sub - t_arr)  # server latency plus the submission lag
        lat.append(total_l)
        by_k[k].append(total_l)
        units += int(counts.sum())
    srv.close()
    lat = np.array(lat)
    local_rate = units / t_end
    # the same requests counted one at a time on the whole GPU
    one_at_a_time = None
    if alone is not None:
        missing = {(g, k) for _, g, k in reqs} - set(alone)
        if missing:
            alone.update(serving_alone_times(env, graphs, tens, missing))
        gpu_s = sum(alone[(g, k)][0] for _, g, k in reqs)
        sub = sum(alone[(g, k)][1] for _, g, k in reqs)
        one_at_a_time = {"value": sub / gpu_s, "unit": UNIT, "requests_per_s": len(reqs) / gpu_s,
                         "gpu_seconds": gpu_s,
                         "how": "each distinct (graph, k) of the request list counted alone by acc_motif_count "
                                "(CUDA events), summed over the requests"}
    value = reduce_sum(dist, local_rate, dev) if dist is not None else local_rate
    if env.rank != 0:
        return None
    pct = lambda a, q: float(np.percentile(a, q) * 1000.0) if len(a) else None  # noqa: E731
    return {
        "value": value, "unit": UNIT, "steps": len(rids), "warmup": 3,
        "ms_per_step": 1000.0 * t_end / max(1, len(rids)),
        "config": {"workload": SERVING_WORKLOAD, "graphs": len(graphs), "requests": len(rids),
                   "arrival_rate_per_s": rate, "window_s": window_s, "slots": slots,
                   "policy": policy, "aging_s": aging_s,
                   "mem_budget_gb": mem_budget_gb, "parallelism": f"replicas{env.world}"},
        "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": pct(lat, 100),
                       "by_k_p50": {str(k): pct(np.array(v), 50) for k, v in by_k.items()},
                       "by_k_p99": {str(k): pct(np.array(v), 99) for k, v in by_k.items()}},
        "completed_per_s": len(lat) / t_end, "offered_per_s": len(rids) / window_s,
        "failed": failed, "wall_s": t_end,
        "gpu_busy_frac": busy / t_end if t_end > 0 else None,
        "subgraphs_served": units,
        "one_request_at_a_time": one_at_a_time,
        "served_over_one_at_a_time": (value / one_at_a_time["value"]) if one_at_a_time else None,
        "clocks": clocks,
        "parity": "every served result equals the oracle's: tests/test_gpu_serving.py",
    }


def run_serving_bench(args):
    env = GpuEnv()
    rec = measure_serving(env, args.serve_seconds, args.serve_rate, args.slots, args.mem_budget_gb,
                          args.serve_policy, args.serve_aging_s, {})
    if env.rank == 0:
        print(json.dumps(bench_line(env, rec, rec["steps"], 3)), flush=True)
    env.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, SERVING_WORKLOAD,
                                                               SIGNIFICANCE_WORKLOAD],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serving: arrival window")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serving: Poisson arrival rate per second")
    ap.add_argument("--sub-serve-seconds", type=float, default=5.0,
                    help="serving window of the default run's serving sub-records (200 and 50 requests/s)")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: print the headline line without the other workloads' sub-records")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent requests")
    ap.add_argument("--mem-budget-gb", type=float, default=96.0, help="serving: workspace budget")
    ap.add_argument("--reference-roots", type=int, default=0,
                    help="reference arm: ESU roots per step (0: all roots, the whole workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-policy", choices=["shortest", "fifo"], default="shortest",
                    help="serving admission order: smallest aged work estimate first, or submission order")
    ap.add_argument("--serve-aging-s", type=float, default=1.0)
    ap.add_argument("--adjacency", choices=["auto", "dense", "hash", "sparse"], default="auto",
                    help="count mode: pair-state probes on the dense block, hashed tables, or hashed tables over "
                         "lists built without the block (same counts)")
    ap.add_argument("--schedule", default="",
                    help="enumeration schedule LIGHT,TARGET for the single-graph workloads (default: the kernels')")
    ap.add_argument("--rand-mode", choices=["swap", "mutual"], default="swap",
                    help="significance workload: double-edge swaps, or swaps that keep mutual arcs mutual")
    ap.add_argument("--mode", choices=["count", "enumerate", "formula", "auto"], default="auto",
                    help="last two levels counted by state-vector groups, every leaf enumerated, the paper's "
                         "formulas, or the library's automatic choice (formulas for k=3 up to 16384 vertices, "
                         "else the count mode)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        if args.workload in (BATCH_WORKLOAD, SERVING_WORKLOAD, SIGNIFICANCE_WORKLOAD):
            args.workload = DEFAULT_WORKLOAD
        return run_reference(args)
    if args.workload == BATCH_WORKLOAD:
        return run_batch_bench(args)
    if args.workload == SERVING_WORKLOAD:
        return run_serving_bench(args)
    if args.workload == SIGNIFICANCE_WORKLOAD:
        return run_significance_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
