#!/usr/bin/env python
"""Throughput of the match-count top-k hot path on one GB300 (or N replicas).

One step = one batch through the whole path: query compile (keyword look-up,
count bounds), the fused postings scan + c-PQ kernel and the per-query
top-k merge, for 1024 LSH queries against 1,000,000 objects x 256 keywords
(k = 100).  ``value`` is queries/s with the inputs already in HBM; ``e2e``
is the same through the C ABI from pinned host buffers with the copies
inside the timed region.  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl genie|reference]
Under torchrun (N > 1) every rank holds an index replica and runs its own
1024 queries (weak scaling); only the timing uses a (gloo) collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "match-count top-k queries/s and posting entries/s (% HBM peak); p99 latency"
UNIT = "queries/s"
N_OBJECTS, N_QUERIES, K = 1_000_000, 1024, 100
WORKLOAD = ("lsh-1m: 1,000,000 objects x 256 p-stable LSH keywords (bucket width 4, "
            "bucket mod 8192), 1024 queries from the same 1000-component mixture, k=100")
REF_SAMPLE = 32      # oracle queries per reference step
CPU_SAMPLE = 64  # oracle queries for the cpu_baseline object


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["genie", "reference"], default="genie")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["lsh1m", "lsh4m-learned", "lsh4m-parts",
                                           "sets4m-batched", "serving", "seq1m"],
                    default="lsh1m",
                    help="lsh1m: the headline batch; lsh4m-learned: plain vs learned-seed "
                         "search on 4M objects / 4096 queries (k=100); lsh4m-parts: the 4M "
                         "objects as 4 host-resident index parts, 1024 queries, against one "
                         "device-resident index; seq1m: sequence search by ordered 3-grams "
                         "with edit-distance verification on 1M sequences; sets4m-batched: plain "
                         "launch vs the persistent graph-captured batch on 4M Zipf sets / 8192 "
                         "queries (k=10); serving: continuous-batching server on 8M x 64 Zipf "
                         "sets, Poisson arrivals at a swept rate, k in {1, 10, 100}")
    ap.add_argument("--queries", type=int, default=N_QUERIES,
                    help="queries per batch (the workload is defined at 1024; smaller "
                         "values are for profiling captures)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(rank: int, world: int, n_queries: int = N_QUERIES):
    import synth
    w = synth.lsh(N_OBJECTS, n_queries * world, K, config=2)
    if world > 1:
        w = w.subset(np.arange(rank * n_queries, (rank + 1) * n_queries))
    return w


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons, each stamped with
    the host clock when it arrives; the summary keeps the samples taken inside
    the timed region (between mark_begin() and mark_end())."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.thread = None
        self.lines = []
        self.t_begin = self.t_end = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.monotonic() + 5.0  # let the sampler run before the timed region
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.01)

    def mark_begin(self):
        self.t_begin = time.monotonic()

    def mark_end(self):
        self.t_end = time.monotonic()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.INTERVAL_MS / 1e3)  # the sample that covers the region's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        stamped = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                stamped.append((t, parts))
        window = "timed region"
        if self.t_begin is not None and self.t_end is not None:
            slack = self.INTERVAL_MS / 1e3
            inside = [p for t, p in stamped if self.t_begin <= t <= self.t_end + slack]
        else:
            inside = []
        if not inside:  # a region shorter than the sampling interval: the samples around it
            inside = [p for _, p in stamped]
            window = "whole run (no sample fell inside the timed region)"
        rows = inside
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows), "window": window,
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                                   default=None)}


KERNEL_SOURCES = ("cpq_device.cuh", "device_util.cuh", "search.cu")


def kernel_source_sha() -> str:
    """sha256 of the scan kernel's code: the KERNEL_SOURCES concatenated in
    order, with comments removed and every run of blank space made one space
    (so that a comment edit does not retire the profile)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1603_08390_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def traffic_from_profile():
    """Per-launch DRAM bytes of the scan kernel from the committed ncu summary,
    valid only while the kernel sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "scan_cpq_lsh1m_ncu.md")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        text = f.read()
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b:
        return None
    return float(m_b.group(1)) if kernel_source_sha() == m_sha.group(1) else None


def cpu_baseline(w, n_sample: int) -> dict:
    import oracle
    sub = w.subset(np.arange(n_sample))
    oracle.topk(sub.subset(np.arange(2)))  # load and warm
    t0 = time.perf_counter()
    oracle.topk(sub)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "first %d of the %d queries, brute force over all %d objects "
                      "(%.1f s wall)" % (n_sample, w.n_queries, w.n_objects, dt)}


def config_dict(w, world, entries):
    return {"workload": WORKLOAD, "n_objects": w.n_objects, "n_queries": w.n_queries, "k": K,
            "postings": int(w.nnz), "entries_per_step": int(entries),
            "l2": "inputs larger than L2 (index %.2f GB vs 126 MB L2), not flushed" % (
                (w.nnz * 4 + (w.vocab + 1) * 8 + w.vocab * 33 * 4) / 1e9),
            "parallelism": "replicas x%d (query batches, no data-path collective)" % world}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    w = workload(0, 1)
    sub = w.subset(np.arange(REF_SAMPLE))
    oracle.topk(sub.subset(np.arange(2)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.topk(sub)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    step_s = sum(times) / len(times)
    value = REF_SAMPLE / step_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "impl": "reference",
            "config": config_dict(w, 1, 0),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": "%d queries per step (first %d of %d), brute force over "
                                       "%d objects" % (REF_SAMPLE, REF_SAMPLE, w.n_queries,
                                                       w.n_objects)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_genie(args, rank, world, local):
    import torch
    from paper_1603_08390_gb300 import _build, genie, runner

    _build.build()
    torch.cuda.set_device(local)
    w = workload(rank, world, args.queries)
    idx = runner.build_index(w)
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    out = runner.Outputs(Q, K)
    stream = torch.cuda.current_stream()

    def step(events=None):
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        opts = genie.make_opts(scan_events=events) if events is not None else None
        genie.genie_search(idx, qs, K, out.ids, out.counts, out.n_valid, opts=opts, stream=stream)
        return qs

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        qs = step()
    torch.cuda.synchronize()
    entries = qs.n_entries
    del qs
    scan_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    for b, e in scan_ev:  # materialise the events before handing them to the library
        b.record(stream)
        e.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark_begin()
    step_ev[0].record(stream)
    for i in range(args.steps):
        step(scan_ev[i])
        step_ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(world)
    clk = clocks.stop()
    total_ms = step_ev[0].elapsed_time(step_ev[-1])
    per_step = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    scan_ms = statistics.mean(b.elapsed_time(e) for b, e in scan_ev)
    total_ms = max_over_ranks(total_ms, world)
    value = Q * world * args.steps / (total_ms / 1e3)

    # end to end through the C ABI from pinned host memory
    h_q_off = torch.from_numpy(w.q_off.view(np.int32)).pin_memory()
    h_q_kw = torch.from_numpy(w.q_kw.view(np.int32)).pin_memory()
    h_ids = torch.empty(Q * K, dtype=torch.int32).pin_memory()
    h_counts = torch.empty(Q * K, dtype=torch.int32).pin_memory()
    h_nv = torch.empty(Q, dtype=torch.int32).pin_memory()
    e_q_off = torch.empty_like(d_q_off)
    e_q_kw = torch.empty_like(d_q_kw)

    def e2e_step():
        e_q_off.copy_(h_q_off, non_blocking=True)
        e_q_kw.copy_(h_q_kw, non_blocking=True)
        qs = genie.genie_make_queries(idx, e_q_off, e_q_kw, Q, stream)
        genie.genie_search(idx, qs, K, out.ids, out.counts, out.n_valid, stream=stream)
        h_ids.copy_(out.ids, non_blocking=True)
        h_counts.copy_(out.counts, non_blocking=True)
        h_nv.copy_(out.n_valid, non_blocking=True)

    for _ in range(max(3, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    h2d = (Q + 1) * 4 + int(w.q_off[-1]) * 4
    d2h = 2 * Q * K * 4 + Q * 4

    # the same batch with the Gate idle (count, then select from the counters):
    # the on-chip form of the paper's GEN-SPQ comparison, timed after the run
    ng_opts = genie.make_opts(flags=genie.GENIE_SEARCH_NO_GATE)

    def step_no_gate():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        genie.genie_search(idx, qs, K, out.ids, out.counts, out.n_valid, opts=ng_opts,
                           stream=stream)

    step_no_gate()
    ng_ms, _ = timed_steps(step_no_gate, max(3, args.steps // 3), stream)
    ng_ms /= max(3, args.steps // 3)
    cal = genie.genie_calibrate()

    # c-PQ counters from one more (untimed) pass
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    kernel = genie.genie_search_shape(idx, qs, K).kernel_name()
    genie.genie_search(idx, qs, K, out.ids, out.counts, out.n_valid,
                       opts=genie.make_opts(d_stats=stats), stream=stream)
    st = stats.cpu().numpy()
    cpq = {"gate_passes_per_posting": float(st[0]) / entries, "ht_inserts": int(st[1]),
           "blocks": int(st[4]), "blocks_bitmap_fallback": int(st[2]),
           "blocks_gateless_unseeded": int(st[6]), "bad_ids": int(st[5])}
    del qs

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    algo_bytes = 4.0 * entries  # one 4-byte object id read per posting scanned
    achieved = algo_bytes / (scan_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_dict(w, world, entries),
        "entries_per_s": entries * world * args.steps / (total_ms / 1e3),
        "latency_ms": {"batch_p50": float(np.percentile(per_step, 50)),
                       "batch_p99": float(np.percentile(per_step, 99))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_from_profile(),
                     "kernel": kernel, "peak_kind": peak_kind + " hbm_gbs",
                     "scan_ms": scan_ms, "algorithmic_bytes_per_launch": algo_bytes},
        "smem_atomic_roofline": {
            "bound": "shared-memory atomic adds (one per posting)",
            "achieved": entries / (scan_ms / 1e3), "peak": cal.smem_atomics_per_s,
            "unit": "updates/s", "frac": entries / (scan_ms / 1e3) / cal.smem_atomics_per_s,
            "peak_kind": "measured by genie_calibrate on this GPU"},
        "ablation_no_gate": {"ms_per_step": ng_ms, "value": Q * world / (ng_ms / 1e3),
                             "c_pq_vs_no_gate": ng_ms / (total_ms / args.steps)},
        "e2e": {"value": Q * world * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "cpq": cpq,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, CPU_SAMPLE)
    print(json.dumps(line), flush=True)


def timed_steps(step, steps, stream):
    """CUDA-event time of `steps` calls of step(); returns (total ms, per-step ms)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]), per


def run_learned(args, rank, world, local):
    """Plain vs learned-seed search on the 4M-object LSH workload."""
    import torch
    import synth
    from paper_1603_08390_gb300 import _build, genie, learned, runner

    _build.build()
    torch.cuda.set_device(local)
    k = 100
    w = synth.config(4)
    idx = runner.build_index(w)
    t0 = time.perf_counter()
    tq_off, tq_kw = synth.lsh_training_queries(100_000, config=4)
    tr = learned.train_predictor(idx, tq_off, tq_kw, k, epochs=20, batch=256, lr=2e-3)
    train_s = time.perf_counter() - t0
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    stream = torch.cuda.current_stream()
    out_p, out_l = runner.Outputs(Q, k), runner.Outputs(Q, k)
    seeds = torch.empty(Q, dtype=torch.int32, device="cuda")

    def plain():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        genie.genie_search(idx, qs, k, out_p.ids, out_p.counts, out_p.n_valid, stream=stream)

    def seeded(stats=None):
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        tr["mlp"].seeds(qs, tr["margin"], seeds, stream)
        genie.genie_search(idx, qs, k, out_l.ids, out_l.counts, out_l.n_valid,
                           opts=genie.make_opts(d_seed=seeds, d_stats=stats), stream=stream)

    for _ in range(args.warmup):
        plain()
        seeded()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.mark_begin()
    p_ms, _ = timed_steps(plain, args.steps, stream)
    l_ms, per = timed_steps(seeded, args.steps, stream)
    clocks.mark_end()
    clk = clocks.stop()
    st_p = torch.zeros(8, dtype=torch.int64, device="cuda")
    st_l = torch.zeros(8, dtype=torch.int64, device="cuda")
    qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    genie.genie_search(idx, qs, k, out_p.ids, out_p.counts, out_p.n_valid,
                       opts=genie.make_opts(d_stats=st_p), stream=stream)
    seeded(st_l)
    a, b = out_p.host(), out_l.host()
    identical = all(np.array_equal(a[key], b[key]) for key in a)
    sp, sl = st_p.cpu().numpy(), st_l.cpu().numpy()
    entries = qs.n_entries
    line = {
        "metric": METRIC, "value": Q * args.steps / (l_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": l_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "impl": "genie-learned",
        "config": {"workload": "lsh-4m learned threshold: 4,000,000 objects x 256 LSH keywords, "
                               "4096 queries, k=100; 64-128-1 bf16 MLP trained on 100k query / "
                               "k-th-count pairs from the plain search",
                   "n_objects": w.n_objects, "n_queries": Q, "k": k, "entries_per_step": int(entries)},
        "plain": {"value": Q * args.steps / (p_ms / 1e3), "ms_per_step": p_ms / args.steps,
                  "gate_passes": int(sp[0]), "ht_inserts": int(sp[1])},
        "learned": {"value": Q * args.steps / (l_ms / 1e3), "ms_per_step": l_ms / args.steps,
                    "gate_passes": int(sl[0]), "ht_inserts": int(sl[1]),
                    "reruns": int(sl[3]), "rerun_rate": float(sl[3]) / Q,
                    "batch_p50_ms": float(np.percentile(per, 50)),
                    "batch_p99_ms": float(np.percentile(per, 99))},
        "speedup_vs_plain": p_ms / l_ms, "identical_results": bool(identical),
        "training": {"seconds": train_s, "train_loss": tr["train_loss"], "margin": tr["margin"],
                     "n_train": tr["n_train"], "n_val": tr["n_val"],
                     "target_mean": tr["target_mean"]},
        "entries_per_s": entries * args.steps / (l_ms / 1e3),
        "gpu_launches": 5 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_parts(args, rank, world, local):
    """Multiple loadings (Sec. 3.4): the 4M-object LSH objects as four parts of
    1M held in pinned host memory, 1024 queries per batch, against one
    device-resident index of the same objects."""
    import torch
    import synth
    from paper_1603_08390_gb300 import _build, genie, runner

    _build.build()
    torch.cuda.set_device(local)
    k, P = 100, 4
    w = synth.config(4).subset(np.arange(N_QUERIES))
    N, Q = w.n_objects, w.n_queries
    parts = runner.build_parts(w, [(p * N // P, (p + 1) * N // P) for p in range(P)])
    info = parts.info
    idx = runner.build_index(w)
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    stream = torch.cuda.current_stream()
    out_p, out_d = runner.Outputs(Q, k), runner.Outputs(Q, k)

    def step_parts():
        parts.search(d_q_off, d_q_kw, Q, k, out_p.ids, out_p.counts, out_p.n_valid, stream=stream)

    def step_device():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        genie.genie_search(idx, qs, k, out_d.ids, out_d.counts, out_d.n_valid, stream=stream)

    for _ in range(max(3, args.warmup)):
        step_parts()
        step_device()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.mark_begin()
    p_ms, per = timed_steps(step_parts, args.steps, stream)
    d_ms, _ = timed_steps(step_device, args.steps, stream)
    clocks.mark_end()
    clk = clocks.stop()
    a, b = out_p.host(), out_d.host()
    identical = all(np.array_equal(a[key], b[key]) for key in a)
    qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    entries = qs.n_entries
    line = {
        "metric": METRIC, "value": Q * args.steps / (p_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": p_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "impl": "genie-parts",
        "config": {"workload": "lsh-4m multiple loadings: the 4,000,000 LSH objects (256 keywords "
                               "each) as 4 index parts of 1,000,000 in pinned host memory, copied "
                               "to the device part by part during each batch; 1024 queries, k=100",
                   "n_objects": N, "n_queries": Q, "k": k, "parts": P,
                   "entries_per_step": int(entries)},
        "h2d_bytes_per_step": int(info.host_bytes),
        "h2d_gb_per_s": info.host_bytes * args.steps / (p_ms / 1e3) / 1e9,
        "device_resident": {"value": Q * args.steps / (d_ms / 1e3), "ms_per_step": d_ms / args.steps,
                            "device_index_bytes": int(idx.device_bytes)},
        "parts_vs_device_resident": d_ms / p_ms, "identical_results": bool(identical),
        "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                       "batch_p99": float(np.percentile(per, 99))},
        "entries_per_s": entries * args.steps / (p_ms / 1e3),
        "gpu_launches": (4 * P + 2) * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_seq(args, rank, world, local):
    """Sequence search by ordered n-grams (Sec. 5.1): 1M sequences of 40-100
    characters, 1024 queries with 1-6 edits, K = 128 candidates, k = 1."""
    import torch
    import synth
    from paper_1603_08390_gb300 import _build, runner

    _build.build()
    torch.cuda.set_device(local)
    n, R, K, k = 3, 32, 128, 1
    seqs = synth.sequences(1_000_000, (40, 100), 26, N_QUERIES, (1, 6), config=6)
    si = runner.SeqIndex(seqs.s_off, seqs.s_chars, n, seqs.sigma, R)
    Q = seqs.n_queries
    d_q = (runner.to_dev(seqs.q_off), runner.to_dev(seqs.q_chars))
    out = runner.SeqOutputs(Q, K, k)
    stream = torch.cuda.current_stream()

    def step():
        runner.sa_search(si, seqs.q_off, seqs.q_chars, K, k, out=out, stream=stream, d_q=d_q)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.mark_begin()
    ms, per = timed_steps(step, args.steps, stream)
    clocks.mark_end()
    clk = clocks.stop()
    res = out.host()
    line = {
        "metric": METRIC, "value": Q * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "impl": "genie-sequences",
        "config": {"workload": "seq-1m: 1,000,000 sequences of 40-100 characters over 26 letters "
                               "(Zipf(1) frequencies), ordered 3-grams; 1024 queries, each a data "
                               "sequence with 1-6 random edits; top-128 candidates by match count, "
                               "verified by edit distance (k=1)",
                   "n_sequences": seqs.n_seqs, "n_queries": Q, "n": n, "K": K, "k": k},
        "certified_fraction": float(res["certified"].mean()),
        "examined_mean": float(res["examined"].mean()),
        "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                       "batch_p99": float(np.percentile(per, 99))},
        "gpu_launches": 7 * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        import oracle
        from oracle import sa
        n_s = 16
        sub = seqs.subset(np.arange(n_s))
        t0 = time.perf_counter()
        truth = sa.topk_ed(seqs.s_off, seqs.s_chars, sub.q_off, sub.q_chars, k)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n_s / cpu_s, "unit": UNIT, "cores": oracle.threads(),
                                "kind": "oracle",
                                "sample": "%d queries: brute-force edit distance to all 1M sequences"
                                          % n_s}
        cert = res["certified"][:n_s]
        line["sampled_certified_equal_truth"] = bool(np.all(
            res["ed"][:n_s][cert, 0] == truth["ed"][cert, 0]))
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local):
    """Plain one-launch-per-kernel search vs the persistent, graph-captured,
    autotuned batch on the 4M-object Zipf-set workload."""
    import torch
    import synth
    from paper_1603_08390_gb300 import _build, genie, runner

    _build.build()
    torch.cuda.set_device(local)
    k = 10
    w = synth.config(3)
    idx = runner.build_index(w)
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    stream = torch.cuda.current_stream()
    # autotune on a sample of 512 queries
    sample = w.subset(np.arange(0, Q, Q // 512)[:512])
    sq = runner.compile_queries(idx, sample)
    t0 = time.perf_counter()
    tuned = genie.genie_autotune(idx, sq, k, os.path.join(tempfile.gettempdir(), "genie_tune.txt"))
    tune_s = time.perf_counter() - t0
    qs0 = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    batch = genie.Batch(idx, Q, qs0.max_bound, k, tuned)
    entries = qs0.n_entries
    out_p, out_b = runner.Outputs(Q, k), runner.Outputs(Q, k)
    topt = genie.make_opts(block_shift=tuned.block_shift, threads=tuned.threads,
                           unroll=tuned.unroll, ht_slots=tuned.ht_slots)

    def plain():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        genie.genie_search(idx, qs, k, out_p.ids, out_p.counts, out_p.n_valid, stream=stream)

    def plain_tuned():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        genie.genie_search(idx, qs, k, out_p.ids, out_p.counts, out_p.n_valid, opts=topt,
                           stream=stream)

    def batched():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        batch.run(qs, out_b.ids, out_b.counts, out_b.n_valid, stream=stream)

    for _ in range(args.warmup):
        plain()
        batched()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.mark_begin()
    p_ms, _ = timed_steps(plain, args.steps, stream)
    pt_ms, _ = timed_steps(plain_tuned, args.steps, stream)
    b_ms, per = timed_steps(batched, args.steps, stream)
    clocks.mark_end()
    clk = clocks.stop()
    a, b = out_p.host(), out_b.host()
    identical = all(np.array_equal(a[key], b[key]) for key in a)
    rows = np.arange(0, Q, Q // 8)[:8]
    import oracle
    ref = oracle.topk(w.subset(rows))
    sampled_ok = all(np.array_equal(b["ids"][q, :int(ref["n_valid"][j])],
                                    ref["ids"][j, :int(ref["n_valid"][j])]) and
                     b["n_valid"][q] == ref["n_valid"][j] for j, q in enumerate(rows))
    line = {
        "metric": METRIC, "value": Q * args.steps / (b_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "impl": "genie-batched",
        "config": {"workload": "sets-4m batched: 4,000,000 Zipf(1.1) keyword sets of 16-256 over "
                               "a 2^20 vocabulary, 8192 queries of 8-512 keywords, k=10; one "
                               "persistent CUDA-graph launch per batch, autotuned shape",
                   "n_objects": w.n_objects, "n_queries": Q, "k": k, "entries_per_step": int(entries)},
        "plain_default": {"value": Q * args.steps / (p_ms / 1e3), "ms_per_step": p_ms / args.steps},
        "plain_tuned": {"value": Q * args.steps / (pt_ms / 1e3), "ms_per_step": pt_ms / args.steps},
        "batched": {"value": Q * args.steps / (b_ms / 1e3), "ms_per_step": b_ms / args.steps,
                    "batch_p50_ms": float(np.percentile(per, 50)),
                    "batch_p99_ms": float(np.percentile(per, 99))},
        "autotune": {"block_shift": tuned.block_shift, "threads": tuned.threads,
                     "unroll": tuned.unroll, "ht_slots": tuned.ht_slots,
                     "sample_ms": tuned.tuned_ms, "seconds": tune_s,
                     "from_cache": bool(tuned.from_cache)},
        "speedup_vs_plain_default": p_ms / b_ms, "identical_results": bool(identical),
        "oracle_sampled_queries_ok": bool(sampled_ok),
        "entries_per_s": entries * args.steps / (b_ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": 4.0 * entries / (b_ms / args.steps / 1e3) / 1e9,
                     "peak": measured_peaks()[0], "unit": "GB/s",
                     "frac": 4.0 * entries / (b_ms / args.steps / 1e3) / 1e9 / measured_peaks()[0],
                     "traffic": None, "kernel": "batch_cpq_kernel (whole step)"},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_serving(args, rank, world, local):
    """Continuous-batching server: saturation throughput and p50/p99 latency
    under Poisson arrivals at fractions of it (8M x 64 Zipf sets)."""
    import torch
    import synth
    from paper_1603_08390_gb300 import _build, genie, runner

    _build.build()
    torch.cuda.set_device(local)
    w = synth.sets(8_000_000, (64, 64), 1 << 22, 16, (8, 512), 10, config=5)  # the objects
    idx = runner.build_index(w)
    n_req = 4000
    q_off, q_kw, ks, _ = synth.serving_requests(n_req, 1.0, config=5)
    budget = 512 * w.n_objects  # counter bytes of 512 queries at 8 bits per object
    opts = genie.ServerOpts(bc_budget_bytes=budget, bits_per_object=8, max_batch=256,
                            max_query_keywords=512, k_max=100, streams=2)
    srv = genie.Server(idx, opts)
    # warm-up, then saturation: every request at t = 0
    srv.replay(q_off[:201] - q_off[0], q_kw[:q_off[200]], ks[:200], np.zeros(200))
    t0 = time.perf_counter()
    lat0, ids0, _, nv0 = srv.replay(q_off, q_kw, ks, np.zeros(n_req))
    sat_s = time.perf_counter() - t0
    sat_qps = n_req / sat_s
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    clocks.mark_begin()
    sweep = []
    rng = np.random.default_rng(123)
    for frac in (0.25, 0.5, 0.75, 0.9):
        rate = frac * sat_qps
        arrival = np.cumsum(rng.exponential(1.0 / rate, n_req))
        t1 = time.perf_counter()
        lat, ids, _, nv = srv.replay(q_off, q_kw, ks, arrival)
        wall = time.perf_counter() - t1
        same = bool(np.array_equal(nv, nv0) and all(
            np.array_equal(ids[i, :nv[i]], ids0[i, :nv0[i]]) for i in range(n_req)))
        sweep.append({"offered_qps": rate, "achieved_qps": n_req / wall,
                      "p50_ms": float(np.percentile(lat, 50) * 1e3),
                      "p99_ms": float(np.percentile(lat, 99) * 1e3),
                      "mean_ms": float(lat.mean() * 1e3), "results_same_as_saturation": same})
    clocks.mark_end()
    clk = clocks.stop()
    st = srv.stats()
    qsz = np.diff(q_off.astype(np.int64))
    line = {
        "metric": METRIC, "value": sat_qps, "unit": UNIT, "n_gpus": 1, "steps": len(sweep) + 1,
        "warmup": 1, "ms_per_step": sat_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "genie-serving",
        "config": {"workload": "serving: 8,000,000 objects x 64 Zipf(1.1) keywords over 2^22, "
                               "requests of 8-512 keywords, k uniform in {1, 10, 100}, Poisson "
                               "arrivals; admission by Bitmap-Counter bytes (8 bits per object "
                               "per query), budget = 512 queries",
                   "n_objects": w.n_objects, "n_requests": n_req,
                   "mean_request_keywords": float(qsz.mean()), "streams": 2, "max_batch": 256},
        "saturation": {"qps": sat_qps, "p50_ms": float(np.percentile(lat0, 50) * 1e3),
                       "p99_ms": float(np.percentile(lat0, 99) * 1e3)},
        "sweep": sweep,
        "server": {"launches": int(st.launches), "queries": int(st.queries),
                   "mean_batch": float(st.queries) / max(1, st.launches),
                   "deferred_admissions": int(st.deferred_admissions),
                   "max_queries_in_flight": int(st.max_queries_in_flight)},
        "clocks": clk,
    }
    srv.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "lsh4m-learned":
        if rank == 0:
            run_learned(args, rank, world, local)
    elif args.workload == "seq1m":
        if rank == 0:
            run_seq(args, rank, world, local)
    elif args.workload == "lsh4m-parts":
        if rank == 0:
            run_parts(args, rank, world, local)
    elif args.workload == "sets4m-batched":
        if rank == 0:
            run_batched(args, rank, world, local)
    elif args.workload == "serving":
        if rank == 0:
            run_serving(args, rank, world, local)
    else:
        run_genie(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
