#!/usr/bin/env python
"""Throughput of the match-count top-k hot path on one GB300 (or N replicas).

One step = one batch through the whole path: query compile (keyword look-up,
count bounds), the fused postings scan + c-PQ kernel and the per-query
top-k merge.  The headline batch is the largest single-GPU workload of the
suite: 4096 LSH queries against 4,000,000 objects x 256 keywords (k = 100).
``value`` is queries/s with the inputs already in HBM; ``e2e`` is the same
through the C ABI from pinned host buffers (``genie_search_host``: copy in,
compile, search, copy back, synchronise; one call per batch).

After the headline the default run measures every other workload once, each
as a sub-object of the same JSON line with its own timing, roofline and an
oracle check of sampled queries: the 1M-object LSH batch, the batched Zipf
sets (plain launch vs the persistent graph-captured batch), the learned
threshold (plain vs seeded on the headline batch), the serving loop
(saturation and p50/p99 under Poisson arrivals), multiple loadings, the tiny
relational batch and sequence search.  ``--workload NAME`` runs one of them
alone; ``--impl reference`` times the CPU oracle on a bounded sample of the
headline batch instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl genie|reference]
Under torchrun (N > 1) every rank holds an index replica and runs its own
4096 queries (weak scaling); only the timing uses a (gloo) collective, and
only the headline runs.
"""
from __future__ import annotations

import argparse
import gc
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
N_OBJECTS, N_QUERIES, K = 4_000_000, 4096, 100
WORKLOAD = ("lsh-4m: 4,000,000 objects x 256 p-stable LSH keywords (bucket width 4, "
            "bucket mod 8192), 4096 queries from the same 1000-component mixture, k=100")
REF_SAMPLE = 16   # oracle queries per reference step
CPU_SAMPLE = 96   # oracle queries for the cpu_baseline object
LEGS = ("lsh1m", "sets4m-batched", "lsh4m-learned", "serving", "lsh4m-parts", "relational",
        "seq1m", "gen-spq")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["genie", "reference"], default="genie")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=("all", "lsh4m") + LEGS, default="all",
                    help="all: the lsh-4m headline plus every other workload as a sub-object; "
                         "lsh4m: the headline alone; any other name: that workload alone")
    ap.add_argument("--queries", type=int, default=0,
                    help="queries per headline batch (0: the workload's 4096; smaller values "
                         "are for profiling captures)")
    return ap.parse_args(argv)


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


def headline_workload(rank: int, world: int, n_queries: int = N_QUERIES):
    """The lsh-4m objects and this rank's n_queries queries."""
    import synth
    w = synth.lsh(N_OBJECTS, n_queries * world, K, config=4)
    if world > 1:
        w = w.subset(np.arange(rank * n_queries, (rank + 1) * n_queries))
    return w


def postings_per_batch(w) -> int:
    """Postings a batch scans: the sum over query keywords of the keyword's
    list length (host numpy; the library reports the same from the device)."""
    df = np.bincount(w.obj_kw, minlength=w.vocab).astype(np.int64)
    return int(df[w.q_kw].sum())


def config_dict(w, world, workload=WORKLOAD, k=K):
    return {"workload": workload, "n_objects": int(w.n_objects), "n_queries": int(w.n_queries),
            "k": k, "postings": int(w.nnz),
            "l2": "inputs larger than L2 (List Array %.2f GB vs 126 MB L2), not flushed" % (
                w.nnz * 4 / 1e9),
            "parallelism": "replicas x%d (query batches, no data-path collective)" % world}


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


def traffic_from_profile(name: str = "scan_cpq_lsh4m_ncu.md"):
    """Per-launch DRAM bytes of the scan kernel from a committed ncu summary,
    valid only while the kernel sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        text = f.read()
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b:
        return None
    return float(m_b.group(1)) if kernel_source_sha() == m_sha.group(1) else None


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


def sampled_rows(n_queries: int, n: int = 8):
    return np.unique(np.linspace(0, n_queries - 1, n).astype(np.int64))


def parity_sampled(w, res: dict, rows) -> bool:
    """Result rows `rows` of `res` (host arrays ids/counts/n_valid, one row per
    query of w) against the oracle's brute force of the same queries: n_valid
    equal, and the ranked ids and counts equal up to it."""
    import oracle
    ref = oracle.topk(w.subset(rows))
    for j, q in enumerate(rows):
        n = int(ref["n_valid"][j])
        if int(res["n_valid"][q]) != n:
            return False
        if not (np.array_equal(res["ids"][q, :n], ref["ids"][j, :n]) and
                np.array_equal(res["counts"][q, :n], ref["counts"][j, :n])):
            return False
    return True


def scan_roofline(entries: int, scan_ms: float, kernel: str, traffic=None) -> dict:
    """The scan kernel against the measured copy peak, in the metric's
    algorithmic bytes (4 B per posting); DRAM traffic beside it when an ncu
    capture of the same kernel code gives it."""
    peak, peak_kind = measured_peaks()
    algo = 4.0 * entries
    achieved = algo / (scan_ms / 1e3) / 1e9
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
         "peak_kind": peak_kind + " hbm_gbs", "scan_ms": scan_ms,
         "algorithmic_bytes_per_launch": algo,
         "bytes": "logical: 4 B per posting scanned; range-major block order serves most of "
                  "them from L2, so DRAM moves far less (dram_gbs); the binding resource is "
                  "the shared-memory atomic pipe (smem_atomic_roofline)"}
    if traffic:
        r["dram_gbs"] = traffic / (scan_ms / 1e3) / 1e9
        r["dram_frac"] = r["dram_gbs"] / peak
    return r


def read_bytes(entries: int, dense: dict, dense_added: int, block_shift: int) -> int:
    """Bytes a scan reads when dense keywords are added as bitmaps: 4 B per
    posting of the other keywords, and a 2^block_shift-bit bitmap slice per
    (query, range, dense keyword) added."""
    sparse = entries * (1.0 - dense["batch_postings_share"]) if dense_added else entries
    return int(4 * sparse + dense_added * ((1 << block_shift) // 8))


def read_roofline(entries, dense, stats, shape, scan_ms, kernel) -> dict:
    """The scan against the measured copy peak in the bytes it must read
    (bitmap slices of the dense keywords, 4 B per other posting); the logical
    4 B per posting beside it."""
    peak, peak_kind = measured_peaks()
    b = read_bytes(entries, dense, stats["dense_bitmaps_added"], shape.block_shift)
    achieved = b / (scan_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "kernel": kernel,
            "peak_kind": peak_kind + " hbm_gbs", "scan_ms": scan_ms,
            "algorithmic_bytes_per_launch": b,
            "bytes": "read: the dense keywords' bitmap slices (2^block_shift bits per query, range "
                     "and keyword) and 4 B per posting of the other keywords",
            "logical_gbs": 4.0 * entries / (scan_ms / 1e3) / 1e9}


def atomic_roofline(entries: int, scan_ms: float, cal) -> dict:
    rate = entries / (scan_ms / 1e3)
    return {"bound": "shared-memory atomic adds (one per posting)", "achieved": rate,
            "peak": cal.smem_atomics_per_s, "unit": "updates/s",
            "frac": rate / cal.smem_atomics_per_s,
            "peak_kind": "measured by genie_calibrate on this GPU (atom with return)",
            "peak_red_no_return": cal.smem_red_per_s}


def search_step(genie, idx, d_q_off, d_q_kw, Q, k, out, stream, opts=None, d_k=None):
    qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    genie.genie_search(idx, qs, k, out.ids, out.counts, out.n_valid, d_k=d_k, opts=opts,
                       stream=stream)
    return qs


def cpq_stats(genie, idx, d_q_off, d_q_kw, Q, k, out, stream, entries, opts_kw=None):
    """c-PQ counters of one more (untimed) pass."""
    import torch
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    search_step(genie, idx, d_q_off, d_q_kw, Q, k, out, stream,
                opts=genie.make_opts(d_stats=stats, **(opts_kw or {})))
    st = stats.cpu().numpy()
    return {"gate_passes_per_posting": float(st[0]) / max(1, entries), "gate_passes": int(st[0]),
            "ht_inserts": int(st[1]), "blocks": int(st[4]), "blocks_bitmap_fallback": int(st[2]),
            "blocks_gateless_unseeded": int(st[6]), "reruns": int(st[3]), "bad_ids": int(st[5]),
            "dense_bitmaps_added": int(st[7])}


def dense_info(idx, qs) -> dict:
    """The index's dense keywords (object bitmaps) and the batch's share."""
    from paper_1603_08390_gb300 import genie
    qi = genie.QueriesInfo()
    genie.load().genie_queries_get_info(qs.handle, genie.ctypes.byref(qi))
    return {"keywords": int(idx.info.dense_keywords), "min_df": int(idx.info.dense_min_df),
            "bytes": int(idx.info.dense_bytes),
            "batch_postings_share": float(qi.n_dense_entries) / max(1, qi.n_entries)}


def run_headline(args, rank, world, local, keep=None):
    """lsh-4m, 4096 queries, k = 100: the headline line.  keep: a dict that
    receives the workload, index and device queries for the legs that reuse
    them (learned threshold, multiple loadings)."""
    import torch
    from paper_1603_08390_gb300 import genie, runner

    w = headline_workload(rank, world, args.queries or N_QUERIES)
    # index build on the device (Table 2's index-build time; one-time, not
    # part of a step): the object keyword sets are copied in first
    d_obj_off, d_obj_kw = runner.to_dev(w.obj_off), runner.to_dev(w.obj_kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = genie.genie_build_index(d_obj_off, d_obj_kw, w.n_objects, w.vocab, 0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del d_obj_off, d_obj_kw
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    out = runner.Outputs(Q, K)
    stream = torch.cuda.current_stream()

    def step(events=None):
        opts = genie.make_opts(scan_events=events) if events is not None else None
        return search_step(genie, idx, d_q_off, d_q_kw, Q, K, out, stream, opts=opts)

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        qs = step()
    torch.cuda.synchronize()
    entries = qs.n_entries
    kernel = genie.genie_search_shape(idx, qs, K).kernel_name()
    dense = dense_info(idx, qs)
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
    res = out.host()
    total_ms = step_ev[0].elapsed_time(step_ev[-1])
    per_step = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    scan_ms = statistics.mean(b.elapsed_time(e) for b, e in scan_ev)
    total_ms = max_over_ranks(total_ms, world)
    value = Q * world * args.steps / (total_ms / 1e3)

    # end to end through the C ABI: pinned host queries in, host results out,
    # one genie_search_host call per batch (it returns when the results are
    # in host memory)
    import torch as _t
    h_q_off = _t.from_numpy(w.q_off.view(np.int32)).pin_memory()
    h_q_kw = _t.from_numpy(w.q_kw.view(np.int32)).pin_memory()
    h_ids = _t.empty(Q * K, dtype=_t.int32).pin_memory()
    h_counts = _t.empty(Q * K, dtype=_t.int32).pin_memory()
    h_nv = _t.empty(Q, dtype=_t.int32).pin_memory()

    def e2e_step():
        genie.genie_search_host(idx, h_q_off, h_q_kw, Q, K, h_ids, h_counts, h_nv, stream=stream)

    for _ in range(max(3, args.warmup)):
        e2e_step()
    barrier(world)
    e2e_lat = []
    t_e0 = time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        e2e_step()
        e2e_lat.append((time.perf_counter() - t1) * 1e3)
    e2e_ms = max_over_ranks((time.perf_counter() - t_e0) * 1e3, world)
    barrier(world)
    h2d = (Q + 1) * 4 + int(w.q_off[-1]) * 4
    d2h = 2 * Q * K * 4 + Q * 4
    e2e_same = bool(np.array_equal(h_ids.numpy().view(np.uint32).reshape(Q, K), res["ids"]) and
                    np.array_equal(h_nv.numpy().view(np.uint32), res["n_valid"]))

    cal = genie.genie_calibrate()
    cpq = cpq_stats(genie, idx, d_q_off, d_q_kw, Q, K, out, stream, entries)
    rows = sampled_rows(Q)
    parity = parity_sampled(w, res, rows) if rank == 0 else None
    if keep is not None:
        keep.update(w=w, idx=idx, d_q_off=d_q_off, d_q_kw=d_q_kw, plain_ms=total_ms / args.steps,
                    plain_res=res)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_dict(w, world),
        "entries_per_step": int(entries),
        "entries_per_s": entries * world * args.steps / (total_ms / 1e3),
        "latency_ms": {"batch_p50": float(np.percentile(per_step, 50)),
                       "batch_p99": float(np.percentile(per_step, 99)),
                       "e2e_batch_p50": float(np.percentile(e2e_lat, 50)),
                       "e2e_batch_p99": float(np.percentile(e2e_lat, 99))},
        "roofline": scan_roofline(entries, scan_ms, kernel, traffic_from_profile()),
        "smem_atomic_roofline": atomic_roofline(entries, scan_ms, cal),
        "e2e": {"value": Q * world * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "genie_search_host (synchronous: each batch's copies, compile, search "
                       "and copy-back complete before the next call)",
                "results_equal_device_path": e2e_same},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "cpq": cpq,
        "dense_keywords": dense,
        "parity_sampled": {"queries": [int(r) for r in rows], "ok": bool(parity)},
        "index_build_s": build_s,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, CPU_SAMPLE)
    return line


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


def run_reference(args, rank, world):
    """The oracle on a bounded sample of the headline batch, on the host cores."""
    if rank != 0:
        return
    import oracle
    w = headline_workload(0, 1)
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
            "config": config_dict(w, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": "%d queries per step (first %d of %d), brute force over "
                                       "%d objects" % (REF_SAMPLE, REF_SAMPLE, w.n_queries,
                                                       w.n_objects)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def leg_steps(args) -> int:
    return max(3, min(args.steps, 10))


def leg_lsh1m(args):
    """C2: 1,000,000 LSH objects, 1024 queries, k = 100 (plain path), with the
    gateless ablation (count, then select from the counters) beside it."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, runner

    k = 100
    w = synth.config(2)
    if args.queries:  # a smaller batch of the same queries (profiling captures)
        w = w.subset(np.arange(min(args.queries, w.n_queries)))
    idx = runner.build_index(w)
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    out = runner.Outputs(Q, k)
    stream = torch.cuda.current_stream()
    steps = leg_steps(args)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for b, e in ev:
        b.record(stream)
        e.record(stream)
    it = iter(range(10 ** 9))

    def step():
        i = next(it)
        opts = genie.make_opts(scan_events=ev[i - W0]) if i >= W0 else None
        return search_step(genie, idx, d_q_off, d_q_kw, Q, k, out, stream, opts=opts)

    W0 = 3
    for _ in range(W0):
        qs = step()
    entries = qs.n_entries
    kernel = genie.genie_search_shape(idx, qs, k).kernel_name()
    del qs
    ms, per = timed_steps(step, steps, stream)
    scan_ms = statistics.mean(b.elapsed_time(e) for b, e in ev)
    res = out.host()
    ng = genie.make_opts(flags=genie.GENIE_SEARCH_NO_GATE)
    step_ng = lambda: search_step(genie, idx, d_q_off, d_q_kw, Q, k, out, stream, opts=ng)
    step_ng()
    ng_ms, _ = timed_steps(step_ng, steps, stream)
    res_ng = out.host()
    cal = genie.genie_calibrate()
    return {"config": config_dict(w, 1, "lsh-1m: 1,000,000 objects x 256 p-stable LSH keywords, "
                                        "1024 queries, k=100", k),
            "value": Q * steps / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
            "entries_per_step": int(entries), "entries_per_s": entries * steps / (ms / 1e3),
            "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                           "batch_p99": float(np.percentile(per, 99))},
            "roofline": scan_roofline(entries, scan_ms, kernel,
                                      traffic_from_profile("scan_cpq_lsh1m_ncu.md")),
            "smem_atomic_roofline": atomic_roofline(entries, scan_ms, cal),
            "cpq": cpq_stats(genie, idx, d_q_off, d_q_kw, Q, k, out, stream, entries),
            "ablation_no_gate": {"ms_per_step": ng_ms / steps, "value": Q * steps / (ng_ms / 1e3),
                                 "c_pq_speedup": ng_ms / ms,
                                 "identical_results": all(np.array_equal(res[x], res_ng[x])
                                                          for x in res)},
            "parity_sampled": {"ok": parity_sampled(w, res, sampled_rows(Q))},
            "gpu_launches": 3 * steps}


def leg_learned(args, keep):
    """C4 learned threshold on the headline batch: a 64-128-1 network trained
    on the GPU predicts each query's k-th count and seeds the AuditThreshold;
    plain vs seeded, plus the ceiling of any predictor (seeds = the exact
    k-th counts the plain search returned)."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, learned, runner

    k = K
    w, idx = keep["w"], keep["idx"]
    d_q_off, d_q_kw = keep["d_q_off"], keep["d_q_kw"]
    Q = w.n_queries
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tq_off, tq_kw = synth.lsh_training_queries(100_000, config=4)
    tr = learned.train_predictor(idx, tq_off, tq_kw, k, epochs=20, batch=256, lr=2e-3)
    train_s = time.perf_counter() - t0
    out_p, out_l, out_c = runner.Outputs(Q, k), runner.Outputs(Q, k), runner.Outputs(Q, k)
    seeds = torch.empty(Q, dtype=torch.int32, device="cuda")

    def plain():
        search_step(genie, idx, d_q_off, d_q_kw, Q, k, out_p, stream)

    def seeded(stats=None):
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        tr["mlp"].seeds(qs, tr["margin"], seeds, stream)
        genie.genie_search(idx, qs, k, out_l.ids, out_l.counts, out_l.n_valid,
                           opts=genie.make_opts(d_seed=seeds, d_stats=stats), stream=stream)

    plain()
    torch.cuda.synchronize()
    # the best any predictor can do: seed each query with its exact k-th count
    exact = out_p.counts.view(Q, k)[:, k - 1].clone().clamp_(min=1)

    def ceiling(stats=None):
        search_step(genie, idx, d_q_off, d_q_kw, Q, k, out_c, stream,
                    opts=genie.make_opts(d_seed=exact, d_stats=stats))

    steps = leg_steps(args)
    for _ in range(2):
        plain()
        seeded()
        ceiling()
    p_ms, _ = timed_steps(plain, steps, stream)
    l_ms, per = timed_steps(seeded, steps, stream)
    c_ms, _ = timed_steps(ceiling, steps, stream)
    st = {}
    for name, fn in (("plain", None), ("learned", seeded), ("ceiling", ceiling)):
        s = torch.zeros(8, dtype=torch.int64, device="cuda")
        if fn is None:
            search_step(genie, idx, d_q_off, d_q_kw, Q, k, out_p, stream,
                        opts=genie.make_opts(d_stats=s))
        else:
            fn(s)
        st[name] = s.cpu().numpy()
    a, b, c = out_p.host(), out_l.host(), out_c.host()
    same = all(np.array_equal(a[x], b[x]) and np.array_equal(a[x], c[x]) for x in a)
    return {"config": {"workload": "lsh-4m learned threshold: the headline batch; 64-128-1 bf16 "
                                   "MLP trained on the GPU on 100k query / k-th-count pairs "
                                   "from the plain search", "n_queries": Q, "k": k},
            "plain": {"value": Q * steps / (p_ms / 1e3), "ms_per_step": p_ms / steps,
                      "gate_passes": int(st["plain"][0]), "ht_inserts": int(st["plain"][1])},
            "learned": {"value": Q * steps / (l_ms / 1e3), "ms_per_step": l_ms / steps,
                        "gate_passes": int(st["learned"][0]), "ht_inserts": int(st["learned"][1]),
                        "reruns": int(st["learned"][3]), "rerun_rate": float(st["learned"][3]) / Q,
                        "batch_p50_ms": float(np.percentile(per, 50)),
                        "batch_p99_ms": float(np.percentile(per, 99))},
            "ceiling_exact_seeds": {"value": Q * steps / (c_ms / 1e3), "ms_per_step": c_ms / steps,
                                    "gate_passes": int(st["ceiling"][0])},
            "speedup_vs_plain": p_ms / l_ms, "ceiling_speedup_vs_plain": p_ms / c_ms,
            "identical_results": bool(same),
            "training": {"seconds": train_s, "train_loss": tr["train_loss"],
                         "margin": tr["margin"], "n_train": tr["n_train"], "n_val": tr["n_val"],
                         "target_mean": tr["target_mean"]},
            "parity_sampled": {"ok": parity_sampled(w, b, sampled_rows(Q))},
            "gpu_launches": 5 * steps}


def leg_batched(args):
    """C3: 4M Zipf(1.1) sets, 8192 queries of 8-512 keywords, k = 10: plain
    launches vs the persistent, graph-captured, autotuned batch."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, runner

    k = 10
    w = synth.config(3)
    if args.queries:  # a smaller batch of the same queries (profiling captures)
        w = w.subset(np.arange(0, w.n_queries, max(1, w.n_queries // args.queries))[:args.queries])
    idx = runner.build_index(w)
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    stream = torch.cuda.current_stream()
    sample = w.subset(np.arange(0, Q, max(1, Q // 512))[:512])
    sq = runner.compile_queries(idx, sample)
    t0 = time.perf_counter()
    tuned = genie.genie_autotune(idx, sq, k, os.path.join(tempfile.gettempdir(), "genie_tune.txt"))
    tune_s = time.perf_counter() - t0
    qs0 = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    batch = genie.Batch(idx, Q, qs0.max_bound, k, tuned)
    entries = qs0.n_entries
    shape = genie.genie_search_shape(idx, qs0, k)
    kernel = shape.kernel_name()
    dense = dense_info(idx, qs0)
    dstats = cpq_stats(genie, idx, d_q_off, d_q_kw, Q, k, runner.Outputs(Q, k), stream, entries)
    del qs0
    out_p, out_b = runner.Outputs(Q, k), runner.Outputs(Q, k)
    steps = max(3, min(args.steps, 4))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for b, e in ev:
        b.record(stream)
        e.record(stream)
    idx_ev = [0]

    def plain(timed=False):
        opts = None
        if timed:
            opts = genie.make_opts(scan_events=ev[idx_ev[0]])
            idx_ev[0] += 1
        search_step(genie, idx, d_q_off, d_q_kw, Q, k, out_p, stream, opts=opts)

    def batched():
        qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
        batch.run(qs, out_b.ids, out_b.counts, out_b.n_valid, stream=stream)

    plain()
    batched()
    p_ms, _ = timed_steps(lambda: plain(True), steps, stream)
    b_ms, per = timed_steps(batched, steps, stream)
    scan_ms = statistics.mean(b.elapsed_time(e) for b, e in ev)
    a, b = out_p.host(), out_b.host()
    identical = all(np.array_equal(a[x], b[x]) for x in a)
    return {"config": config_dict(w, 1, "sets-4m batched: 4,000,000 Zipf(1.1) keyword sets of "
                                        "16-256 over a 2^20 vocabulary, 8192 queries of 8-512 "
                                        "keywords, k=10", k),
            "value": Q * steps / (b_ms / 1e3), "ms_per_step": b_ms / steps, "steps": steps,
            "entries_per_step": int(entries), "entries_per_s": entries * steps / (b_ms / 1e3),
            "plain": {"value": Q * steps / (p_ms / 1e3), "ms_per_step": p_ms / steps,
                      "kernel": kernel, "scan_ms": scan_ms,
                      "roofline": read_roofline(entries, dense, dstats, shape, scan_ms, kernel),
                      "dense_keywords": dense, "cpq": dstats},
            "batched": {"value": Q * steps / (b_ms / 1e3), "ms_per_step": b_ms / steps,
                        "batch_p50_ms": float(np.percentile(per, 50)),
                        "batch_p99_ms": float(np.percentile(per, 99))},
            "autotune": {"block_shift": tuned.block_shift, "threads": tuned.threads,
                         "unroll": tuned.unroll, "ht_slots": tuned.ht_slots,
                         "sample_ms": tuned.tuned_ms, "seconds": tune_s,
                         "from_cache": bool(tuned.from_cache)},
            "batched_speedup_vs_plain": p_ms / b_ms, "identical_results": bool(identical),
            "parity_sampled": {"ok": parity_sampled(w, b, sampled_rows(Q))},
            "gpu_launches": 5 * steps}


def leg_serving(args):
    """C5: continuous-batching server on 8M x 64 Zipf sets; saturation and
    p50/p99 latency under Poisson arrivals at fractions of it."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, runner

    w = synth.sets(8_000_000, (64, 64), 1 << 22, 16, (8, 512), 10, config=5)  # the objects
    idx = runner.build_index(w)
    n_req = 4000
    q_off, q_kw, ks, _ = synth.serving_requests(n_req, 1.0, config=5)
    opts = genie.ServerOpts(max_batch=256, max_query_keywords=512, k_max=100, streams=2)
    srv = genie.Server(idx, opts)
    srv.replay(q_off[:201] - q_off[0], q_kw[:q_off[200]], ks[:200], np.zeros(200))
    t0 = time.perf_counter()
    lat0, ids0, cnt0, nv0 = srv.replay(q_off, q_kw, ks, np.zeros(n_req))
    sat_s = time.perf_counter() - t0
    sat_qps = n_req / sat_s
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
    st = srv.stats()
    srv.close()
    # oracle check of sampled requests against the same objects
    rows = sampled_rows(n_req)
    wq = synth.Workload(name="serving-requests", kind="keywords", n_objects=w.n_objects,
                        vocab=w.vocab, obj_off=w.obj_off,
                        obj_kw=w.obj_kw, n_queries=n_req, q_off=q_off, q_kw=q_kw,
                        k=np.asarray(ks, dtype=np.uint32))
    res = {"ids": ids0, "counts": cnt0, "n_valid": nv0}
    qsz = np.diff(q_off.astype(np.int64))
    # the plain search on the same requests (one batch, k = 100) for comparison
    d_q_off, d_q_kw = runner.to_dev(q_off), runner.to_dev(q_kw)
    out = runner.Outputs(n_req, 100)
    stream = torch.cuda.current_stream()
    d_k = runner.to_dev(np.asarray(ks, dtype=np.uint32))
    fn = lambda: search_step(genie, idx, d_q_off, d_q_kw, n_req, 100, out, stream, d_k=d_k)
    fn()
    pl_ms, _ = timed_steps(fn, 3, stream)
    return {"config": {"workload": "serving: 8,000,000 objects x 64 Zipf(1.1) keywords over 2^22, "
                                   "requests of 8-512 keywords, k uniform in {1, 10, 100}, Poisson "
                                   "arrivals; admission by the device memory a request holds",
                       "n_objects": w.n_objects, "n_requests": n_req,
                       "mean_request_keywords": float(qsz.mean()), "streams": 2, "max_batch": 256},
            "value": sat_qps,
            "saturation": {"qps": sat_qps, "p50_ms": float(np.percentile(lat0, 50) * 1e3),
                           "p99_ms": float(np.percentile(lat0, 99) * 1e3)},
            "sweep": sweep,
            "plain_one_batch": {"value": n_req * 3 / (pl_ms / 1e3), "ms_per_batch": pl_ms / 3},
            "server": {"launches": int(st.launches), "queries": int(st.queries),
                       "mean_batch": float(st.queries) / max(1, st.launches),
                       "deferred_admissions": int(st.deferred_admissions),
                       "max_queries_in_flight": int(st.max_queries_in_flight)},
            "parity_sampled": {"ok": parity_sampled(wq, res, rows)}}


def leg_parts(args, keep):
    """Multiple loadings (Sec. 3.4): the headline objects as four index parts
    of 1M in pinned host memory (each id kept as its 16-bit place in its object
    range), copied to the device part by part during each batch of 1024
    queries, against the device-resident index."""
    import torch
    from paper_1603_08390_gb300 import genie, runner

    k, P = K, 4
    w = keep["w"].subset(np.arange(1024))
    idx = keep["idx"]
    N, Q = w.n_objects, w.n_queries
    parts = runner.build_parts(w, [(p * N // P, (p + 1) * N // P) for p in range(P)])
    info = parts.info
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    stream = torch.cuda.current_stream()
    out_p, out_d = runner.Outputs(Q, k), runner.Outputs(Q, k)

    def step_parts():
        parts.search(d_q_off, d_q_kw, Q, k, out_p.ids, out_p.counts, out_p.n_valid, stream=stream)

    def step_device():
        search_step(genie, idx, d_q_off, d_q_kw, Q, k, out_d, stream)

    for _ in range(2):
        step_parts()
        step_device()
    steps = leg_steps(args)
    p_ms, per = timed_steps(step_parts, steps, stream)
    d_ms, _ = timed_steps(step_device, steps, stream)
    a, b = out_p.host(), out_d.host()
    identical = all(np.array_equal(a[x], b[x]) for x in a)
    res = {"config": {"workload": "lsh-4m multiple loadings: the 4,000,000 LSH objects as 4 index "
                                  "parts of 1,000,000 in pinned host memory; 1024 queries, k=100",
                      "n_objects": N, "n_queries": Q, "k": k, "parts": P},
           "value": Q * steps / (p_ms / 1e3), "ms_per_step": p_ms / steps,
           # with more than two parts every call copies each part once
           "h2d_bytes_per_step": int(info.host_bytes),
           "h2d_gb_per_s": info.host_bytes * steps / (p_ms / 1e3) / 1e9,
           "device_resident": {"value": Q * steps / (d_ms / 1e3), "ms_per_step": d_ms / steps,
                               "device_index_bytes": int(idx.device_bytes)},
           "parts_vs_device_resident": d_ms / p_ms, "identical_results": bool(identical),
           "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                          "batch_p99": float(np.percentile(per, 99))},
           # per part: 4 search launches + 2 that rebuild the ids from 16-bit places
           "gpu_launches": (6 * P + 2) * steps}
    del parts
    return res


def leg_relational(args):
    """C1: 10,000 x 16 relational tuples, 64 range queries of 16 items, k = 10."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, runner

    w = synth.config(1)
    idx = runner.build_index(w)
    stream = torch.cuda.current_stream()
    args_ = (runner.to_dev(w.item_off), runner.to_dev(w.item_dim), runner.to_dev(w.item_lo),
             runner.to_dev(w.item_hi))
    k = int(w.k)
    out = runner.Outputs(w.n_queries, k)

    def step():
        qs = genie.genie_compile_ranges(idx, w.values_per_dim, *args_, w.n_queries, stream)
        genie.genie_search(idx, qs, k, out.ids, out.counts, out.n_valid, stream=stream)

    for _ in range(3):
        step()
    steps = leg_steps(args)
    ms, per = timed_steps(step, steps, stream)
    res = out.host()
    import oracle
    ref = oracle.topk(w)
    ok = all(np.array_equal(res[x], ref[x]) for x in ("ids", "counts", "n_valid"))
    return {"config": {"workload": "relational: 10,000 objects x 16 attributes in [0, 64), 64 "
                                   "queries of 16 range items [v-2, v+2], k=10",
                       "n_objects": w.n_objects, "n_queries": w.n_queries, "k": k},
            "value": w.n_queries * steps / (ms / 1e3), "ms_per_step": ms / steps,
            "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                           "batch_p99": float(np.percentile(per, 99))},
            "parity_all_queries": {"ok": bool(ok)}, "gpu_launches": 3 * steps}


def leg_seq(args):
    """Sequence search by ordered n-grams (Sec. 5.1): 1M sequences of 40-100
    characters, 1024 queries with 1-6 edits, K = 128 candidates, k = 1."""
    import torch
    import synth
    from paper_1603_08390_gb300 import runner

    n, R, Kc, k = 3, 32, 128, 1
    seqs = synth.sequences(1_000_000, (40, 100), 26, 1024, (1, 6), config=6)
    si = runner.SeqIndex(seqs.s_off, seqs.s_chars, n, seqs.sigma, R)
    Q = seqs.n_queries
    d_q = (runner.to_dev(seqs.q_off), runner.to_dev(seqs.q_chars))
    out = runner.SeqOutputs(Q, Kc, k)
    stream = torch.cuda.current_stream()

    def step():
        runner.sa_search(si, seqs.q_off, seqs.q_chars, Kc, k, out=out, stream=stream, d_q=d_q)

    for _ in range(3):
        step()
    steps = leg_steps(args)
    ms, per = timed_steps(step, steps, stream)
    res = out.host()
    from oracle import sa
    n_s = 4
    sub = seqs.subset(np.arange(n_s))
    truth = sa.topk_ed(seqs.s_off, seqs.s_chars, sub.q_off, sub.q_chars, k)
    cert = res["certified"][:n_s]
    return {"config": {"workload": "seq-1m: 1,000,000 sequences of 40-100 characters over 26 "
                                   "letters, ordered 3-grams; 1024 queries with 1-6 random edits; "
                                   "top-128 candidates verified by edit distance (k=1)",
                       "n_sequences": seqs.n_seqs, "n_queries": Q, "n": n, "K": Kc, "k": k},
            "value": Q * steps / (ms / 1e3), "ms_per_step": ms / steps,
            "certified_fraction": float(res["certified"].mean()),
            "examined_mean": float(res["examined"].mean()),
            "latency_ms": {"batch_p50": float(np.percentile(per, 50)),
                           "batch_p99": float(np.percentile(per, 99))},
            "parity_sampled": {"ok": bool(np.all(res["ed"][:n_s][cert, 0] ==
                                                  truth["ed"][cert, 0])),
                               "queries": n_s, "certified": int(cert.sum())},
            "gpu_launches": 7 * steps}


def leg_spq(args):
    """The GEN-SPQ ablation (Sec. 6.1.2, Appendix A) on the 1M-object LSH
    batch: a dense Count Table per query filled with global atomics, then the
    bucket k-selection, against c-PQ -- time and device memory per query
    (Table 5's comparison)."""
    import torch
    import synth
    from paper_1603_08390_gb300 import genie, runner

    k = 100
    w = synth.config(2)
    idx = runner.build_index(w)
    Q = w.n_queries
    d_q_off, d_q_kw = runner.to_dev(w.q_off), runner.to_dev(w.q_kw)
    out_s, out_c = runner.Outputs(Q, k), runner.Outputs(Q, k)
    stream = torch.cuda.current_stream()
    qs = genie.genie_make_queries(idx, d_q_off, d_q_kw, Q, stream)
    info = genie.genie_search_spq(idx, qs, k, out_s.ids, out_s.counts, out_s.n_valid)
    shape = genie.genie_search_shape(idx, qs, k)
    spq = lambda: genie.genie_search_spq(idx, qs, k, out_s.ids, out_s.counts, out_s.n_valid,
                                         stream=stream, want_info=False)
    cpq = lambda: genie.genie_search(idx, qs, k, out_c.ids, out_c.counts, out_c.n_valid,
                                     stream=stream)
    spq()
    cpq()
    steps = 3
    s_ms, _ = timed_steps(spq, steps, stream)
    c_ms, _ = timed_steps(cpq, steps, stream)
    a, b = out_s.host(), out_c.host()
    same = all(np.array_equal(a[x], b[x]) for x in a)
    # c-PQ's device memory per query: its per-range candidate lists, the
    # shared k-th count and count histogram, and its result rows (the
    # counters themselves live in shared memory of the blocks)
    cpq_bytes = shape.n_groups * k * 8 + 4 + (qs.max_bound + 2) * 4 + 2 * k * 4 + 4
    spq_bytes = info.count_table_bytes_per_query + info.list_bytes_per_query + 2 * k * 4 + 4
    return {"config": {"workload": "GEN-SPQ vs c-PQ on lsh-1m: 1,000,000 objects x 256 LSH "
                                   "keywords, 1024 queries, k=100", "n_queries": Q, "k": k},
            "value": Q * steps / (s_ms / 1e3), "ms_per_step": s_ms / steps,
            "gen_spq": {"ms_per_step": s_ms / steps, "value": Q * steps / (s_ms / 1e3),
                        "bytes_per_query": spq_bytes, "queries_per_pass": info.queries_per_pass,
                        "passes": info.passes, "bucket_iterations_mean": info.mean_iterations},
            "c_pq": {"ms_per_step": c_ms / steps, "value": Q * steps / (c_ms / 1e3),
                     "bytes_per_query": cpq_bytes},
            "c_pq_speedup": s_ms / c_ms, "memory_ratio": spq_bytes / cpq_bytes,
            "identical_results": bool(same),
            "parity_sampled": {"ok": parity_sampled(w, a, sampled_rows(Q))}}


LEG_FUNCS = {"lsh1m": leg_lsh1m, "gen-spq": leg_spq, "sets4m-batched": leg_batched, "serving": leg_serving,
             "relational": leg_relational, "seq1m": leg_seq}


def run_leg(name, args, keep):
    import torch
    t0 = time.perf_counter()
    try:
        if name == "lsh4m-learned":
            r = leg_learned(args, keep)
        elif name == "lsh4m-parts":
            r = leg_parts(args, keep)
        else:
            r = LEG_FUNCS[name](args)
    except Exception as e:  # a failed leg is reported, and the others still run
        r = {"error": "%s: %s" % (type(e).__name__, e)}
    r["wall_s"] = time.perf_counter() - t0
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return r


def run_genie(args, rank, world, local):
    import torch
    from paper_1603_08390_gb300 import _build

    _build.build()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    if args.workload in ("all", "lsh4m"):
        keep = {}
        line = run_headline(args, rank, world, local, keep)
        if rank == 0 and args.workload == "all" and world == 1:
            legs = {}
            for name in ("lsh4m-learned", "lsh4m-parts"):  # they reuse the headline index
                legs[name] = run_leg(name, args, keep)
            keep.clear()
            gc.collect()
            torch.cuda.empty_cache()
            for name in ("lsh1m", "gen-spq", "sets4m-batched", "serving", "relational", "seq1m"):
                legs[name] = run_leg(name, args, keep)
            line["legs"] = legs
            line["suite_wall_s"] = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if rank != 0:
        return
    keep = {}
    if args.workload in ("lsh4m-learned", "lsh4m-parts"):
        import synth  # noqa: F401
        from paper_1603_08390_gb300 import runner
        w = headline_workload(0, 1, args.queries or N_QUERIES)
        keep.update(w=w, idx=runner.build_index(w), d_q_off=runner.to_dev(w.q_off),
                    d_q_kw=runner.to_dev(w.q_kw))
    r = run_leg(args.workload, args, keep)
    line = {"metric": METRIC, "value": r.get("value"), "unit": UNIT, "n_gpus": 1,
            "steps": r.get("steps", leg_steps(args)), "warmup": 3,
            "ms_per_step": r.get("ms_per_step"), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "genie-" + args.workload,
            "config": r.get("config", {"workload": args.workload}), "leg": r}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_genie(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
