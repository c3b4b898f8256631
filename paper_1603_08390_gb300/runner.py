"""Host-side driver: moves host arrays to the device and calls the C ABI.

Argument marshalling only.  A workload is any object with the attributes of
``synth.Workload`` (``obj_off``, ``obj_kw``, ``n_objects``, ``vocab``, and
either ``q_off``/``q_kw`` or ``item_off``/``item_dim``/``item_lo``/
``item_hi``/``values_per_dim``).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import genie


def to_dev(a: np.ndarray, device: str = "cuda") -> torch.Tensor:
    """Copy a uint32 / int32 / uint64 / float32 array to the device (32-bit
    unsigned data travels as int32 bit patterns)."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(device)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def build_index(w, chunk_shift: int = 0, stream=None, dense_min_df=None) -> genie.Index:
    off, kw = to_dev(w.obj_off), to_dev(w.obj_kw)
    idx = genie.genie_build_index(off, kw, w.n_objects, w.vocab, chunk_shift, stream,
                                  dense_min_df=dense_min_df)
    return idx


def compile_queries(index: genie.Index, w, stream=None) -> genie.Queries:
    if w.kind == "keywords":
        return genie.genie_make_queries(index, to_dev(w.q_off), to_dev(w.q_kw), w.n_queries, stream)
    return genie.genie_compile_ranges(index, w.values_per_dim, to_dev(w.item_off),
                                      to_dev(w.item_dim), to_dev(w.item_lo), to_dev(w.item_hi),
                                      w.n_queries, stream)


class Outputs:
    """Device result buffers for n queries with row stride k."""

    def __init__(self, n_queries: int, k: int, device: str = "cuda"):
        self.k = k
        self.ids = torch.empty(n_queries * k, dtype=torch.int32, device=device)
        self.counts = torch.empty(n_queries * k, dtype=torch.int32, device=device)
        self.n_valid = torch.empty(n_queries, dtype=torch.int32, device=device)

    def host(self) -> dict:
        n = self.n_valid.numel()
        return {"ids": u32(self.ids).reshape(n, self.k),
                "counts": u32(self.counts).reshape(n, self.k),
                "n_valid": u32(self.n_valid)}


def search(index: genie.Index, queries: genie.Queries, k, opts: Optional[genie.SearchOpts] = None,
           out: Optional[Outputs] = None, stream=None) -> Outputs:
    """Run genie_search; ``k`` is an int or a per-query array (row stride = max)."""
    if np.isscalar(k):
        kmax, d_k = int(k), None
    else:
        karr = np.asarray(k, dtype=np.uint32)
        kmax, d_k = int(karr.max()), to_dev(karr)
    if out is None:
        out = Outputs(queries.n_queries, kmax)
    genie.genie_search(index, queries, kmax, out.ids, out.counts, out.n_valid, d_k=d_k, opts=opts,
                       stream=stream)
    return out


def build_parts(w, ranges, chunk_shift: int = 0, stream=None) -> genie.Parts:
    """A part store over the ascending, disjoint object-id ranges
    ``[(start, end), ...]`` of a keyword workload; each part is indexed with
    local ids and placed at global id ``start``."""
    parts = genie.Parts()
    off = w.obj_off.astype(np.int64)
    for a, b in ranges:
        sub_off = (off[a:b + 1] - off[a]).astype(np.uint32)
        sub_kw = w.obj_kw[off[a]:off[b]]
        idx = genie.genie_build_index(to_dev(sub_off), to_dev(sub_kw), b - a, w.vocab, chunk_shift,
                                      stream)
        parts.add(idx, a, stream)
        idx.close()
    return parts


def search_parts(parts: genie.Parts, w, k, out: Optional[Outputs] = None, stream=None) -> Outputs:
    """genie_parts_search over a keyword workload's queries."""
    if np.isscalar(k):
        kmax, d_k = int(k), None
    else:
        karr = np.asarray(k, dtype=np.uint32)
        kmax, d_k = int(karr.max()), to_dev(karr)
    if out is None:
        out = Outputs(w.n_queries, kmax)
    parts.search(to_dev(w.q_off), to_dev(w.q_kw), w.n_queries, kmax, out.ids, out.counts,
                 out.n_valid, d_k=d_k, stream=stream)
    return out


class SeqIndex:
    """Device copies of data sequences and the index of their ordered n-grams."""

    def __init__(self, s_off: np.ndarray, s_chars: np.ndarray, n: int, sigma: int, R: int,
                 chunk_shift: int = 0, stream=None):
        self.n, self.sigma, self.R = n, sigma, R
        self.vocab = sigma ** n * R
        self.n_seqs = len(s_off) - 1
        self.d_off, self.d_chars = to_dev(s_off), to_dev(s_chars)
        d_kw_off, d_kw, _ = sa_grams(self.d_off, self.d_chars, s_off, n, sigma, R, stream)
        self.index = genie.genie_build_index(d_kw_off, d_kw, self.n_seqs, self.vocab, chunk_shift,
                                             stream)


def sa_grams(d_off, d_chars, off: np.ndarray, n: int, sigma: int, R: int, stream=None):
    """Ordered n-gram keyword CSR (device) of sequences already on the device."""
    lens = np.diff(off.astype(np.int64))
    cap = max(int(np.maximum(lens - n + 1, 0).sum()), 1)
    d_kw_off = torch.empty(len(off), dtype=torch.int32, device="cuda")
    d_kw = torch.empty(cap, dtype=torch.int32, device="cuda")
    total = genie.genie_sa_grams(d_off, d_chars, len(off) - 1, n, sigma, R, d_kw_off, d_kw, cap,
                                 stream)
    return d_kw_off, d_kw, total


class SeqOutputs:
    """Device results of a sequence search: K candidates and the k verified."""

    def __init__(self, n_queries: int, K: int, k: int):
        self.K, self.k = K, k
        self.cand = Outputs(n_queries, K)
        z = lambda m: torch.empty(m, dtype=torch.int32, device="cuda")
        self.ids, self.ed = z(n_queries * k), z(n_queries * k)
        self.n_out, self.certified, self.examined = z(n_queries), z(n_queries), z(n_queries)

    def host(self) -> dict:
        n = self.n_out.numel()
        return {"ids": u32(self.ids).reshape(n, self.k), "ed": u32(self.ed).reshape(n, self.k),
                "n_out": u32(self.n_out), "certified": u32(self.certified).astype(bool),
                "examined": u32(self.examined), "candidates": self.cand.host()}


def sa_search(si: SeqIndex, q_off: np.ndarray, q_chars: np.ndarray, K: int, k: int,
              out: Optional[SeqOutputs] = None, stream=None, d_q=None) -> SeqOutputs:
    """Shotgun and assembly (Sec. 5.1): the queries' ordered n-grams, the top-K
    sequences by match count, then the verification of the candidates."""
    d_q_off, d_q_chars = d_q if d_q is not None else (to_dev(q_off), to_dev(q_chars))
    n_q = len(q_off) - 1
    if out is None:
        out = SeqOutputs(n_q, K, k)
    qk_off, qk, _ = sa_grams(d_q_off, d_q_chars, q_off, si.n, si.sigma, si.R, stream)
    qs = genie.genie_make_queries(si.index, qk_off, qk, n_q, stream)
    genie.genie_search(si.index, qs, K, out.cand.ids, out.cand.counts, out.cand.n_valid,
                       stream=stream)
    max_len = int(np.diff(q_off.astype(np.int64)).max()) if n_q else 0
    genie.genie_sa_verify(d_q_off, d_q_chars, n_q, si.d_off, si.d_chars, out.cand.ids,
                          out.cand.counts, out.cand.n_valid, K, k, si.n, max_len, out.ids, out.ed,
                          out.n_out, out.certified, out.examined, stream)
    return out


def query_facts(queries: genie.Queries) -> dict:
    n = queries.n_queries
    bound = torch.empty(n, dtype=torch.int32, device="cuda")
    entries = torch.empty(n, dtype=torch.int64, device="cuda")
    feats = torch.empty(n * genie.N_FEATURES, dtype=torch.float32, device="cuda")
    genie.genie_queries_export(queries, bound, entries, feats)
    return {"bound": u32(bound), "entries": entries.cpu().numpy().view(np.uint64),
            "features": feats.cpu().numpy().reshape(n, genie.N_FEATURES)}


def shard_range(n_objects: int, rank: int, world: int):
    """Object ids [lo, hi) of shard `rank` of `world` (contiguous, balanced)."""
    return n_objects * rank // world, n_objects * (rank + 1) // world


def gather_merge(ids: np.ndarray, counts: np.ndarray, k: int, dst: int = 0):
    """The exchange of an object-sharded search over the ranks of the default
    torch.distributed group: every rank gives its shard's results (uint32
    [Q, k_part], global ids), they are gathered on rank `dst` and merged
    exactly there by genie_merge_host.  Returns (ids, counts, n_valid) on
    `dst`, None elsewhere."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(), dist.get_rank()
    q, kp = ids.shape
    mine = torch.from_numpy(np.stack([ids, counts]).astype(np.uint32).view(np.int32).copy())
    parts = [torch.empty_like(mine) for _ in range(world)] if rank == dst else None
    dist.gather(mine, gather_list=parts, dst=dst)
    if rank != dst:
        return None
    arrs = [p.numpy().view(np.uint32) for p in parts]
    return genie.genie_merge_host([a[0] for a in arrs], [a[1] for a in arrs], k)
