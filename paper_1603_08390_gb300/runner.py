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


def build_index(w, chunk_shift: int = 0, stream=None) -> genie.Index:
    off, kw = to_dev(w.obj_off), to_dev(w.obj_kw)
    idx = genie.genie_build_index(off, kw, w.n_objects, w.vocab, chunk_shift, stream)
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


def query_facts(queries: genie.Queries) -> dict:
    n = queries.n_queries
    bound = torch.empty(n, dtype=torch.int32, device="cuda")
    entries = torch.empty(n, dtype=torch.int64, device="cuda")
    feats = torch.empty(n * genie.N_FEATURES, dtype=torch.float32, device="cuda")
    genie.genie_queries_export(queries, bound, entries, feats)
    return {"bound": u32(bound), "entries": entries.cpu().numpy().view(np.uint64),
            "features": feats.cpu().numpy().reshape(n, genie.N_FEATURES)}
