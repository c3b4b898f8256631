"""Seeded synthetic workloads for match-count top-k search.

Input generation only: relational tuples and range queries (Example 2.1,
Sec. 5.3), Gaussian-mixture vectors mapped to p-stable LSH keywords (Sec. 4.1,
Eqn. (plsh), with the bucket re-hash of Sec. 4.1.2 taken as ``bucket mod
8192``), and Zipf(1.1) keyword sets (stand-ins for the word / n-gram sets of
Sec. 5.1-5.2).  None of the match-count arithmetic lives here; the CUDA path
and the CPU oracle both consume these arrays.

Seeds: ``160308390 + config`` with separate streams for the model (mixture
means, hash functions, keyword permutation), the objects, the queries and the
training queries.  The paper's datasets (OCR, SIFT, DBLP, Tweets, Adult) are
not available; these shapes stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 160308390
ROLE_OBJECTS, ROLE_QUERIES, ROLE_TRAIN = 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C sampler (gcc, OpenMP) into synth/_build/libsynth.so."""
    out_dir = os.path.join(_HERE, "_build")
    so = os.path.join(out_dir, "libsynth.so")
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    os.makedirs(out_dir, exist_ok=True)
    tmp = so + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            u64, u32, dbl, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
            lib.synth_lsh.argtypes = [u64, u64, u64, u32, u32, dbl, dbl, u32, dbl, u32, p, p, p]
            lib.synth_lsh.restype = ctypes.c_int
            lib.synth_set_lengths.argtypes = [u64, u64, u32, u32, p]
            lib.synth_set_lengths.restype = None
            lib.synth_permutation.argtypes = [u64, u32, p]
            lib.synth_permutation.restype = None
            lib.synth_zipf_sets.argtypes = [u64, u64, u32, dbl, p, p, p]
            lib.synth_chars.argtypes = [u64, u64, u32, dbl, p, p]
            lib.synth_chars.restype = None
            lib.synth_zipf_sets.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _seed(config: int, role: int) -> int:
    return (SEED_BASE + config) * 1000003 + role


@dataclass
class Workload:
    """One synthetic workload.

    Objects are keyword sets in CSR form (``obj_off[N+1]``, ``obj_kw[nnz]``,
    uint32, keyword ids < ``vocab``).  Queries are either keyword multisets
    (``q_off[Q+1]``, ``q_kw``) or relational range items (``item_off[Q+1]``,
    ``item_dim``, ``item_lo``, ``item_hi``) over ``values[N, D]``, where object
    ``o`` holds keyword ``d * values_per_dim + values[o, d]`` for each ``d``.
    ``k`` is an int or a per-query uint32 array.
    """
    name: str
    kind: str
    n_objects: int
    vocab: int
    obj_off: np.ndarray
    obj_kw: np.ndarray
    n_queries: int
    k: object
    q_off: Optional[np.ndarray] = None
    q_kw: Optional[np.ndarray] = None
    values: Optional[np.ndarray] = None
    values_per_dim: int = 0
    item_off: Optional[np.ndarray] = None
    item_dim: Optional[np.ndarray] = None
    item_lo: Optional[np.ndarray] = None
    item_hi: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.obj_off[-1])

    def query_items(self) -> int:
        return int((self.q_off if self.kind == "keywords" else self.item_off)[-1])

    def subset(self, qids) -> "Workload":
        """Same objects, only the queries ``qids`` (in that order)."""
        qids = np.asarray(qids, dtype=np.int64)
        k = self.k if np.isscalar(self.k) else np.asarray(self.k)[qids]
        if self.kind == "keywords":
            off, kw = _gather_rows(self.q_off, self.q_kw, qids)
            return Workload(self.name + "[sub]", self.kind, self.n_objects, self.vocab,
                            self.obj_off, self.obj_kw, len(qids), k, q_off=off, q_kw=kw,
                            extra=dict(self.extra))
        off, dim = _gather_rows(self.item_off, self.item_dim, qids)
        _, lo = _gather_rows(self.item_off, self.item_lo, qids)
        _, hi = _gather_rows(self.item_off, self.item_hi, qids)
        return Workload(self.name + "[sub]", self.kind, self.n_objects, self.vocab,
                        self.obj_off, self.obj_kw, len(qids), k, values=self.values,
                        values_per_dim=self.values_per_dim, item_off=off, item_dim=dim,
                        item_lo=lo, item_hi=hi, extra=dict(self.extra))


def _gather_rows(off: np.ndarray, vals: np.ndarray, rows: np.ndarray):
    off = off.astype(np.int64)
    lens = off[rows + 1] - off[rows]
    new_off = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=new_off[1:])
    idx = np.repeat(off[rows] - new_off[:-1], lens) + np.arange(new_off[-1])
    return new_off.astype(np.uint32), vals[idx]


# ----------------------------------------------------------------------------
# Relational tuples with range queries (Example 2.1; Sec. 5.3)
# ----------------------------------------------------------------------------

def relational(n_objects: int = 10_000, n_dims: int = 16, values_per_dim: int = 64,
               n_queries: int = 64, half_width: int = 2, k: int = 10, config: int = 1,
               items_per_query: Optional[int] = None) -> Workload:
    """Tuples with values U[0, values_per_dim); each query takes a random
    anchor object and puts the item ``(d, [v_d - hw, v_d + hw])`` on dimension
    ``d`` for ``d < items_per_query`` (ranges are NOT clipped: the query
    compiler clips them to the value domain)."""
    rng_o = np.random.default_rng([SEED_BASE + config, ROLE_OBJECTS])
    rng_q = np.random.default_rng([SEED_BASE + config, ROLE_QUERIES])
    values = rng_o.integers(0, values_per_dim, size=(n_objects, n_dims)).astype(np.uint32)
    obj_off = (np.arange(n_objects + 1, dtype=np.uint64) * n_dims).astype(np.uint32)
    obj_kw = (np.arange(n_dims, dtype=np.uint32)[None, :] * values_per_dim + values).ravel()
    m = n_dims if items_per_query is None else items_per_query
    anchors = rng_q.integers(0, n_objects, size=n_queries)
    item_off = (np.arange(n_queries + 1, dtype=np.int64) * m).astype(np.uint32)
    item_dim = np.tile(np.arange(m, dtype=np.uint32), n_queries)
    centre = values[anchors][:, :m].astype(np.int32).ravel()
    item_lo = (centre - half_width).astype(np.int32)
    item_hi = (centre + half_width).astype(np.int32)
    return Workload("relational", "relational", n_objects, n_dims * values_per_dim, obj_off,
                    obj_kw, n_queries, k, values=values, values_per_dim=values_per_dim,
                    item_off=item_off, item_dim=item_dim, item_lo=item_lo, item_hi=item_hi,
                    extra={"anchors": anchors, "n_dims": n_dims})


# ----------------------------------------------------------------------------
# Gaussian-mixture vectors -> p-stable LSH keywords (Sec. 4.1.1, Eqn. (plsh))
# ----------------------------------------------------------------------------

def lsh_keywords(n_vec: int, config: int, role: int, dim: int = 128, n_comp: int = 1000,
                 comp_sd: float = 4.0, within_sd: float = 1.0, n_hash: int = 256,
                 width: float = 4.0, n_buckets: int = 8192, want_vectors: bool = False):
    kw = np.empty((n_vec, n_hash), dtype=np.uint32)
    vec = np.empty((n_vec, dim), dtype=np.float32) if want_vectors else None
    comp = np.empty(n_vec, dtype=np.uint32)
    rc = _lib().synth_lsh(_seed(config, 0), _seed(config, role), n_vec, dim, n_comp, comp_sd,
                          within_sd, n_hash, width, n_buckets, _ptr(vec), _ptr(kw), _ptr(comp))
    if rc != 0:
        raise MemoryError("synth_lsh failed (%d)" % rc)
    return kw, vec, comp


def lsh(n_objects: int = 1 << 20, n_queries: int = 1024, k: int = 100, config: int = 2,
        n_hash: int = 256, n_buckets: int = 8192, **kw_args) -> Workload:
    """Objects and queries drawn from one 1000-component mixture; each vector
    becomes ``n_hash`` keywords ``i * n_buckets + bucket_i``."""
    okw, _, ocomp = lsh_keywords(n_objects, config, ROLE_OBJECTS, n_hash=n_hash,
                                 n_buckets=n_buckets, **kw_args)
    qkw, _, qcomp = lsh_keywords(n_queries, config, ROLE_QUERIES, n_hash=n_hash,
                                 n_buckets=n_buckets, **kw_args)
    obj_off = (np.arange(n_objects + 1, dtype=np.uint64) * n_hash).astype(np.uint32)
    q_off = (np.arange(n_queries + 1, dtype=np.uint64) * n_hash).astype(np.uint32)
    return Workload("lsh", "keywords", n_objects, n_hash * n_buckets, obj_off, okw.ravel(),
                    n_queries, k, q_off=q_off, q_kw=qkw.ravel(),
                    extra={"n_hash": n_hash, "n_buckets": n_buckets, "obj_comp": ocomp,
                           "q_comp": qcomp})


def lsh_training_queries(n: int, config: int = 4, n_hash: int = 256, n_buckets: int = 8192):
    """Extra queries from the training stream (same mixture and hashes)."""
    qkw, _, _ = lsh_keywords(n, config, ROLE_TRAIN, n_hash=n_hash, n_buckets=n_buckets)
    q_off = (np.arange(n + 1, dtype=np.uint64) * n_hash).astype(np.uint32)
    return q_off, qkw.ravel()


# ----------------------------------------------------------------------------
# Zipf keyword sets (Sec. 5.1-5.2 stand-ins)
# ----------------------------------------------------------------------------

def zipf_sets(n_sets: int, len_lo: int, len_hi: int, vocab: int, config: int, role: int,
              s: float = 1.1):
    lens = np.empty(n_sets, dtype=np.uint32)
    _lib().synth_set_lengths(_seed(config, role), n_sets, len_lo, len_hi, _ptr(lens))
    off = np.zeros(n_sets + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    perm = np.empty(vocab, dtype=np.uint32)
    _lib().synth_permutation(_seed(config, 0), vocab, _ptr(perm))
    kw = np.empty(int(off[-1]), dtype=np.uint32)
    rc = _lib().synth_zipf_sets(_seed(config, role), n_sets, vocab, s, _ptr(perm), _ptr(off),
                                _ptr(kw))
    if rc != 0:
        raise ValueError("synth_zipf_sets failed (%d)" % rc)
    return off, kw


def sets(n_objects: int = 1 << 22, obj_len=(16, 256), vocab: int = 1 << 20,
         n_queries: int = 8192, q_len=(8, 512), k=10, config: int = 3, s: float = 1.1) -> Workload:
    """Objects and queries are Zipf(s) keyword sets (distinct keywords; ranks
    mapped to ids by a seeded permutation)."""
    ooff, okw = zipf_sets(n_objects, obj_len[0], obj_len[1], vocab, config, ROLE_OBJECTS, s)
    qoff, qkw = zipf_sets(n_queries, q_len[0], q_len[1], vocab, config, ROLE_QUERIES, s)
    if int(ooff[-1]) >= 1 << 32:
        raise ValueError("more than 2^32 postings")
    return Workload("sets", "keywords", n_objects, vocab, ooff.astype(np.uint32), okw,
                    n_queries, k, q_off=qoff.astype(np.uint32), q_kw=qkw,
                    extra={"obj_len": obj_len, "q_len": q_len, "zipf_s": s})


def serving_requests(n_requests: int, rate_qps: float, config: int = 5, vocab: int = 1 << 22,
                     q_len=(8, 512), ks=(1, 10, 100), s: float = 1.1):
    """Request stream: Poisson arrivals at ``rate_qps``, Zipf keyword sets and
    k drawn uniformly from ``ks``."""
    qoff, qkw = zipf_sets(n_requests, q_len[0], q_len[1], vocab, config, ROLE_QUERIES, s)
    rng = np.random.default_rng([SEED_BASE + config, ROLE_QUERIES, 7])
    arrivals = np.cumsum(rng.exponential(1.0 / rate_qps, size=n_requests))
    k = np.asarray(ks, dtype=np.uint32)[rng.integers(0, len(ks), size=n_requests)]
    return qoff.astype(np.uint32), qkw, k, arrivals


# ----------------------------------------------------------------------------
# The five named workloads at full size
# ----------------------------------------------------------------------------

def config(n: int) -> Workload:
    if n == 1:
        return relational()
    if n == 2:
        return lsh(1_000_000, 1024, 100, config=2)
    if n == 3:
        return sets(4_000_000, (16, 256), 1 << 20, 8192, (8, 512), 10, config=3)
    if n == 4:
        return lsh(4_000_000, 4096, 100, config=4)
    if n == 5:
        w = sets(8_000_000, (64, 64), 1 << 22, 1024, (8, 512), 10, config=5)
        rng = np.random.default_rng([SEED_BASE + 5, ROLE_QUERIES, 9])
        w.k = np.asarray([1, 10, 100], dtype=np.uint32)[rng.integers(0, 3, size=w.n_queries)]
        return w
    raise ValueError("config must be 1..5")


@dataclass
class Sequences:
    """Data and query sequences over the alphabet 0 .. sigma-1, in CSR form
    (``s_off[N+1]``, ``s_chars``; ``q_off[Q+1]``, ``q_chars``, uint8 chars).
    ``q_src[q]`` is the data sequence query q was edited from and
    ``q_edits[q]`` how many edits were applied."""
    n_seqs: int
    sigma: int
    s_off: np.ndarray
    s_chars: np.ndarray
    n_queries: int
    q_off: np.ndarray
    q_chars: np.ndarray
    q_src: np.ndarray
    q_edits: np.ndarray

    def subset(self, qids) -> "Sequences":
        qids = np.asarray(qids)
        qo = self.q_off.astype(np.int64)
        parts = [self.q_chars[qo[q]:qo[q + 1]] for q in qids]
        lens = np.array([len(p) for p in parts], np.int64)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint32)
        chars = np.concatenate(parts).astype(np.uint8) if len(parts) else np.zeros(0, np.uint8)
        return Sequences(self.n_seqs, self.sigma, self.s_off, self.s_chars, len(qids), off, chars,
                         self.q_src[qids], self.q_edits[qids])


def sequences(n_seqs: int = 1 << 20, length=(40, 100), sigma: int = 26, n_queries: int = 1024,
              edits=(1, 6), config: int = 6, s: float = 1.0) -> Sequences:
    """Strings for sequence search under edit distance (the DBLP-like case of
    Sec. 5.1): lengths uniform in ``length``, characters drawn with Zipf(s)
    frequencies over the alphabet; each query is a random data sequence with
    a uniform number of random edits in ``edits`` (substitution, insertion or
    deletion at a random position)."""
    assert 2 <= sigma <= 256
    rng_q = np.random.default_rng([SEED_BASE + config, ROLE_QUERIES])
    w = 1.0 / np.arange(1, sigma + 1, dtype=np.float64) ** s
    p = w / w.sum()
    lens = np.empty(n_seqs, np.uint32)
    _lib().synth_set_lengths(_seed(config, ROLE_OBJECTS), n_seqs, length[0], length[1],
                             _ptr(lens))
    off64 = np.concatenate([[0], np.cumsum(lens, dtype=np.uint64)]).astype(np.uint64)
    s_chars = np.empty(max(int(off64[-1]), 1), np.uint8)
    _lib().synth_chars(_seed(config, ROLE_OBJECTS), n_seqs, sigma, s, _ptr(off64), _ptr(s_chars))
    s_chars = s_chars[:int(off64[-1])]
    s_off = off64.astype(np.uint32)
    q_src = rng_q.integers(0, n_seqs, n_queries).astype(np.uint32)
    q_edits = rng_q.integers(edits[0], edits[1] + 1, n_queries).astype(np.uint32)
    qs = []
    for q in range(n_queries):
        a = list(s_chars[s_off[q_src[q]]:s_off[q_src[q] + 1]])
        for _ in range(int(q_edits[q])):
            op = rng_q.integers(0, 3)
            pos = int(rng_q.integers(0, len(a) + (1 if op == 1 else 0))) if a else 0
            c = int(rng_q.choice(sigma, p=p))
            if op == 0 and a:
                a[pos] = c
            elif op == 1 or not a:
                a.insert(pos, c)
            else:
                del a[pos]
        qs.append(np.array(a, np.uint8))
    q_off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.uint32)
    q_chars = np.concatenate(qs).astype(np.uint8)
    return Sequences(n_seqs, sigma, s_off, s_chars, n_queries, q_off, q_chars, q_src, q_edits)


def lsh_params(family: str, dim: int, n_hash: int, scale: float, config: int = 7):
    """Random draws of the LSH functions, passed to both the CUDA path and the
    oracle.  family "pstable": a_i ~ N(0, I) (n_hash x dim), b_i ~ U[0, scale)
    with scale = the bucket width w.  family "rbh": grid cell sizes
    g_i[d] ~ Gamma(2, scale) with scale = the Laplacian kernel width sigma,
    shifts u_i[d] ~ U[0, g_i[d]), and 32-bit re-hash keys."""
    rng = np.random.default_rng([SEED_BASE + config, 11, 0 if family == "pstable" else 1])
    if family == "pstable":
        a = rng.standard_normal((n_hash, dim)).astype(np.float32)
        b = (rng.random(n_hash) * scale).astype(np.float32)
        return {"a": a, "b": b, "w": np.float32(scale)}
    g = np.maximum(rng.gamma(2.0, scale, (n_hash, dim)), 1e-6).astype(np.float32)
    u = (rng.random((n_hash, dim)) * g).astype(np.float32)
    key = rng.integers(0, 1 << 32, n_hash, dtype=np.uint64).astype(np.uint32)
    return {"g": g, "u": u, "key": key}
