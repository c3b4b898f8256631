"""CPU oracle for match-count top-k search.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1603_08390_gb300``)
and never imports it; both sides take their inputs from ``synth``.

Contents
  * ``topk``      -- brute force of Definition 2.1 over every (query, object)
                     pair, then the (count desc, id asc) ranking (C++,
                     ``mc_oracle.cpp``).
  * ``cpuidx_topk`` -- an independent inverted-index scan into a dense count
                     array plus partial sort, after the CPU-Idx competitor of
                     Sec. 6.1.2 (C++).
  * ``counts``    -- the full count matrix for small cases.
  * ``cpq``       -- a serial replay of Algorithm 1 (pure Python, small cases).
  * ``mlp``       -- the k-th-count predictor network in float64 numpy.
  * ``lsh``       -- LSH keywords of points (Sec. 4.1): p-stable hashing and
                     random binning with its re-hash (C++, ``lsh_oracle.cpp``).
  * ``sa``        -- sequence search by ordered n-grams (Sec. 5.1): n-gram
                     keywords, edit distance (C++, ``sa_oracle.cpp``), the
                     verification of Algorithm 2 and the check of Theorem 5.2.

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``mc_oracle.cpp``, ``sa_oracle.cpp`` and ``lsh_oracle.cpp``
    (g++ -O3, OpenMP, no floating-point contraction) into ``oracle/_build``."""
    out_dir = os.path.join(_HERE, "_build")
    so = os.path.join(out_dir, "liboracle.so")
    srcs = [os.path.join(_HERE, x) for x in ("mc_oracle.cpp", "sa_oracle.cpp", "lsh_oracle.cpp")]
    if (not force and os.path.exists(so)
            and all(os.path.getmtime(so) >= os.path.getmtime(x) for x in srcs)):
        return so
    os.makedirs(out_dir, exist_ok=True)
    tmp = so + ".%d.tmp" % os.getpid()
    subprocess.check_call(["g++", "-O3", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", tmp] + srcs)
    os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            u32, p, i = ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
            lib.oracle_max_threads.argtypes = [i]
            lib.oracle_max_threads.restype = i
            lib.oracle_topk_keywords.argtypes = [u32, p, p, u32, u32, p, p, p, u32, u32, u32,
                                                 p, p, p, p, p, i]
            lib.oracle_topk_keywords.restype = i
            lib.oracle_topk_relational.argtypes = [u32, u32, p, u32, p, p, p, p, p, u32, u32,
                                                   u32, p, p, p, p, p, i]
            lib.oracle_topk_relational.restype = i
            lib.oracle_counts_keywords.argtypes = [u32, p, p, u32, u32, p, p, p]
            lib.oracle_counts_keywords.restype = i
            lib.cpuidx_topk_keywords.argtypes = [u32, p, p, u32, u32, p, p, p, u32, p, p, p,
                                                 p, p, i]
            lib.cpuidx_topk_keywords.restype = i
            u64 = ctypes.c_uint64
            lib.oracle_ed.argtypes = [p, u32, p, u32]
            lib.oracle_ed.restype = u32
            lib.oracle_ed_pairs.argtypes = [p, p, p, p, u64, p, p]
            lib.oracle_ed_pairs.restype = i
            lib.oracle_sa_grams.argtypes = [u32, p, p, u32, u32, u32, p, p]
            lib.oracle_sa_grams.restype = i
            lib.oracle_sa_topk_ed.argtypes = [u32, p, p, u32, p, p, u32, p, p]
            lib.oracle_sa_topk_ed.restype = i
            f32 = ctypes.c_float
            lib.oracle_lsh_pstable.argtypes = [u64, u32, p, u32, p, p, f32, u32, p]
            lib.oracle_lsh_pstable.restype = i
            lib.oracle_lsh_rbh.argtypes = [u64, u32, p, u32, p, p, p, u32, p]
            lib.oracle_lsh_rbh.restype = i
            _LIB = lib
    return _LIB


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads(n: int = 0) -> int:
    """Threads the oracle will use (``n > 0`` sets it)."""
    return int(_lib().oracle_max_threads(n))


def _karr(k, n_q):
    if np.isscalar(k):
        return np.full(n_q, int(k), dtype=np.uint32)
    return _c(k, np.uint32)


def _outputs(n_q, stride):
    return (np.empty((n_q, stride), np.uint32), np.empty((n_q, stride), np.uint32),
            np.empty(n_q, np.uint32), np.empty(n_q, np.uint32), np.empty(n_q, np.uint64))


def topk(w, k=None, obj_range=None, n_threads: int = 0) -> dict:
    """Brute-force top-k of every query of workload ``w`` (a ``synth.Workload``).

    Returns ``ids``/``counts`` (Q x max k; unused slots id 0xFFFFFFFF, count 0),
    ``n_valid``, ``tk`` (k-th count, 0 if fewer than k objects match) and
    ``mcsum`` (sum of MC over all ranked objects).  ``obj_range=(lo, hi)``
    ranks only objects with lo <= id < hi.
    """
    k = w.k if k is None else k
    karr = _karr(k, w.n_queries)
    stride = int(karr.max()) if len(karr) else 1
    lo, hi = (0, w.n_objects) if obj_range is None else obj_range
    ids, counts, nv, tk, ms = _outputs(w.n_queries, stride)
    if w.kind == "keywords":
        oo, ok = _c(w.obj_off, np.uint32), _c(w.obj_kw, np.uint32)
        qo, qk = _c(w.q_off, np.uint32), _c(w.q_kw, np.uint32)
        rc = _lib().oracle_topk_keywords(w.n_objects, _p(oo), _p(ok), w.vocab, w.n_queries,
                                         _p(qo), _p(qk), _p(karr), stride, lo, hi, _p(ids),
                                         _p(counts), _p(nv), _p(tk), _p(ms), n_threads)
    else:
        vals = _c(w.values, np.uint32)
        io, idim = _c(w.item_off, np.uint32), _c(w.item_dim, np.uint32)
        ilo, ihi = _c(w.item_lo, np.int32), _c(w.item_hi, np.int32)
        rc = _lib().oracle_topk_relational(w.n_objects, vals.shape[1], _p(vals), w.n_queries,
                                           _p(io), _p(idim), _p(ilo), _p(ihi), _p(karr), stride,
                                           lo, hi, _p(ids), _p(counts), _p(nv), _p(tk), _p(ms),
                                           n_threads)
    if rc != 0:
        raise ValueError("oracle rejected the input (status %d)" % rc)
    return {"ids": ids, "counts": counts, "n_valid": nv, "tk": tk, "mcsum": ms, "k": karr}


def cpuidx_topk(w, k=None, n_threads: int = 0) -> dict:
    """Top-k by the inverted-index scan (keyword workloads only)."""
    assert w.kind == "keywords"
    k = w.k if k is None else k
    karr = _karr(k, w.n_queries)
    stride = int(karr.max()) if len(karr) else 1
    ids, counts, nv, tk, ms = _outputs(w.n_queries, stride)
    oo, ok = _c(w.obj_off, np.uint32), _c(w.obj_kw, np.uint32)
    qo, qk = _c(w.q_off, np.uint32), _c(w.q_kw, np.uint32)
    rc = _lib().cpuidx_topk_keywords(w.n_objects, _p(oo), _p(ok), w.vocab, w.n_queries, _p(qo),
                                     _p(qk), _p(karr), stride, _p(ids), _p(counts), _p(nv),
                                     _p(tk), _p(ms), n_threads)
    if rc != 0:
        raise ValueError("cpuidx rejected the input (status %d)" % rc)
    return {"ids": ids, "counts": counts, "n_valid": nv, "tk": tk, "mcsum": ms, "k": karr}


def counts(obj_off, obj_kw, vocab, q_off, q_kw) -> np.ndarray:
    """MC(Q, O) for every pair, as a (Q, N) uint32 matrix (keyword queries)."""
    oo, ok = _c(obj_off, np.uint32), _c(obj_kw, np.uint32)
    qo, qk = _c(q_off, np.uint32), _c(q_kw, np.uint32)
    n_obj, n_q = len(oo) - 1, len(qo) - 1
    mc = np.empty((n_q, n_obj), np.uint32)
    rc = _lib().oracle_counts_keywords(n_obj, _p(oo), _p(ok), int(vocab), n_q, _p(qo), _p(qk),
                                       _p(mc))
    if rc != 0:
        raise ValueError("oracle rejected the input (status %d)" % rc)
    return mc
