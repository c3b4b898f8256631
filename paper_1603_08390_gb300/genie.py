"""Python binding of the C ABI in ``include/genie.h`` (ctypes, same names).

Argument marshalling only: device buffers are passed as torch CUDA tensors
(or raw integer addresses), streams as ``torch.cuda.Stream`` (or a raw
``cudaStream_t`` integer; default: torch's current stream).  Every step of
the search runs in ``libgenie.so``; if that library is missing this module
raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgenie.so")

GENIE_OK = 0
GENIE_ERR_INVALID_ARG = 1
GENIE_ERR_OUT_OF_MEMORY = 2
GENIE_ERR_CUDA = 3
GENIE_ERR_CAPACITY = 4
GENIE_ERR_TIMEOUT = 5
GENIE_MAX_K = 1024
GENIE_MAX_BOUND = 4095
GENIE_SEARCH_PER_RANGE_AT = 1
GENIE_SEARCH_NO_GATE = 2
GENIE_SEARCH_NO_DENSE = 4
GENIE_SEARCH_DENSE = 8
GENIE_NO_DENSE = 0xFFFFFFFF
N_FEATURES = 64

EXPORTED = (
    "genie_last_error", "genie_version", "genie_build_index", "genie_index_destroy",
    "genie_index_get_info", "genie_index_export", "genie_make_queries", "genie_compile_ranges",
    "genie_queries_destroy", "genie_queries_get_info", "genie_queries_export", "genie_search",
    "genie_search_shape", "genie_search_noalloc", "genie_mlp_num_params", "genie_mlp_create", "genie_mlp_destroy",
    "genie_mlp_set_params", "genie_mlp_get_params", "genie_mlp_forward", "genie_mlp_gradients",
    "genie_mlp_adam_step", "genie_mlp_train", "genie_mlp_seeds", "genie_autotune",
    "genie_batch_create", "genie_batch_get_info", "genie_batch_destroy", "genie_batch_run",
    "genie_server_clock", "genie_server_create", "genie_server_destroy", "genie_server_submit",
    "genie_server_poll", "genie_server_get_stats", "genie_server_replay", "genie_calibrate",
    "genie_search_host", "genie_search_spq", "genie_merge_host", "genie_build_index_ex",
    "genie_parts_create", "genie_parts_destroy", "genie_parts_add", "genie_parts_get_info",
    "genie_parts_search", "genie_sa_grams", "genie_sa_verify", "genie_lsh_pstable",
    "genie_lsh_rbh",
)


class GenieError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("genie status %d: %s" % (status, message))
        self.status = status


class PartsInfo(ctypes.Structure):
    _fields_ = [("n_parts", ctypes.c_uint32), ("vocab", ctypes.c_uint32),
                ("n_objects", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("host_bytes", ctypes.c_uint64), ("max_part_bytes", ctypes.c_uint64)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("n_objects", ctypes.c_uint32), ("vocab", ctypes.c_uint32),
                ("nnz", ctypes.c_uint64), ("max_object_len", ctypes.c_uint32),
                ("chunk_shift", ctypes.c_uint32), ("n_chunks", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
                ("dense_keywords", ctypes.c_uint32), ("dense_min_df", ctypes.c_uint32),
                ("dense_bytes", ctypes.c_uint64)]


class IndexOpts(ctypes.Structure):
    _fields_ = [("chunk_shift", ctypes.c_uint32), ("dense_min_df", ctypes.c_uint32)]


class QueriesInfo(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_uint32), ("max_bound", ctypes.c_uint32),
                ("n_keywords", ctypes.c_uint64), ("n_entries", ctypes.c_uint64),
                ("n_dense_entries", ctypes.c_uint64)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("block_shift", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("unroll", ctypes.c_uint32), ("ht_slots", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("tuned_ms", ctypes.c_float),
                ("from_cache", ctypes.c_uint32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("max_query_keywords", ctypes.c_uint32),
                ("k_max", ctypes.c_uint32), ("streams", ctypes.c_uint32),
                ("queue_capacity", ctypes.c_uint32)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("k", ctypes.c_uint32), ("n_valid", ctypes.c_uint32),
                ("t_submit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("queries", ctypes.c_uint64),
                ("deferred_admissions", ctypes.c_uint64),
                ("max_queries_in_flight", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("reserved_bytes", ctypes.c_uint64), ("slot_bytes", ctypes.c_uint64),
                ("request_bytes_base", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_uint64),
                ("bc_bytes_in_flight", ctypes.c_uint64)]


class Calibration(ctypes.Structure):
    _fields_ = [("smem_atomics_per_s", ctypes.c_double), ("sms", ctypes.c_uint32),
                ("seconds", ctypes.c_double), ("smem_red_per_s", ctypes.c_double),
                ("smem_f16_atomics_per_s", ctypes.c_double),
                ("smem_f16_red_per_s", ctypes.c_double)]


class SpqOpts(ctypes.Structure):
    _fields_ = [("buckets", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("max_bytes", ctypes.c_uint64)]


class SpqInfo(ctypes.Structure):
    _fields_ = [("count_table_bytes_per_query", ctypes.c_uint64),
                ("list_bytes_per_query", ctypes.c_uint64), ("queries_per_pass", ctypes.c_uint32),
                ("passes", ctypes.c_uint32), ("mean_iterations", ctypes.c_double)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("d_seed", ctypes.c_void_p), ("block_shift", ctypes.c_uint32),
                ("threads", ctypes.c_uint32), ("ht_slots", ctypes.c_uint32),
                ("unroll", ctypes.c_uint32),
                ("d_chunk_at", ctypes.c_void_p), ("d_stats", ctypes.c_void_p),
                ("h_blocks_per_query", ctypes.POINTER(ctypes.c_uint32)),
                ("scan_event_begin", ctypes.c_void_p), ("scan_event_end", ctypes.c_void_p),
                ("flags", ctypes.c_uint32)]


class SearchShape(ctypes.Structure):
    _fields_ = [("counter_bits", ctypes.c_uint32), ("block_shift", ctypes.c_uint32),
                ("n_groups", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("unroll", ctypes.c_uint32), ("ht_slots", ctypes.c_uint32),
                ("smem_bytes", ctypes.c_uint64), ("dense", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def kernel_name(self) -> str:
        """Name of the scan kernel this shape launches, as profilers print it."""
        log2w = {4: 2, 8: 3, 16: 4}[self.counter_bits]
        return "scan_cpq_kernel<%d, %d, %d, %s>" % (log2w, self.unroll, self.threads,
                                                   "true" if self.dense else "false")


_LIB = None
_LOCK = threading.Lock()


def load(path: Optional[str] = None):
    """Load libgenie.so (built by ``__graft_entry__.build()``)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise GenieError(GENIE_ERR_CUDA, "libgenie.so is not built (%s); run "
                             "paper_1603_08390_gb300._build.build()" % p)
        lib = ctypes.CDLL(p)
        vp, u32, u64, st = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.genie_last_error.restype = ctypes.c_char_p
        lib.genie_last_error.argtypes = []
        lib.genie_version.restype = st
        lib.genie_build_index.argtypes = [vp, vp, u32, u32, u32, vp, ctypes.POINTER(vp)]
        lib.genie_build_index.restype = st
        lib.genie_build_index_ex.argtypes = [vp, vp, u32, u32, ctypes.POINTER(IndexOpts), vp,
                                             ctypes.POINTER(vp)]
        lib.genie_build_index_ex.restype = st
        lib.genie_index_destroy.argtypes = [vp]
        lib.genie_index_destroy.restype = None
        lib.genie_index_get_info.argtypes = [vp, ctypes.POINTER(IndexInfo)]
        lib.genie_index_get_info.restype = st
        lib.genie_index_export.argtypes = [vp, vp, vp, vp]
        lib.genie_index_export.restype = st
        lib.genie_make_queries.argtypes = [vp, vp, vp, u32, vp, ctypes.POINTER(vp)]
        lib.genie_make_queries.restype = st
        lib.genie_compile_ranges.argtypes = [vp, u32, vp, vp, vp, vp, u32, vp, ctypes.POINTER(vp)]
        lib.genie_compile_ranges.restype = st
        lib.genie_queries_destroy.argtypes = [vp]
        lib.genie_queries_destroy.restype = None
        lib.genie_queries_get_info.argtypes = [vp, ctypes.POINTER(QueriesInfo)]
        lib.genie_queries_get_info.restype = st
        lib.genie_queries_export.argtypes = [vp, vp, vp, vp, vp]
        lib.genie_queries_export.restype = st
        lib.genie_search.argtypes = [vp, vp, u32, vp, ctypes.POINTER(SearchOpts), vp, vp, vp, vp]
        lib.genie_search.restype = st
        lib.genie_search_noalloc.argtypes = lib.genie_search.argtypes
        lib.genie_search_noalloc.restype = st
        lib.genie_search_host.argtypes = [vp, vp, vp, u32, u32, vp, ctypes.POINTER(SearchOpts),
                                          vp, vp, vp, vp]
        lib.genie_search_host.restype = st
        lib.genie_search_spq.argtypes = [vp, vp, u32, vp, ctypes.POINTER(SpqOpts), vp, vp, vp,
                                         ctypes.POINTER(SpqInfo), vp]
        lib.genie_search_spq.restype = st
        lib.genie_merge_host.argtypes = [u32, vp, vp, u32, u32, u32, vp, vp, vp]
        lib.genie_merge_host.restype = st
        lib.genie_search_shape.argtypes = [vp, vp, u32, ctypes.POINTER(SearchOpts),
                                           ctypes.POINTER(SearchShape)]
        lib.genie_search_shape.restype = st
        f32 = ctypes.c_float
        lib.genie_mlp_num_params.restype = u32
        lib.genie_mlp_num_params.argtypes = []
        lib.genie_mlp_create.argtypes = [u64, vp, ctypes.POINTER(vp)]
        lib.genie_mlp_destroy.argtypes = [vp]
        lib.genie_mlp_destroy.restype = None
        lib.genie_mlp_set_params.argtypes = [vp, vp, vp]
        lib.genie_mlp_get_params.argtypes = [vp, vp, vp]
        lib.genie_mlp_forward.argtypes = [vp, vp, u32, vp, vp]
        lib.genie_mlp_gradients.argtypes = [vp, vp, vp, u32, vp, vp]
        lib.genie_mlp_adam_step.argtypes = [vp, f32, vp]
        lib.genie_mlp_train.argtypes = [vp, vp, vp, u32, u32, u32, f32, ctypes.POINTER(f32), vp]
        lib.genie_mlp_seeds.argtypes = [vp, vp, f32, vp, vp]
        lib.genie_autotune.argtypes = [vp, vp, u32, ctypes.c_char_p, ctypes.POINTER(BatchOpts)]
        lib.genie_batch_create.argtypes = [vp, u32, u32, u32, ctypes.POINTER(BatchOpts),
                                           ctypes.POINTER(vp)]
        lib.genie_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchOpts)]
        lib.genie_batch_destroy.argtypes = [vp]
        lib.genie_batch_destroy.restype = None
        lib.genie_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.genie_calibrate.argtypes = [ctypes.POINTER(Calibration)]
        lib.genie_calibrate.restype = st
        lib.genie_server_clock.restype = ctypes.c_double
        lib.genie_server_clock.argtypes = []
        lib.genie_server_create.argtypes = [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
        lib.genie_server_destroy.argtypes = [vp]
        lib.genie_server_destroy.restype = None
        lib.genie_server_submit.argtypes = [vp, vp, u32, u32, u64]
        lib.genie_server_poll.argtypes = [vp, u32, u32, ctypes.POINTER(ResultInfo), vp, vp,
                                          ctypes.POINTER(u32)]
        lib.genie_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.genie_server_replay.argtypes = [vp, vp, vp, vp, vp, u32, u32, vp, vp, vp, vp]
        lib.genie_parts_create.argtypes = [ctypes.POINTER(vp)]
        lib.genie_parts_destroy.argtypes = [vp]
        lib.genie_parts_destroy.restype = None
        lib.genie_parts_add.argtypes = [vp, vp, u32, vp]
        lib.genie_parts_get_info.argtypes = [vp, ctypes.POINTER(PartsInfo)]
        lib.genie_parts_search.argtypes = [vp, vp, vp, u32, u32, vp, vp, vp, vp, vp]
        for name in ("genie_parts_create", "genie_parts_add", "genie_parts_get_info",
                     "genie_parts_search"):
            getattr(lib, name).restype = st
        lib.genie_sa_grams.argtypes = [vp, vp, u32, u32, u32, u32, vp, vp, u64,
                                       ctypes.POINTER(u64), vp]
        lib.genie_sa_grams.restype = st
        lib.genie_sa_verify.argtypes = [vp, vp, u32, vp, vp, vp, vp, vp, u32, u32, u32, u32,
                                        vp, vp, vp, vp, vp, vp]
        lib.genie_sa_verify.restype = st
        lib.genie_lsh_pstable.argtypes = [vp, u64, u32, vp, vp, u32, f32, u32, vp, vp]
        lib.genie_lsh_pstable.restype = st
        lib.genie_lsh_rbh.argtypes = [vp, u64, u32, vp, vp, vp, u32, u32, vp, vp]
        lib.genie_lsh_rbh.restype = st
        for name in ("genie_autotune", "genie_batch_create", "genie_batch_get_info",
                     "genie_batch_run", "genie_server_create", "genie_server_submit",
                     "genie_server_poll", "genie_server_get_stats", "genie_server_replay"):
            getattr(lib, name).restype = st
        for name in ("genie_mlp_create", "genie_mlp_set_params", "genie_mlp_get_params",
                     "genie_mlp_forward", "genie_mlp_gradients", "genie_mlp_adam_step",
                     "genie_mlp_train", "genie_mlp_seeds"):
            getattr(lib, name).restype = st
        _LIB = lib
        return lib


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, lib) -> None:
    if status != GENIE_OK:
        raise GenieError(status, lib.genie_last_error().decode())


def genie_last_error() -> str:
    return load().genie_last_error().decode()


def genie_version() -> int:
    return load().genie_version()


class Index:
    """Owning wrapper of a ``genie_index*``."""

    def __init__(self, handle: int):
        self.handle = handle
        info = IndexInfo()
        _check(load().genie_index_get_info(handle, ctypes.byref(info)), load())
        self.info = info

    def __getattr__(self, name):
        return getattr(self.__dict__["info"], name)

    def close(self):
        if self.handle:
            load().genie_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Queries:
    """Owning wrapper of a ``genie_queries*``."""

    def __init__(self, handle: int, index: Index):
        self.handle = handle
        self.index = index  # keeps the index alive
        info = QueriesInfo()
        _check(load().genie_queries_get_info(handle, ctypes.byref(info)), load())
        self.info = info

    def __getattr__(self, name):
        return getattr(self.__dict__["info"], name)

    def close(self):
        if self.handle:
            load().genie_queries_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def genie_build_index(d_obj_off, d_obj_kw, n_objects: int, vocab: int, chunk_shift: int = 0,
                      stream=None, dense_min_df: Optional[int] = None) -> Index:
    """Build the index; dense_min_df: None = the library's default threshold
    for object bitmaps, GENIE_NO_DENSE = none, else that list length."""
    lib = load()
    out = ctypes.c_void_p()
    if dense_min_df is None:
        _check(lib.genie_build_index(_ptr(d_obj_off), _ptr(d_obj_kw), n_objects, vocab,
                                     chunk_shift, _stream(stream), ctypes.byref(out)), lib)
    else:
        opts = IndexOpts(chunk_shift=chunk_shift, dense_min_df=dense_min_df)
        _check(lib.genie_build_index_ex(_ptr(d_obj_off), _ptr(d_obj_kw), n_objects, vocab,
                                        ctypes.byref(opts), _stream(stream), ctypes.byref(out)),
               lib)
    return Index(out.value)


def genie_index_export(index: Index, d_kw_off=None, d_post_ids=None, stream=None) -> None:
    lib = load()
    _check(lib.genie_index_export(index.handle, _ptr(d_kw_off), _ptr(d_post_ids), _stream(stream)),
           lib)


def genie_make_queries(index: Index, d_q_off, d_q_kw, n_queries: int, stream=None) -> Queries:
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.genie_make_queries(index.handle, _ptr(d_q_off), _ptr(d_q_kw), n_queries,
                                  _stream(stream), ctypes.byref(out)), lib)
    return Queries(out.value, index)


def genie_compile_ranges(index: Index, values_per_dim: int, d_item_off, d_dim, d_lo, d_hi,
                         n_queries: int, stream=None) -> Queries:
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.genie_compile_ranges(index.handle, values_per_dim, _ptr(d_item_off), _ptr(d_dim),
                                    _ptr(d_lo), _ptr(d_hi), n_queries, _stream(stream),
                                    ctypes.byref(out)), lib)
    return Queries(out.value, index)


def genie_queries_export(queries: Queries, d_bound=None, d_entries=None, d_features=None,
                         stream=None) -> None:
    lib = load()
    _check(lib.genie_queries_export(queries.handle, _ptr(d_bound), _ptr(d_entries),
                                    _ptr(d_features), _stream(stream)), lib)


def make_opts(d_seed=None, block_shift: int = 0, threads: int = 0, ht_slots: int = 0,
              d_chunk_at=None, d_stats=None, scan_events=None, unroll: int = 0,
              flags: int = 0) -> SearchOpts:
    o = SearchOpts()
    o.d_seed = _ptr(d_seed)
    o.block_shift = block_shift
    o.threads = threads
    o.ht_slots = ht_slots
    o.unroll = unroll
    o.flags = flags
    o.d_chunk_at = _ptr(d_chunk_at)
    o.d_stats = _ptr(d_stats)
    o._blocks = ctypes.c_uint32(0)
    o.h_blocks_per_query = ctypes.pointer(o._blocks)
    if scan_events is not None:  # (begin, end): torch.cuda.Event or raw cudaEvent_t
        b, e = scan_events
        o.scan_event_begin = b if isinstance(b, int) else b.cuda_event
        o.scan_event_end = e if isinstance(e, int) else e.cuda_event
    return o


def genie_search(index: Index, queries: Queries, k: int, d_ids, d_counts, d_n_valid, d_k=None,
                 opts: Optional[SearchOpts] = None, stream=None) -> None:
    lib = load()
    _check(lib.genie_search(index.handle, queries.handle, k, _ptr(d_k),
                            ctypes.byref(opts) if opts is not None else None, _ptr(d_ids),
                            _ptr(d_counts), _ptr(d_n_valid), _stream(stream)), lib)


def genie_search_host(index: Index, h_q_off, h_q_kw, n_queries: int, k: int, h_ids, h_counts,
                      h_n_valid, h_k=None, opts: Optional[SearchOpts] = None, stream=None) -> None:
    """Queries and results in host memory: copy in, compile, search, copy back
    (one C call; returns when the results are in the host buffers).  Host
    buffers are CPU tensors (pinned for full copy speed) or raw addresses."""
    lib = load()
    _check(lib.genie_search_host(index.handle, _ptr(h_q_off), _ptr(h_q_kw), n_queries, k,
                                 _ptr(h_k), ctypes.byref(opts) if opts is not None else None,
                                 _ptr(h_ids), _ptr(h_counts), _ptr(h_n_valid), _stream(stream)),
           lib)


def genie_search_spq(index: Index, queries: Queries, k: int, d_ids, d_counts, d_n_valid, d_k=None,
                     buckets: int = 0, max_bytes: int = 0, stream=None,
                     want_info: bool = True) -> Optional[SpqInfo]:
    """The GEN-SPQ ablation: dense Count Table + bucket k-selection (same
    results).  want_info=False skips the statistics (and their synchronisation)."""
    lib = load()
    info = SpqInfo() if want_info else None
    opts = SpqOpts(buckets=buckets, max_bytes=max_bytes)
    _check(lib.genie_search_spq(index.handle, queries.handle, k, _ptr(d_k), ctypes.byref(opts),
                                _ptr(d_ids), _ptr(d_counts), _ptr(d_n_valid),
                                ctypes.byref(info) if info is not None else None,
                                _stream(stream)), lib)
    return info


def genie_merge_host(ids_parts, counts_parts, k: int):
    """Exact host merge of per-part result lists (numpy uint32 [Q, k_part]
    each, global ids) into the top-k (ids, counts, n_valid)."""
    import numpy as np
    lib = load()
    P = len(ids_parts)
    ids_parts = [np.ascontiguousarray(a, dtype=np.uint32) for a in ids_parts]
    counts_parts = [np.ascontiguousarray(a, dtype=np.uint32) for a in counts_parts]
    Q, kp = ids_parts[0].shape
    pi = (ctypes.c_void_p * P)(*[a.ctypes.data for a in ids_parts])
    pc = (ctypes.c_void_p * P)(*[a.ctypes.data for a in counts_parts])
    ids = np.empty((Q, k), dtype=np.uint32)
    cnt = np.empty((Q, k), dtype=np.uint32)
    nv = np.empty(Q, dtype=np.uint32)
    _check(lib.genie_merge_host(P, pi, pc, Q, kp, k, ids.ctypes.data, cnt.ctypes.data,
                                nv.ctypes.data), lib)
    return ids, cnt, nv


def genie_search_shape(index: Index, queries: Queries, k: int,
                       opts: Optional[SearchOpts] = None) -> SearchShape:
    """The scan kernel's launch shape genie_search would use (host only)."""
    lib = load()
    out = SearchShape()
    _check(lib.genie_search_shape(index.handle, queries.handle, k,
                                  ctypes.byref(opts) if opts is not None else None,
                                  ctypes.byref(out)), lib)
    return out


def genie_search_noalloc(index: Index, queries: Queries, k: int, d_ids, d_counts, d_n_valid,
                         d_k=None, opts: Optional[SearchOpts] = None, stream=None) -> None:
    """genie_search with its scratch in the library's fixed device array: for
    callers that cannot allocate device memory while answering queries (see
    include/genie.h for the size limit and the sharing rules)."""
    lib = load()
    _check(lib.genie_search_noalloc(index.handle, queries.handle, k, _ptr(d_k),
                                    ctypes.byref(opts) if opts is not None else None, _ptr(d_ids),
                                    _ptr(d_counts), _ptr(d_n_valid), _stream(stream)), lib)


class MLP:
    """Owning wrapper of a ``genie_mlp*`` (the k-th-count predictor)."""

    def __init__(self, seed: int = 0, stream=None):
        lib = load()
        out = ctypes.c_void_p()
        _check(lib.genie_mlp_create(seed, _stream(stream), ctypes.byref(out)), lib)
        self.handle = out.value
        self.n_params = lib.genie_mlp_num_params()

    def close(self):
        if self.handle:
            load().genie_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, d_theta, stream=None):
        _check(load().genie_mlp_set_params(self.handle, _ptr(d_theta), _stream(stream)), load())

    def get_params(self, d_theta, stream=None):
        _check(load().genie_mlp_get_params(self.handle, _ptr(d_theta), _stream(stream)), load())

    def forward(self, d_x, n: int, d_y, stream=None):
        _check(load().genie_mlp_forward(self.handle, _ptr(d_x), n, _ptr(d_y), _stream(stream)), load())

    def gradients(self, d_x, d_t, n: int, d_grad=None, stream=None):
        _check(load().genie_mlp_gradients(self.handle, _ptr(d_x), _ptr(d_t), n, _ptr(d_grad),
                                          _stream(stream)), load())

    def adam_step(self, lr: float, stream=None):
        _check(load().genie_mlp_adam_step(self.handle, lr, _stream(stream)), load())

    def train(self, d_x, d_t, n: int, epochs: int, batch: int, lr: float, stream=None) -> float:
        loss = ctypes.c_float(0.0)
        _check(load().genie_mlp_train(self.handle, _ptr(d_x), _ptr(d_t), n, epochs, batch, lr,
                                      ctypes.byref(loss), _stream(stream)), load())
        return float(loss.value)

    def seeds(self, queries: Queries, margin: float, d_seed, stream=None):
        _check(load().genie_mlp_seeds(self.handle, queries.handle, margin, _ptr(d_seed),
                                      _stream(stream)), load())


def genie_autotune(index: Index, sample: Queries, k: int, cache_path: Optional[str] = None) -> BatchOpts:
    lib = load()
    out = BatchOpts()
    _check(lib.genie_autotune(index.handle, sample.handle, k,
                              cache_path.encode() if cache_path else None, ctypes.byref(out)), lib)
    return out


def genie_lsh_pstable(d_points, n_points: int, dim: int, d_a, d_b, m: int, w: float, D: int,
                      d_kw, stream=None) -> None:
    lib = load()
    _check(lib.genie_lsh_pstable(_ptr(d_points), n_points, dim, _ptr(d_a), _ptr(d_b), m, w, D,
                                 _ptr(d_kw), _stream(stream)), lib)


def genie_lsh_rbh(d_points, n_points: int, dim: int, d_g, d_u, d_key, m: int, D: int, d_kw,
                  stream=None) -> None:
    lib = load()
    _check(lib.genie_lsh_rbh(_ptr(d_points), n_points, dim, _ptr(d_g), _ptr(d_u), _ptr(d_key), m,
                             D, _ptr(d_kw), _stream(stream)), lib)


def genie_sa_grams(d_off, d_chars, n_seqs: int, n: int, sigma: int, R: int, d_kw_off, d_kw,
                   kw_capacity: int, stream=None) -> int:
    """Ordered n-gram keywords of sequences; returns the number written."""
    lib = load()
    total = ctypes.c_uint64()
    _check(lib.genie_sa_grams(_ptr(d_off), _ptr(d_chars), n_seqs, n, sigma, R, _ptr(d_kw_off),
                              _ptr(d_kw), kw_capacity, ctypes.byref(total), _stream(stream)), lib)
    return int(total.value)


def genie_sa_verify(d_q_off, d_q_chars, n_queries: int, d_s_off, d_s_chars, d_cand_ids,
                    d_cand_counts, d_cand_n, K: int, k: int, n: int, max_query_len: int, d_ids,
                    d_ed, d_n_out, d_certified, d_examined, stream=None) -> None:
    lib = load()
    _check(lib.genie_sa_verify(_ptr(d_q_off), _ptr(d_q_chars), n_queries, _ptr(d_s_off),
                               _ptr(d_s_chars), _ptr(d_cand_ids), _ptr(d_cand_counts),
                               _ptr(d_cand_n), K, k, n, max_query_len, _ptr(d_ids), _ptr(d_ed),
                               _ptr(d_n_out), _ptr(d_certified), _ptr(d_examined),
                               _stream(stream)), lib)


class Parts:
    """Owning wrapper of a ``genie_parts*``: an index in parts held in pinned
    host memory and searched part by part (multiple loadings)."""

    def __init__(self):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.genie_parts_create(ctypes.byref(h)), lib)
        self.handle = h.value

    def add(self, index: "Index", id_base: int, stream=None) -> None:
        lib = load()
        _check(lib.genie_parts_add(self.handle, index.handle, id_base, _stream(stream)), lib)

    @property
    def info(self) -> PartsInfo:
        lib = load()
        out = PartsInfo()
        _check(lib.genie_parts_get_info(self.handle, ctypes.byref(out)), lib)
        return out

    def search(self, d_q_off, d_q_kw, n_queries: int, k: int, d_ids, d_counts, d_n_valid,
               d_k=None, stream=None) -> None:
        lib = load()
        _check(lib.genie_parts_search(self.handle, _ptr(d_q_off), _ptr(d_q_kw), n_queries, k,
                                      _ptr(d_k), _ptr(d_ids), _ptr(d_counts), _ptr(d_n_valid),
                                      _stream(stream)), lib)

    def close(self):
        if self.handle:
            load().genie_parts_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper of a ``genie_batch*`` (persistent, graph-captured plan)."""

    def __init__(self, index: Index, max_queries: int, max_bound: int, k: int,
                 opts: Optional[BatchOpts] = None):
        lib = load()
        out = ctypes.c_void_p()
        _check(lib.genie_batch_create(index.handle, max_queries, max_bound, k,
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.byref(out)), lib)
        self.handle = out.value
        self.index = index
        self.k = k
        info = BatchOpts()
        _check(lib.genie_batch_get_info(self.handle, ctypes.byref(info)), lib)
        self.info = info

    def run(self, queries: Queries, d_ids, d_counts, d_n_valid, d_k=None, stream=None):
        lib = load()
        _check(lib.genie_batch_run(self.handle, queries.handle, _ptr(d_k), _ptr(d_ids),
                                   _ptr(d_counts), _ptr(d_n_valid), _stream(stream)), lib)

    def close(self):
        if self.handle:
            load().genie_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of a ``genie_server*`` (continuous-batching serving loop).
    Host arrays are numpy arrays."""

    def __init__(self, index: Index, opts: Optional[ServerOpts] = None):
        lib = load()
        out = ctypes.c_void_p()
        _check(lib.genie_server_create(index.handle, ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(out)), lib)
        self.handle = out.value
        self.index = index
        self.k_max = opts.k_max if (opts is not None and opts.k_max) else 100

    @staticmethod
    def clock() -> float:
        return load().genie_server_clock()

    def submit(self, kw, k: int, tag: int):
        import numpy as np
        kw = np.ascontiguousarray(kw, dtype=np.uint32)
        _check(load().genie_server_submit(self.handle, kw.ctypes.data_as(ctypes.c_void_p), len(kw),
                                          k, tag), load())

    def poll(self, max_results: int = 64, timeout_us: int = 0):
        """List of (info, ids, counts) for completed requests."""
        import numpy as np
        info = (ResultInfo * max(1, max_results))()
        ids = np.empty((max(1, max_results), self.k_max), dtype=np.uint32)
        cnt = np.empty_like(ids)
        n = ctypes.c_uint32(0)
        _check(load().genie_server_poll(self.handle, max_results, timeout_us, info,
                                        ids.ctypes.data_as(ctypes.c_void_p),
                                        cnt.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)), load())
        return [(info[j], ids[j, :info[j].k].copy(), cnt[j, :info[j].k].copy())
                for j in range(n.value)]

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(load().genie_server_get_stats(self.handle, ctypes.byref(st)), load())
        return st

    def replay(self, q_off, q_kw, ks, arrival_s, timeout_ms: int = 600000):
        """Open-loop replay; returns (latency_s, ids, counts, n_valid)."""
        import numpy as np
        q_off = np.ascontiguousarray(q_off, dtype=np.uint32)
        q_kw = np.ascontiguousarray(q_kw, dtype=np.uint32)
        ks = np.ascontiguousarray(ks, dtype=np.uint32)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        n = len(ks)
        lat = np.empty(n, dtype=np.float64)
        ids = np.empty((n, self.k_max), dtype=np.uint32)
        cnt = np.empty_like(ids)
        nv = np.empty(n, dtype=np.uint32)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().genie_server_replay(self.handle, p(q_off), p(q_kw), p(ks), p(arr), n,
                                          timeout_ms, p(lat), p(ids), p(cnt), p(nv)), load())
        return lat, ids, cnt, nv

    def close(self):
        if self.handle:
            load().genie_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def genie_calibrate() -> Calibration:
    lib = load()
    out = Calibration()
    _check(lib.genie_calibrate(ctypes.byref(out)), lib)
    return out
