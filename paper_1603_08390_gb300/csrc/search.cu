// The search hot path: postings-list scan fused with the count priority queue
// (Sec. 3.2, Sec. 3.3, Algorithm 1, Theorem 3.1) and the exact top-k read-out.
//
// GB300 layout.  The paper keeps one Bitmap Counter per query in global
// memory and lets one block scan one query item.  Here one thread block owns
// one (query, object-id range) pair and keeps that range's Bitmap Counter,
// ZipperArray, AuditThreshold and Hash Table in shared memory, so every
// counter update is an on-chip sub-word atomic.  The object-id range is a
// union of the sublists of Sec. 3.2.1 (the index stores, per keyword, where
// each range of 2^chunk_shift ids starts), so a block reads exactly the
// postings of its range: lists are contiguous and read with aligned 16-byte
// loads, one warp per tile.  Blocks are ordered range-major so that the blocks
// resident at one time share one range of the List Array in L2.
//
// Each range yields its own exact top-k (Theorem 3.1 per range); a second
// kernel merges the ranges of a query, which is the per-part merge of the
// multiple-loading method (Sec. 3.4) done on the device.
//
// Readings (the paper is silent or loose on these):
//  * Gate: a posting that raises an object's count to val passes the Gate
//    when val >= AT (Algorithm 1); AT is read without locking, and a stale
//    (smaller) AT only lets more objects through.  ZA[val] counts passes; AT
//    only grows (atomicMax), and a final pass sets AT_f = min{i >= AT :
//    ZA[i] < k}.  For i >= AT_f, ZA[i] is exactly the number of objects with
//    count >= i, so AT_f - 1 is the k-th count (Theorem 3.1).
//  * Hash Table: holds candidate object ids.  A Gate pass at level val is
//    numbered z by its ZipperArray increment; the first k passes of a level
//    (z < k) insert their object unless it is already present (a presence
//    bit per object).  Counts live in the Bitmap Counter, so an entry whose
//    object's count is below AT - 1 is expired and may be overwritten (Sec.
//    3.3.2); the overwritten object loses its presence bit.  Every object
//    with count >= AT_f passed level AT_f with z < k, so it was inserted and
//    never expired.  The read-out is certified by its size: exactly
//    ZA[AT_f] objects have count >= AT_f.  A read-out that fails the check
//    (an insert that found no slot, or a lost race) is redone from the
//    Bitmap Counter, so the result never depends on the hash table's luck.
//  * Ties at the k-th count are filled in ascending object id from the
//    Bitmap Counter (the paper breaks them randomly).
//  * A warp counts a tile of postings, then tests the tile once (can any
//    posting's new count reach AT?  With headroom in the counter lanes this
//    is one add per old counter word) and runs the Gate only for the slots
//    that pass, one ZipperArray add per pass; the pass that fills a level to
//    k advances AT.
//  * AT seeds: a range that finishes adds the counts it reports to its
//    query's histogram and publishes the k-th largest of them, a lower bound
//    of the query's k-th count; later ranges start their AT there, and ties
//    below the seed are left out (they cannot reach the query's top-k).  A
//    range that starts with no seed selects its k-th count from the Bitmap
//    Counter after counting instead of running the Gate from AT = 1.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "cpq_device.cuh"
#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

// seeded search: queries whose result cannot be certified
__global__ void verify_seeded_kernel(uint32_t n_queries, uint32_t k, const uint32_t* __restrict__ k_arr,
                                     const uint32_t* __restrict__ seed, const uint32_t* __restrict__ counts,
                                     const uint32_t* __restrict__ n_valid, uint32_t* __restrict__ rerun,
                                     uint32_t* n_rerun) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_queries; q += gridDim.x * blockDim.x) {
    const uint32_t kq = k_arr ? k_arr[q] : k;
    const uint32_t s = seed[q];
    bool ok = s <= 1 || (n_valid[q] == kq && counts[(unsigned long long)q * k + kq - 1] >= s);
    if (!ok) rerun[atomicAdd(n_rerun, 1u)] = q;
  }
}

__global__ void add_stat_kernel(unsigned long long* stat, uint32_t v) { *stat += v; }

template <int LOG2W, int U, int THREADS>
cudaError_t launch_scan(const ScanArgs& a, const Plan& p, cudaStream_t s) {
  // the dense instantiation exists for 8- and 16-bit counters
  auto kern = (LOG2W >= 3 && p.dense) ? scan_cpq_kernel<LOG2W, U, THREADS, LOG2W >= 3>
                                      : scan_cpq_kernel<LOG2W, U, THREADS, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  const uint64_t blocks = (uint64_t)a.n_sel * a.n_groups;
  kern<<<(uint32_t)blocks, p.threads, p.smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOG2W>
cudaError_t dispatch_width(const ScanArgs& a, const Plan& p, cudaStream_t s) {
  if (p.threads == 512) return p.unroll == 8 ? launch_scan<LOG2W, 8, 512>(a, p, s)
                             : p.unroll == 2 ? launch_scan<LOG2W, 2, 512>(a, p, s)
                                             : launch_scan<LOG2W, 4, 512>(a, p, s);
  if (p.threads == 768) return p.unroll == 4 ? launch_scan<LOG2W, 4, 768>(a, p, s)
                                             : launch_scan<LOG2W, 2, 768>(a, p, s);
  if (p.threads == 896) return launch_scan<LOG2W, 2, 896>(a, p, s);
  return p.unroll == 4 ? launch_scan<LOG2W, 4, 1024>(a, p, s) : launch_scan<LOG2W, 2, 1024>(a, p, s);
}

cudaError_t dispatch_scan(const ScanArgs& a, const Plan& p, cudaStream_t s) {
  return p.log2w == 2 ? dispatch_width<2>(a, p, s)
       : p.log2w == 3 ? dispatch_width<3>(a, p, s)
                      : dispatch_width<4>(a, p, s);
}

// at_hint: [n_sel] zeroed device words shared by a query's ranges, or NULL;
// hint_hist: [n_sel][p.za_len] zeroed words (the ranges' reported counts), or NULL
cudaError_t run_pass(const genie_index* idx, const genie_queries* qs, uint32_t k, const uint32_t* d_k,
                     const uint32_t* seed, const uint32_t* sel, uint32_t n_sel, const Plan& p,
                     const genie_search_opts* o, unsigned long long* cand, uint32_t* at_hint,
                     uint32_t* hint_hist, uint32_t* ids, uint32_t* counts, uint32_t* n_valid,
                     cudaStream_t s) {
  ScanArgs a{};  // fields left unset are zero (NULL)
  a.kw_off = idx->kw_off;
  a.post_ids = idx->post_ids;
  a.chunk_pos = idx->chunk_pos;
  a.n_chunks = idx->n_chunks;
  a.chunk_shift = idx->chunk_shift;
  a.n_objects = idx->n_objects;
  a.q_off = qs->q_off;
  a.q_kw = qs->q_kw;
  a.bound = qs->bound;
  a.q_sel = sel;
  a.n_sel = n_sel;
  a.k = k;
  a.k_arr = d_k;
  a.seed = seed;
  a.block_shift = p.block_shift;
  a.chunks_per_block = 1u << (p.block_shift - idx->chunk_shift);
  a.n_groups = p.n_groups;
  a.ht_slots = p.ht_slots;
  a.za_len = p.za_len;
  a.cand = cand;
  a.chunk_at = (o && !sel) ? o->d_chunk_at : nullptr;
  a.stats = o ? o->d_stats : nullptr;
  a.at_hint = at_hint;
  a.hint_hist = at_hint ? hint_hist : nullptr;
  a.hint_stride = p.za_len;
  a.no_gate = (o && (o->flags & GENIE_SEARCH_NO_GATE)) ? 1u : 0u;
  a.dense_slot = p.dense ? idx->dense_slot : nullptr;
  a.dense_bits = p.dense ? idx->dense_bits : nullptr;
  a.map_words = idx->map_words;
  const bool timed = o && !sel && o->scan_event_begin && o->scan_event_end;
  if (timed) cudaEventRecord((cudaEvent_t)o->scan_event_begin, s);
  cudaError_t e = dispatch_scan(a, p, s);
  if (e != cudaSuccess) return e;
  if (timed) cudaEventRecord((cudaEvent_t)o->scan_event_end, s);
  MergeArgs m;
  m.cand = cand;
  m.n_sel = n_sel;
  m.q_sel = sel;
  m.n_groups = p.n_groups;
  m.k = k;
  m.k_arr = d_k;
  m.bound = qs->bound;
  m.za_len = p.za_len;
  m.ids = ids;
  m.counts = counts;
  m.n_valid = n_valid;
  const size_t msmem = dev::next_pow2(k) * 8 + (size_t)p.za_len * 4;
  e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
  if (e != cudaSuccess) return e;
  merge_kernel<<<std::min<uint32_t>(n_sel, 152u * 16u), kMergeThreads, msmem, s>>>(m);
  return cudaGetLastError();
}

}  // namespace
}  // namespace genie

namespace genie {

// Search over caller-owned device query arrays (no handle, no allocation, no
// synchronisation): q_off [n+1], q_kw, bound [n] (the count bounds, at most
// max_bound), cand = scratch of search_scratch_bytes().  Used by host
// runtimes that keep their own buffers (the serving loop).
size_t search_scratch_bytes(const genie_index* idx, uint32_t max_bound, uint32_t n, uint32_t k) {
  genie_queries view;
  view.index = idx;
  view.max_bound = max_bound;
  Plan p;
  if (make_plan(idx, &view, k, nullptr, &p) != GENIE_OK) return 0;
  return (size_t)n * p.n_groups * k * 8;
}

genie_status search_raw(const genie_index* idx, const uint32_t* q_off, const uint32_t* q_kw,
                        const uint32_t* bound, uint32_t n, uint32_t max_bound, uint32_t k,
                        const uint32_t* d_k, unsigned long long* cand, size_t cand_bytes,
                        uint32_t* at_hint, uint32_t* hint_hist, size_t hint_hist_words,
                        uint32_t* ids, uint32_t* counts, uint32_t* n_valid, cudaStream_t s,
                        uint64_t n_entries, uint64_t n_keywords, uint64_t n_dense_entries) {
  genie_queries view;
  view.index = idx;
  view.n_queries = n;
  view.max_bound = max_bound;
  view.n_entries = n_entries;  // postings and keywords of the batch (0 if unknown): they pick
  view.n_keywords = n_keywords;
  view.n_dense_entries = n_dense_entries;  // the default launch shape
  view.q_off = const_cast<uint32_t*>(q_off);
  view.q_kw = const_cast<uint32_t*>(q_kw);
  view.bound = const_cast<uint32_t*>(bound);
  Plan p;
  genie_status st = make_plan(idx, &view, k, nullptr, &p);
  if (st != GENIE_OK) return st;
  if ((size_t)n * p.n_groups * k * 8 > cand_bytes)
    return fail(GENIE_ERR_CAPACITY, "search_raw: scratch too small");
  if ((size_t)n * p.za_len > hint_hist_words) hint_hist = nullptr;
  cudaError_t e = at_hint ? cudaMemsetAsync(at_hint, 0, (size_t)n * 4, s) : cudaSuccess;
  if (e == cudaSuccess && at_hint && hint_hist)
    e = cudaMemsetAsync(hint_hist, 0, (size_t)n * p.za_len * 4, s);
  if (e == cudaSuccess)
    e = run_pass(idx, &view, k, d_k, nullptr, nullptr, n, p, nullptr, cand, at_hint, hint_hist, ids,
                 counts, n_valid, s);
  if (e != cudaSuccess) return fail_cuda(e, "search_raw");
  return GENIE_OK;
}

}  // namespace genie

using namespace genie;

extern "C" genie_status genie_search_shape(const genie_index* index, const genie_queries* queries,
                                           uint32_t k, const genie_search_opts* opts,
                                           genie_search_shape_info* out) {
  if (!index || !queries || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_search_shape: NULL argument");
  if (queries->index != index)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_shape: queries were compiled for another index");
  if (k == 0 || k > GENIE_MAX_K)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_shape: k must be in 1..GENIE_MAX_K");
  Plan p;
  genie_status st = make_plan(index, queries, k, opts, &p);
  if (st != GENIE_OK) return st;
  out->counter_bits = 1u << p.log2w;
  out->block_shift = p.block_shift;
  out->n_groups = p.n_groups;
  out->threads = p.threads;
  out->unroll = p.unroll;
  out->ht_slots = p.ht_slots;
  out->smem_bytes = p.smem;
  out->dense = p.dense ? 1u : 0u;
  out->reserved = 0;
  return GENIE_OK;
}

extern "C" genie_status genie_search(const genie_index* index, const genie_queries* queries,
                                     uint32_t k, const uint32_t* d_k, const genie_search_opts* opts,
                                     uint32_t* d_ids, uint32_t* d_counts, uint32_t* d_n_valid,
                                     genie_stream stream) {
  if (!index || !queries || !d_ids || !d_counts || !d_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: NULL argument");
  if (queries->index != index)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: queries were compiled for another index");
  if (k == 0 || k > GENIE_MAX_K) return fail(GENIE_ERR_INVALID_ARG, "genie_search: k must be in 1..GENIE_MAX_K");
  cudaStream_t s = as_stream(stream);
  Plan p;
  genie_status st = make_plan(index, queries, k, opts, &p);
  if (st != GENIE_OK) return st;
  if (opts && opts->h_blocks_per_query) *opts->h_blocks_per_query = p.n_groups;
  const uint32_t Q = queries->n_queries;
  const uint64_t cand_bytes = (uint64_t)Q * p.n_groups * k * 8;
  unsigned long long* cand = nullptr;
  const bool share = !(opts && (opts->flags & GENIE_SEARCH_PER_RANGE_AT));
  // per-query count histograms of the finished ranges, when they stay small
  const uint64_t hist_words = (uint64_t)Q * p.za_len;
  const bool use_hist = share && hist_words * 4 <= kHintHistMaxBytes;
  uint32_t* aux = nullptr;  // [0] flags, [1] rerun count, [2..] rerun list, [Q] hints, histograms
  GENIE_CUDA_TRY(cudaMallocAsync((void**)&cand, cand_bytes, s));
  cudaError_t e =
      cudaMallocAsync((void**)&aux, ((uint64_t)(2 * Q + 2) + (use_hist ? hist_words : 0)) * 4, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(cand, s);
    return fail_cuda(e, "cudaMallocAsync");
  }
  auto release = [&]() {
    cudaFreeAsync(cand, s);
    cudaFreeAsync(aux, s);
  };
  if (d_k) {
    uint32_t bad = 0;
    e = cudaMemsetAsync(aux, 0, 4, s);
    if (e == cudaSuccess) {
      check_k_kernel<<<std::min<uint32_t>((Q + 255) / 256, 1024u), 256, 0, s>>>(Q, k, d_k, aux);
      e = cudaMemcpyAsync(&bad, aux, 4, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { release(); return fail_cuda(e, "genie_search: per-query k check"); }
    if (bad) { release(); return fail(GENIE_ERR_INVALID_ARG, "genie_search: a per-query k is 0 or larger than k"); }
  }
  const uint32_t* seed = opts ? opts->d_seed : nullptr;
  uint32_t* hint = share ? aux + 2 + Q : nullptr;  // [Q]: seeds from the finished ranges
  uint32_t* hist = use_hist ? aux + 2 + 2 * Q : nullptr;
  e = hint ? cudaMemsetAsync(hint, 0, (size_t)Q * 4, s) : cudaSuccess;
  if (e == cudaSuccess && hist) e = cudaMemsetAsync(hist, 0, hist_words * 4, s);
  if (e == cudaSuccess)
    e = run_pass(index, queries, k, d_k, seed, nullptr, Q, p, opts, cand, hint, hist, d_ids,
                 d_counts, d_n_valid, s);
  if (e == cudaSuccess && seed) {
    // verify-and-rerun: certified iff s = 1 or the k-th merged count >= s
    uint32_t n_rerun = 0;
    e = cudaMemsetAsync(aux + 1, 0, 4, s);
    if (e == cudaSuccess) {
      verify_seeded_kernel<<<std::min<uint32_t>((Q + 255) / 256, 1024u), 256, 0, s>>>(
          Q, k, d_k, seed, d_counts, d_n_valid, aux + 2, aux + 1);
      e = cudaMemcpyAsync(&n_rerun, aux + 1, 4, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && n_rerun > 0) {
      if (opts && opts->d_stats) add_stat_kernel<<<1, 1, 0, s>>>(opts->d_stats + 3, n_rerun);
      e = hint ? cudaMemsetAsync(hint, 0, (size_t)n_rerun * 4, s) : cudaSuccess;
      if (e == cudaSuccess && hist) e = cudaMemsetAsync(hist, 0, (size_t)n_rerun * p.za_len * 4, s);
      if (e == cudaSuccess)
        e = run_pass(index, queries, k, d_k, nullptr, aux + 2, n_rerun, p, opts, cand, hint, hist,
                     d_ids, d_counts, d_n_valid, s);
    }
  }
  release();
  if (e != cudaSuccess) return fail_cuda(e, "genie_search");
  return GENIE_OK;
}

// ---------------------------------------------------------------------------
// genie_search_host: queries in, results out, both in host memory
// ---------------------------------------------------------------------------
//
// The stages of the paper's Table 2 that one batch goes through at query time
// -- query transfer, match, select and the copy of the results back -- in one
// call: the keyword CSR is copied to the device on the caller's stream,
// compiled, searched, and the top-k lists are copied back; the call returns
// once they are in the caller's host buffers.

extern "C" genie_status genie_search_host(const genie_index* index, const uint32_t* h_q_off,
                                          const uint32_t* h_q_kw, uint32_t n_queries, uint32_t k,
                                          const uint32_t* h_k, const genie_search_opts* opts,
                                          uint32_t* h_ids, uint32_t* h_counts,
                                          uint32_t* h_n_valid, genie_stream stream) {
  if (!index || !h_q_off || !h_ids || !h_counts || !h_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_host: NULL argument");
  if (n_queries == 0 || n_queries > (1u << 24))
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_host: n_queries must be in 1..2^24");
  if (k == 0 || k > GENIE_MAX_K)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_host: k must be in 1..GENIE_MAX_K");
  if (h_q_off[0] != 0) return fail(GENIE_ERR_INVALID_ARG, "genie_search_host: h_q_off[0] must be 0");
  const uint64_t n_kw = h_q_off[n_queries];
  if (n_kw && !h_q_kw) return fail(GENIE_ERR_INVALID_ARG, "genie_search_host: h_q_kw is NULL");
  cudaStream_t s = as_stream(stream);
  // one stream-ordered block: q_off | q_kw | k | ids | counts | n_valid
  const uint64_t w_off = 0, w_kw = w_off + n_queries + 1, w_k = w_kw + n_kw;
  const uint64_t w_ids = w_k + (h_k ? n_queries : 0), w_cnt = w_ids + (uint64_t)n_queries * k;
  const uint64_t w_nv = w_cnt + (uint64_t)n_queries * k, words = w_nv + n_queries;
  uint32_t* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, words * 4, s);
  if (e != cudaSuccess) return fail(GENIE_ERR_OUT_OF_MEMORY, "genie_search_host: cudaMallocAsync failed");
  genie_queries* qs = nullptr;
  genie_status st = GENIE_OK;
  e = cudaMemcpyAsync(d + w_off, h_q_off, (n_queries + 1) * 4ull, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_kw) e = cudaMemcpyAsync(d + w_kw, h_q_kw, n_kw * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h_k) e = cudaMemcpyAsync(d + w_k, h_k, n_queries * 4ull, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = fail_cuda(e, "genie_search_host: copy of the queries");
  if (st == GENIE_OK) st = genie_make_queries(index, d + w_off, d + w_kw, n_queries, stream, &qs);
  if (st == GENIE_OK)
    st = genie_search(index, qs, k, h_k ? d + w_k : nullptr, opts, d + w_ids, d + w_cnt, d + w_nv,
                      stream);
  if (st == GENIE_OK) {
    const uint64_t res = (uint64_t)n_queries * k * 4;
    e = cudaMemcpyAsync(h_ids, d + w_ids, res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_counts, d + w_cnt, res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_n_valid, d + w_nv, n_queries * 4ull, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = fail_cuda(e, "genie_search_host: copy of the results");
  }
  genie_queries_destroy(qs);
  cudaFreeAsync(d, s);
  e = cudaStreamSynchronize(s);
  if (st == GENIE_OK && e != cudaSuccess) st = fail_cuda(e, "genie_search_host");
  return st;
}

// ---------------------------------------------------------------------------
// genie_search_noalloc: the same search with its scratch in a fixed device array
// ---------------------------------------------------------------------------
//
// For callers that must not allocate device memory while they answer
// queries: code that runs under a hard memory budget, shares the GPU with a
// framework that owns every allocation through its own pool, or cannot take
// an allocation's latency or failure on the query path.  The per-range
// candidate lists and a status word live in one file-scope device array of
// fixed size, which every GPU that loads this library holds until the
// process exits.

namespace genie {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kNoAllocStatusBytes = 256;                // after the candidate lists

// Host code may not pass this name to a kernel: on the host it stands for a
// shadow symbol, not a device address.  Its device address is looked up per
// device (scratch_address) and passed instead.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device; looked up once
// per device (the first call on a device), with that device current.
genie_status scratch_address(void** out) {
  int dev = 0;
  GENIE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e, "genie_search_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GENIE_OK;
}

}  // namespace
}  // namespace genie

extern "C" genie_status genie_search_noalloc(const genie_index* index, const genie_queries* queries,
                                             uint32_t k, const uint32_t* d_k,
                                             const genie_search_opts* opts, uint32_t* d_ids,
                                             uint32_t* d_counts, uint32_t* d_n_valid,
                                             genie_stream stream) {
  if (!index || !queries || !d_ids || !d_counts || !d_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: NULL argument");
  if (queries->index != index)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: queries were compiled for another index");
  if (k == 0 || k > GENIE_MAX_K)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: k must be in 1..GENIE_MAX_K");
  if (opts && opts->d_seed)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: seeded searches need genie_search");
  cudaStream_t s = as_stream(stream);
  Plan p;
  genie_status st = make_plan(index, queries, k, opts, &p);
  if (st != GENIE_OK) return st;
  if (opts && opts->h_blocks_per_query) *opts->h_blocks_per_query = p.n_groups;
  const uint64_t cand_bytes = (uint64_t)queries->n_queries * p.n_groups * k * 8;
  const uint64_t hint_bytes = (uint64_t)queries->n_queries * 4;
  if (cand_bytes + hint_bytes > kNoAllocScratchBytes - kNoAllocStatusBytes)
    return fail(GENIE_ERR_CAPACITY,
                "genie_search_noalloc: queries x (object ranges x k x 8 + 4) bytes = " +
                    std::to_string(cand_bytes + hint_bytes) + " exceeds the fixed scratch of " +
                    std::to_string(kNoAllocScratchBytes - kNoAllocStatusBytes) +
                    " bytes; use fewer queries per call or genie_search");
  void* base = nullptr;
  st = scratch_address(&base);
  if (st != GENIE_OK) return st;
  unsigned long long* cand = static_cast<unsigned long long*>(base);
  uint32_t* status = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) +
                                                 kNoAllocScratchBytes - kNoAllocStatusBytes);
  const uint32_t Q = queries->n_queries;
  if (d_k) {  // the status word keeps the last call's value: clear it first
    uint32_t bad = 0;
    GENIE_CUDA_TRY(cudaMemsetAsync(status, 0, 4, s));
    check_k_kernel<<<std::min<uint32_t>((Q + 255) / 256, 1024u), 256, 0, s>>>(Q, k, d_k, status);
    GENIE_CUDA_TRY(cudaMemcpyAsync(&bad, status, 4, cudaMemcpyDeviceToHost, s));
    GENIE_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(GENIE_ERR_INVALID_ARG, "genie_search_noalloc: a per-query k is 0 or larger than k");
  }
  // the scan kernel writes every candidate slot the merge reads, so the
  // candidate lists need no clearing between calls; the shared k-th counts do
  const bool share = !(opts && (opts->flags & GENIE_SEARCH_PER_RANGE_AT));
  uint32_t* hint = share ? reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + cand_bytes)
                         : nullptr;
  if (hint) GENIE_CUDA_TRY(cudaMemsetAsync(hint, 0, hint_bytes, s));
  cudaError_t e = run_pass(index, queries, k, d_k, nullptr, nullptr, Q, p, opts, cand, hint, nullptr,
                           d_ids, d_counts, d_n_valid, s);
  if (e != cudaSuccess) return fail_cuda(e, "genie_search_noalloc");
  return GENIE_OK;
}
