// GEN-SPQ: the paper's ablation of c-PQ (Sec. 6.1.2, Appendix A, Table 5).
//
// The same inverted index and query compiler, but counting goes to a dense
// Count Table in global memory (one 32-bit count per object per query, the
// Count Table of Sec. 3.3) and the top-k comes from a bucket k-selection over
// each query's row (Appendix A), instead of the Bitmap Counter, Gate and hash
// table of c-PQ.  It exists to measure what c-PQ saves on this GPU, in time
// and in memory per query; results equal genie_search's.
//
// Counting: one block per query keyword scans the keyword's postings and
// adds 1 to the query's count of each object with a global atomic (the
// one-block-per-query-item design of Sec. 3.2).
//
// Selection: one block per query.  The candidates start as the objects of
// the row with a count of at least 1.  Each iteration (Appendix A) takes the
// smallest and largest candidate count, assigns every candidate the bucket
// floor((count - min) / (max - min) * NB), keeps the candidates of the
// buckets above the one that holds the k-th largest as results, and repeats
// on that bucket's candidates with k reduced by the number kept.  It stops
// when the bucket holds no more candidates than are still needed, or when all
// its candidates have one count (then the smallest ids are taken, the tie rule
// of the rest of the library).  Candidates are stored explicitly, as the
// paper notes the method must: (count, id) keys, compacted in order in a
// per-query list so that ids stay ascending.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kSpqThreads = 1024;
constexpr uint32_t kSpqCountThreads = 256;

// owner[i - kw0] = query of keyword position i (relative to query q0)
__global__ void spq_owner_kernel(const uint32_t* __restrict__ q_off, uint32_t q0, uint32_t n,
                                 uint32_t kw0, uint32_t* __restrict__ owner) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    for (uint32_t i = q_off[q0 + q]; i < q_off[q0 + q + 1]; ++i) owner[i - kw0] = q;
}

// Count Table rows ct[q][0..N) of the sub-batch += 1 per posting of every
// query keyword; one block per keyword position.
__global__ void __launch_bounds__(kSpqCountThreads) spq_count_kernel(
    const uint64_t* __restrict__ kw_off, const uint32_t* __restrict__ post_ids,
    const uint32_t* __restrict__ q_kw, uint32_t kw0, const uint32_t* __restrict__ owner,
    uint32_t* __restrict__ ct, uint32_t n_objects) {
  const uint32_t kw = q_kw[kw0 + blockIdx.x];
  uint32_t* row = ct + (uint64_t)owner[blockIdx.x] * n_objects;
  const uint64_t hi = kw_off[kw + 1];
  for (uint64_t p = kw_off[kw] + threadIdx.x; p < hi; p += blockDim.x) atomicAdd(&row[post_ids[p]], 1u);
}

struct SelShared {
  uint32_t hist[32];
  uint32_t scratch[33];
  uint32_t lo, hi, sel, need, n_out, m;
};

// Ordered compaction of one round: a thread's `m` flagged keys go after those
// of the threads before it; returns its offset, the round's total in *total.
__device__ uint32_t block_offset(uint32_t m, uint32_t* scratch, uint32_t* total) {
  return dev::block_exclusive_scan(m, scratch, total);
}

// Bucket k-selection of one query's Count Table row (Appendix A).  nb: buckets
// per iteration (2..32).  list: [n_objects] keys of scratch.  out_keys: the
// query's results in shared memory (kq of them at most).
__global__ void __launch_bounds__(kSpqThreads) spq_select_kernel(
    const uint32_t* __restrict__ ct, uint32_t n_objects, uint32_t q0, uint32_t k,
    const uint32_t* __restrict__ k_arr, uint32_t nb, unsigned long long* __restrict__ lists,
    uint32_t* __restrict__ ids, uint32_t* __restrict__ counts, uint32_t* __restrict__ n_valid,
    unsigned long long* __restrict__ iters_out) {
  extern __shared__ unsigned long long keys[];  // [next_pow2(k)]
  __shared__ SelShared S;
  const uint32_t qloc = blockIdx.x, q = q0 + qloc, tid = threadIdx.x;
  const uint32_t kq = k_arr ? k_arr[q] : k;
  const uint32_t* row = ct + (uint64_t)qloc * n_objects;
  unsigned long long* list = lists + (uint64_t)qloc * n_objects;
  if (tid == 0) {
    S.n_out = 0;
    S.need = kq;
  }
  __syncthreads();
  // Iteration over candidates: the first reads the dense row (objects with a
  // count of at least 1), later ones the compacted list of the kept bucket.
  uint32_t m = 0;  // candidates in the list (after the first iteration)
  uint32_t iters = 0;
  for (bool first = true;; first = false) {
    ++iters;
    const uint32_t n_in = first ? n_objects : m;
    // (1) smallest and largest candidate count, and how many candidates
    uint32_t lo = 0xFFFFFFFFu, hi = 0, cnt = 0;
    for (uint32_t i = tid; i < n_in; i += blockDim.x) {
      const uint32_t c = first ? row[i] : dev::key_count(list[i]);
      if (c) {
        lo = min(lo, c);
        hi = max(hi, c);
        ++cnt;
      }
    }
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (tid == 0) {
      S.lo = 0xFFFFFFFFu;
      S.hi = 0;
      S.m = 0;
    }
    __syncthreads();
    if (dev::lane_id() == 0) {
      atomicMin(&S.lo, lo);
      atomicMax(&S.hi, hi);
      atomicAdd(&S.m, cnt);
    }
    for (uint32_t b = tid; b < 32; b += blockDim.x) S.hist[b] = 0;
    __syncthreads();
    lo = S.lo;
    hi = S.hi;
    const uint32_t n_cand = S.m, need = S.need;
    // (2) bucket of every candidate; the bucket that holds the need-th largest
    // (all candidates are taken when they are no more than needed; when all
    // have one count, the first `need` in id order are)
    uint32_t sel;  // candidates in buckets above sel are kept; sel's are iterated on
    bool take_all = n_cand <= need, ties = !take_all && lo == hi;
    if (take_all || ties) {
      sel = 0xFFFFFFFFu;
    } else {
      const uint64_t span = hi - lo;
      for (uint32_t i = tid; i < n_in; i += blockDim.x) {
        const uint32_t c = first ? row[i] : dev::key_count(list[i]);
        if (c) atomicAdd(&S.hist[umin(nb - 1, (uint32_t)((uint64_t)(c - lo) * nb / span))], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t acc = 0, b = nb - 1;
        for (;; --b) {
          if (acc + S.hist[b] >= need) break;
          acc += S.hist[b];
        }
        S.sel = b;
      }
      __syncthreads();
      sel = S.sel;
    }
    // (3) keep the candidates above the selected bucket (or all, or the first
    // `need` ties) as results; compact the selected bucket's candidates in id
    // order into the list
    const uint64_t span = hi > lo ? hi - lo : 1;
    uint32_t written = 0, kept_total = 0;
    for (uint32_t r0 = 0; r0 < n_in; r0 += 4 * blockDim.x) {
      unsigned long long kk[4];
      uint32_t fk = 0, fl = 0;  // bit e: entry e is kept / goes to the list
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        const uint32_t i = r0 + 4 * tid + e;
        kk[e] = 0;
        if (i < n_in) {
          if (first) {
            const uint32_t c = row[i];
            if (c) kk[e] = dev::result_key(c, i);
          } else {
            kk[e] = list[i];
          }
        }
        if (kk[e]) {
          const uint32_t c = dev::key_count(kk[e]);
          if (take_all || ties) {
            fk |= 1u << e;
          } else {
            const uint32_t b = umin(nb - 1, (uint32_t)((uint64_t)(c - lo) * nb / span));
            if (b > sel) fk |= 1u << e;
            else if (b == sel) fl |= 1u << e;
          }
        }
      }
      uint32_t tk, tl;
      const uint32_t pk = block_offset(__popc(fk), S.scratch, &tk);
      const uint32_t pl = block_offset(__popc(fl), S.scratch, &tl);
      uint32_t ok = kept_total + pk, ol = written + pl;
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
        if (fk >> e & 1) {
          // ties: only the first `need` (ascending id) are results
          if (!ties || ok < need) keys[S.n_out + ok] = kk[e];
          ++ok;
        }
        if (fl >> e & 1) list[ol++] = kk[e];
      }
      kept_total += tk;
      written += tl;
      __syncthreads();  // every thread has read its entries of this round before the next writes
      if (ties && kept_total >= need) break;
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t kept = ties ? min(kept_total, need) : kept_total;
      S.n_out += kept;
      S.need = need - min(need, kept);
    }
    __syncthreads();
    m = written;
    if (take_all || ties || S.need == 0) break;
  }
  // sort the results by (count desc, id asc) and write the row
  const uint32_t n_out = S.n_out;
  const uint32_t n2 = dev::next_pow2(max(n_out, 1u));
  for (uint32_t i = n_out + tid; i < n2; i += blockDim.x) keys[i] = 0ull;
  __syncthreads();
  dev::bitonic_sort_desc(keys, n2);
  uint32_t* ids_row = ids + (uint64_t)q * k;
  uint32_t* cnt_row = counts + (uint64_t)q * k;
  for (uint32_t i = tid; i < k; i += blockDim.x) {
    const bool v = i < n_out;
    ids_row[i] = v ? dev::key_id(keys[i]) : 0xFFFFFFFFu;
    cnt_row[i] = v ? dev::key_count(keys[i]) : 0u;
  }
  if (tid == 0) {
    n_valid[q] = n_out;
    if (iters_out) atomicAdd(iters_out, (unsigned long long)iters);
  }
}

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_search_spq(const genie_index* index, const genie_queries* queries,
                                         uint32_t k, const uint32_t* d_k,
                                         const genie_spq_opts* opts, uint32_t* d_ids,
                                         uint32_t* d_counts, uint32_t* d_n_valid,
                                         genie_spq_info* info, genie_stream stream) {
  if (!index || !queries || !d_ids || !d_counts || !d_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_spq: NULL argument");
  if (queries->index != index)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search_spq: queries were compiled for another index");
  if (k == 0 || k > GENIE_MAX_K) return fail(GENIE_ERR_INVALID_ARG, "genie_search_spq: k must be in 1..GENIE_MAX_K");
  const uint32_t nb = (opts && opts->buckets) ? opts->buckets : 16;
  if (nb < 2 || nb > 32) return fail(GENIE_ERR_INVALID_ARG, "genie_search_spq: buckets must be in 2..32");
  const uint64_t cap = (opts && opts->max_bytes) ? opts->max_bytes : ((uint64_t)8 << 30);
  cudaStream_t s = as_stream(stream);
  const uint32_t N = index->n_objects, Q = queries->n_queries;
  // per query: its Count Table row (4 B per object) and its candidate list
  // (8 B per object: (count, id) keys)
  const uint64_t per_query = 12ull * N;
  const uint64_t qs_pass = std::min<uint64_t>(Q, cap / per_query);
  if (qs_pass == 0)
    return fail(GENIE_ERR_CAPACITY, "genie_search_spq: one query's Count Table and list exceed max_bytes");
  // keyword positions of the largest pass (host copy of the query offsets)
  std::vector<uint32_t> h_off(Q + 1);
  GENIE_CUDA_TRY(cudaMemcpyAsync(h_off.data(), queries->q_off, (Q + 1) * 4ull, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t max_kw = 0;
  for (uint32_t q0 = 0; q0 < Q; q0 += (uint32_t)qs_pass) {
    const uint32_t q1 = (uint32_t)std::min<uint64_t>(Q, q0 + qs_pass);
    max_kw = std::max(max_kw, h_off[q1] - h_off[q0]);
  }
  uint32_t* ct = nullptr;
  unsigned long long* lists = nullptr;
  uint32_t* owner = nullptr;
  unsigned long long* iters = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&ct, qs_pass * N * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&lists, qs_pass * N * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&owner, std::max<uint64_t>(max_kw, 1) * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&iters, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(iters, 0, 8, s);
  const size_t smem = (size_t)dev::next_pow2(k) * 8;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spq_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  uint32_t passes = 0;
  for (uint32_t q0 = 0; q0 < Q && e == cudaSuccess; q0 += (uint32_t)qs_pass) {
    const uint32_t q1 = (uint32_t)std::min<uint64_t>(Q, q0 + qs_pass), n = q1 - q0;
    const uint32_t kw0 = h_off[q0], nkw = h_off[q1] - kw0;
    ++passes;
    e = cudaMemsetAsync(ct, 0, (uint64_t)n * N * 4, s);
    if (e != cudaSuccess) break;
    if (nkw) {
      spq_owner_kernel<<<std::min<uint32_t>((n + 255) / 256, 1024u), 256, 0, s>>>(queries->q_off, q0, n, kw0, owner);
      spq_count_kernel<<<nkw, kSpqCountThreads, 0, s>>>(
          index->kw_off, index->post_ids, queries->q_kw, kw0, owner, ct, N);
    }
    spq_select_kernel<<<n, kSpqThreads, smem, s>>>(ct, N, q0, k, d_k, nb, lists, d_ids, d_counts,
                                                   d_n_valid, info ? iters : nullptr);
    e = cudaGetLastError();
  }
  unsigned long long h_iters = 0;
  if (e == cudaSuccess && info) e = cudaMemcpyAsync(&h_iters, iters, 8, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(ct, s);
  cudaFreeAsync(lists, s);
  cudaFreeAsync(owner, s);
  cudaFreeAsync(iters, s);
  if (e == cudaSuccess && info) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "genie_search_spq");
  if (info) {
    info->count_table_bytes_per_query = 4ull * N;
    info->list_bytes_per_query = 8ull * N;
    info->queries_per_pass = (uint32_t)qs_pass;
    info->passes = passes;
    info->mean_iterations = Q ? (double)h_iters / Q : 0.0;
  }
  return GENIE_OK;
}
