// Query compiler: items -> keywords (Sec. 2.1, Example 2.1), look-up of each
// keyword's postings list in the Position Map (Sec. 3.2), the count bound of
// each query (Sec. 3.3: "the maximum count for each object is bounded"), its
// scan volume, and the histogram features of the k-th-count predictor.
#include <algorithm>

#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kCompileThreads = 256;
constexpr uint32_t kSortCap = 2048;  // queries up to this length get an exact multiplicity

enum QFlag {
  kBadOffsets = 0, kBadKeyword = 1, kBadDim = 2, kBadRange = 3, kMaxBound = 4,
  kTotalLo = 6, kTotalHi = 7, kDenseLo = 8, kDenseHi = 9, kNumQFlags = 10
};

// Per query: copy of the keywords is already in place; compute B_q, the sum of
// df over its keywords and its feature histogram.  items_off != NULL selects the
// relational bound (expanded keywords, capped by max_object_len * items).
__global__ void __launch_bounds__(kCompileThreads)
compile_kernel(const uint32_t* __restrict__ q_off, const uint32_t* __restrict__ q_kw,
               uint32_t n_queries, uint64_t n_kw, const uint64_t* __restrict__ kw_off,
               uint32_t vocab, uint32_t max_obj_len, uint32_t dense_min_df,
               const uint32_t* __restrict__ items_off,
               uint32_t* __restrict__ bound, uint64_t* __restrict__ entries,
               float* __restrict__ features, uint32_t* flags) {
  __shared__ unsigned long long sorted[kSortCap];
  __shared__ uint32_t hist[kFeatures];
  __shared__ unsigned long long scratch64[33];
  __shared__ uint32_t max_run, bad_kw;
  for (uint32_t q = blockIdx.x; q < n_queries; q += gridDim.x) {
    const uint32_t a = q_off[q], b = q_off[q + 1];
    if (b < a || b > n_kw) {
      if (threadIdx.x == 0) {
        atomicOr(&flags[kBadOffsets], 1u);
        bound[q] = 0;
        entries[q] = 0;
      }
      for (uint32_t f = threadIdx.x; f < kFeatures; f += blockDim.x) features[(uint64_t)q * kFeatures + f] = 0.f;
      continue;
    }
    const uint32_t len = b - a;
    for (uint32_t f = threadIdx.x; f < kFeatures; f += blockDim.x) hist[f] = 0;
    if (threadIdx.x == 0) { max_run = len ? 1u : 0u; bad_kw = 0; }
    __syncthreads();
    unsigned long long df_sum = 0, dense_sum = 0;
    for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x) {
      uint32_t kw = q_kw[i];
      uint32_t bin = 0;
      if (kw >= vocab) {
        bad_kw = 1;
      } else {
        uint64_t df = kw_off[kw + 1] - kw_off[kw];
        df_sum += df;
        if (df >= dense_min_df) dense_sum += df;
        bin = df == 0 ? 0u : min(kFeatures - 1, 64u - (uint32_t)__clzll((long long)df));
      }
      atomicAdd(&hist[bin], 1u);
    }
    df_sum = dev::block_sum(df_sum, scratch64);
    dense_sum = dev::block_sum(dense_sum, scratch64);
    // largest multiplicity of a keyword (exact for short queries)
    uint32_t mult = len;
    if (len <= kSortCap) {
      const uint32_t n2 = dev::next_pow2(max(len, 1u));
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x)
        sorted[i] = i < len ? (unsigned long long)q_kw[a + i] : ~0ull;
      __syncthreads();
      dev::bitonic_sort_desc(sorted, n2);
      // sorted descending with the padding (~0) first; runs of equal keywords
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        unsigned long long v = sorted[i];
        if (v == ~0ull || (i > 0 && sorted[i - 1] == v)) continue;
        uint32_t j = i + 1;
        while (j < n2 && sorted[j] == v) ++j;
        atomicMax(&max_run, j - i);
      }
      __syncthreads();
      mult = max_run;
    }
    if (threadIdx.x == 0) {
      uint64_t cap = (uint64_t)max_obj_len *
                     (items_off ? (uint64_t)(items_off[q + 1] - items_off[q]) : (uint64_t)mult);
      uint32_t bq = (uint32_t)((uint64_t)len < cap ? (uint64_t)len : cap);
      bound[q] = bq;
      entries[q] = df_sum;
      atomicMax(&flags[kMaxBound], bq);
      atomicAdd((unsigned long long*)&flags[kTotalLo], df_sum);
      if (dense_sum) atomicAdd((unsigned long long*)&flags[kDenseLo], dense_sum);
      if (bad_kw) atomicOr(&flags[kBadKeyword], 1u);
    }
    __syncthreads();
    for (uint32_t f = threadIdx.x; f < kFeatures; f += blockDim.x)
      features[(uint64_t)q * kFeatures + f] = (float)hist[f] * kFeatureScale;
    __syncthreads();
  }
}

__global__ void range_count_kernel(const uint32_t* __restrict__ item_off,
                                   const uint32_t* __restrict__ dim, const int32_t* __restrict__ lo,
                                   const int32_t* __restrict__ hi, uint32_t n_queries,
                                   uint32_t n_items, uint32_t vpd, uint32_t n_dims,
                                   uint32_t* __restrict__ cnt, uint32_t* flags) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_queries; q += gridDim.x * blockDim.x) {
    uint32_t a = item_off[q], b = item_off[q + 1];
    uint64_t c = 0;
    if (b < a || b > n_items) {
      atomicOr(&flags[kBadOffsets], 1u);
    } else {
      for (uint32_t i = a; i < b; ++i) {
        if (dim[i] >= n_dims) { atomicOr(&flags[kBadDim], 1u); continue; }
        if (lo[i] > hi[i]) { atomicOr(&flags[kBadRange], 1u); continue; }
        int64_t l = max((int64_t)lo[i], (int64_t)0), h = min((int64_t)hi[i], (int64_t)vpd - 1);
        if (l <= h) c += (uint64_t)(h - l + 1);
      }
    }
    if (c > 0xFFFFFFu) { atomicOr(&flags[kBadRange], 2u); c = 0; }
    cnt[q] = (uint32_t)c;
  }
}

__global__ void range_expand_kernel(const uint32_t* __restrict__ item_off,
                                    const uint32_t* __restrict__ dim, const int32_t* __restrict__ lo,
                                    const int32_t* __restrict__ hi, uint32_t n_queries, uint32_t vpd,
                                    const uint32_t* __restrict__ q_off, uint32_t* __restrict__ q_kw) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_queries; q += gridDim.x * blockDim.x) {
    uint32_t pos = q_off[q];
    for (uint32_t i = item_off[q]; i < item_off[q + 1]; ++i) {
      int64_t l = max((int64_t)lo[i], (int64_t)0), h = min((int64_t)hi[i], (int64_t)vpd - 1);
      for (int64_t v = l; v <= h; ++v) q_kw[pos++] = dim[i] * vpd + (uint32_t)v;
    }
  }
}

void free_queries(genie_queries* q) {
  if (!q) return;
  if (q->base) cudaFreeAsync(q->base, q->stream);
  delete q;
}

// One stream-ordered allocation holds every array of the handle, plus 64 bytes
// of compile flags at the end.
genie_status alloc_queries(const genie_index* index, uint32_t n_queries, uint64_t n_kw,
                           cudaStream_t s, genie_queries** out) {
  genie_queries* q = new (std::nothrow) genie_queries();
  if (!q) return fail(GENIE_ERR_OUT_OF_MEMORY, "query handle");
  q->index = index;
  cudaGetDevice(&q->device);
  q->stream = s;
  q->n_queries = n_queries;
  q->n_keywords = n_kw;
  auto up = [](uint64_t b) { return (b + 255) & ~(uint64_t)255; };
  const uint64_t b_off = up(((uint64_t)n_queries + 1) * 4), b_kw = up(std::max<uint64_t>(n_kw, 1) * 4);
  const uint64_t b_bound = up((uint64_t)n_queries * 4), b_ent = up((uint64_t)n_queries * 8);
  const uint64_t b_feat = up((uint64_t)n_queries * kFeatures * 4);
  cudaError_t e = cudaMallocAsync(&q->base, b_off + b_kw + b_bound + b_ent + b_feat + 256, s);
  if (e != cudaSuccess) {
    delete q;
    return fail_cuda(e, "cudaMallocAsync(queries)");
  }
  char* p = static_cast<char*>(q->base);
  q->q_off = reinterpret_cast<uint32_t*>(p);
  q->q_kw = reinterpret_cast<uint32_t*>(p + b_off);
  q->bound = reinterpret_cast<uint32_t*>(p + b_off + b_kw);
  q->entries = reinterpret_cast<uint64_t*>(p + b_off + b_kw + b_bound);
  q->features = reinterpret_cast<float*>(p + b_off + b_kw + b_bound + b_ent);
  q->flags = reinterpret_cast<uint32_t*>(p + b_off + b_kw + b_bound + b_ent + b_feat);
  *out = q;
  return GENIE_OK;
}

// Runs the compile kernel, reads the flags back and finalises the handle.
genie_status finish(genie_queries* q, const uint32_t* items_off, uint32_t* flags, cudaStream_t s,
                    const char* who) {
  const genie_index* idx = q->index;
  int grid = (int)std::min<uint32_t>(q->n_queries, 152u * 16u);
  compile_kernel<<<grid, kCompileThreads, 0, s>>>(q->q_off, q->q_kw, q->n_queries, q->n_keywords,
                                                  idx->kw_off, idx->vocab, idx->max_object_len,
                                                  idx->n_dense ? idx->dense_min_df : 0xFFFFFFFFu,
                                                  items_off, q->bound, q->entries, q->features, flags);
  cudaError_t e = cudaGetLastError();
  uint32_t h[kNumQFlags];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, who);
  if (h[kBadOffsets]) return fail(GENIE_ERR_INVALID_ARG, std::string(who) + ": query offsets are not non-decreasing");
  if (h[kBadKeyword]) return fail(GENIE_ERR_INVALID_ARG, std::string(who) + ": a query keyword is >= vocab");
  if (h[kMaxBound] > GENIE_MAX_BOUND)
    return fail(GENIE_ERR_INVALID_ARG, std::string(who) + ": a query's count bound exceeds GENIE_MAX_BOUND (too many items)");
  q->max_bound = h[kMaxBound];
  q->n_entries = (uint64_t)h[kTotalLo] | ((uint64_t)h[kTotalHi] << 32);
  q->n_dense_entries = (uint64_t)h[kDenseLo] | ((uint64_t)h[kDenseHi] << 32);
  return GENIE_OK;
}

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_make_queries(const genie_index* index, const uint32_t* d_q_off,
                                           const uint32_t* d_q_kw, uint32_t n_queries,
                                           genie_stream stream, genie_queries** out) {
  if (!index || !d_q_off || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_make_queries: NULL argument");
  if (n_queries == 0 || n_queries > (1u << 24))
    return fail(GENIE_ERR_INVALID_ARG, "genie_make_queries: n_queries must be in 1..2^24");
  cudaStream_t s = as_stream(stream);
  uint32_t ends[2];
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[0], d_q_off, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[1], d_q_off + n_queries, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (ends[0] != 0) return fail(GENIE_ERR_INVALID_ARG, "genie_make_queries: d_q_off[0] != 0");
  const uint64_t n_kw = ends[1];
  if (n_kw > 0 && !d_q_kw) return fail(GENIE_ERR_INVALID_ARG, "genie_make_queries: d_q_kw is NULL");
  genie_queries* q = nullptr;
  genie_status st = alloc_queries(index, n_queries, n_kw, s, &q);
  if (st != GENIE_OK) return st;
  cudaError_t e = cudaMemsetAsync(q->flags, 0, 64, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q->q_off, d_q_off, ((uint64_t)n_queries + 1) * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && n_kw) e = cudaMemcpyAsync(q->q_kw, d_q_kw, n_kw * 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    free_queries(q);
    return fail_cuda(e, "genie_make_queries");
  }
  st = finish(q, nullptr, q->flags, s, "genie_make_queries");
  if (st != GENIE_OK) {
    free_queries(q);
    return st;
  }
  *out = q;
  return GENIE_OK;
}

extern "C" genie_status genie_compile_ranges(const genie_index* index, uint32_t values_per_dim,
                                             const uint32_t* d_item_off, const uint32_t* d_dim,
                                             const int32_t* d_lo, const int32_t* d_hi,
                                             uint32_t n_queries, genie_stream stream,
                                             genie_queries** out) {
  if (!index || !d_item_off || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_compile_ranges: NULL argument");
  if (n_queries == 0 || n_queries > (1u << 24))
    return fail(GENIE_ERR_INVALID_ARG, "genie_compile_ranges: n_queries must be in 1..2^24");
  if (values_per_dim == 0 || values_per_dim > index->vocab)
    return fail(GENIE_ERR_INVALID_ARG, "genie_compile_ranges: values_per_dim must be in 1..vocab");
  cudaStream_t s = as_stream(stream);
  uint32_t ends[2];
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[0], d_item_off, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[1], d_item_off + n_queries, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (ends[0] != 0) return fail(GENIE_ERR_INVALID_ARG, "genie_compile_ranges: d_item_off[0] != 0");
  const uint32_t n_items = ends[1];
  if (n_items > 0 && (!d_dim || !d_lo || !d_hi))
    return fail(GENIE_ERR_INVALID_ARG, "genie_compile_ranges: item arrays are NULL");
  const uint32_t n_dims = index->vocab / values_per_dim;

  uint32_t* buf = nullptr;  // flags[16] then counts/offsets[n_queries + 1]
  GENIE_CUDA_TRY(cudaMallocAsync((void**)&buf, 64 + ((uint64_t)n_queries + 1) * 4, s));
  uint32_t* flags = buf;
  uint32_t* cnt = buf + 16;
  cudaError_t e = cudaMemsetAsync(flags, 0, 64, s);
  int grid = (int)std::max<uint32_t>(1, std::min<uint32_t>((n_queries + 255) / 256, 152u * 8u));
  if (e == cudaSuccess) {
    range_count_kernel<<<grid, 256, 0, s>>>(d_item_off, d_dim, d_lo, d_hi, n_queries, n_items,
                                            values_per_dim, n_dims, cnt, flags);
    launch_exclusive_scan(cnt, n_queries, cnt + n_queries, s);
    e = cudaGetLastError();
  }
  uint32_t h[kNumQFlags], total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cnt + n_queries, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    return fail_cuda(e, "genie_compile_ranges");
  }
  const char* bad = h[kBadOffsets] ? "item offsets are not non-decreasing"
                    : h[kBadDim]   ? "an item's dimension is >= vocab / values_per_dim"
                    : (h[kBadRange] & 1u) ? "an item has lo > hi"
                    : (h[kBadRange] & 2u) ? "a query expands to too many keywords" : nullptr;
  if (bad) {
    cudaFreeAsync(buf, s);
    return fail(GENIE_ERR_INVALID_ARG, std::string("genie_compile_ranges: ") + bad);
  }
  genie_queries* q = nullptr;
  genie_status st = alloc_queries(index, n_queries, total, s, &q);
  if (st != GENIE_OK) {
    cudaFreeAsync(buf, s);
    return st;
  }
  e = cudaMemcpyAsync(q->q_off, cnt, ((uint64_t)n_queries + 1) * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->flags, 0, 64, s);
  if (e == cudaSuccess) {
    range_expand_kernel<<<grid, 256, 0, s>>>(d_item_off, d_dim, d_lo, d_hi, n_queries,
                                             values_per_dim, q->q_off, q->q_kw);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(buf, s);
    free_queries(q);
    return fail_cuda(e, "genie_compile_ranges");
  }
  st = finish(q, d_item_off, q->flags, s, "genie_compile_ranges");
  cudaFreeAsync(buf, s);
  if (st != GENIE_OK) {
    free_queries(q);
    return st;
  }
  *out = q;
  return GENIE_OK;
}

extern "C" void genie_queries_destroy(genie_queries* queries) {
  if (!queries) return;
  free_queries(queries);  // stream-ordered on the stream the queries were compiled on
}

extern "C" genie_status genie_queries_get_info(const genie_queries* queries, genie_queries_info* out) {
  if (!queries || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_queries_get_info: NULL argument");
  out->n_queries = queries->n_queries;
  out->max_bound = queries->max_bound;
  out->n_keywords = queries->n_keywords;
  out->n_entries = queries->n_entries;
  out->n_dense_entries = queries->n_dense_entries;
  return GENIE_OK;
}

extern "C" genie_status genie_queries_export(const genie_queries* queries, uint32_t* d_bound,
                                             uint64_t* d_entries, float* d_features,
                                             genie_stream stream) {
  if (!queries) return fail(GENIE_ERR_INVALID_ARG, "genie_queries_export: queries is NULL");
  cudaStream_t s = as_stream(stream);
  const uint64_t n = queries->n_queries;
  if (d_bound) GENIE_CUDA_TRY(cudaMemcpyAsync(d_bound, queries->bound, n * 4, cudaMemcpyDeviceToDevice, s));
  if (d_entries) GENIE_CUDA_TRY(cudaMemcpyAsync(d_entries, queries->entries, n * 8, cudaMemcpyDeviceToDevice, s));
  if (d_features)
    GENIE_CUDA_TRY(cudaMemcpyAsync(d_features, queries->features, n * kFeatures * 4, cudaMemcpyDeviceToDevice, s));
  return GENIE_OK;
}
