// Host-side definitions shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/genie.h"

namespace genie {

// Records `msg` as the calling thread's last error and returns `status`.
genie_status fail(genie_status status, const std::string& msg);
genie_status fail_cuda(cudaError_t err, const char* what);

// Exclusive prefix sum of v[0..n) in place on the device, total into *total.
void launch_exclusive_scan(uint32_t* v, uint32_t n, uint32_t* total, cudaStream_t s);

inline cudaStream_t as_stream(genie_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Search over caller-owned device query arrays (search.cu).  at_hint: [n]
// words; hint_hist: hint_hist_words words, used when they hold n x
// (max_bound + 2) (per-query count histograms of the finished ranges).
size_t search_scratch_bytes(const genie_index* idx, uint32_t max_bound, uint32_t n, uint32_t k);
genie_status search_raw(const genie_index* idx, const uint32_t* q_off, const uint32_t* q_kw,
                        const uint32_t* bound, uint32_t n, uint32_t max_bound, uint32_t k,
                        const uint32_t* d_k, unsigned long long* cand, size_t cand_bytes,
                        uint32_t* at_hint, uint32_t* hint_hist, size_t hint_hist_words,
                        uint32_t* ids, uint32_t* counts, uint32_t* n_valid, cudaStream_t s,
                        uint64_t n_entries = 0, uint64_t n_keywords = 0,
                        uint64_t n_dense_entries = 0);

// Largest per-query count histograms (bytes) a search allocates to seed the
// AuditThreshold of later object ranges; beyond it the seed is the largest
// k-th count of the finished ranges alone.
constexpr uint64_t kHintHistMaxBytes = (uint64_t)256 << 20;

}  // namespace genie

#define GENIE_CUDA_TRY(expr)                                           \
  do {                                                                 \
    cudaError_t genie_err_ = (expr);                                   \
    if (genie_err_ != cudaSuccess) return genie::fail_cuda(genie_err_, #expr); \
  } while (0)

// The inverted index (Sec. 3.2): List Array, Position Map and the sublist map
// of Sec. 3.2.1, all resident in device memory.
struct genie_index {
  int device = 0;
  uint32_t n_objects = 0;
  uint32_t vocab = 0;
  uint64_t nnz = 0;
  uint32_t max_object_len = 0;
  uint32_t chunk_shift = 15;
  uint32_t n_chunks = 0;
  uint64_t* kw_off = nullptr;    // [vocab + 1]: list of keyword v = post_ids[kw_off[v] .. kw_off[v+1])
  uint32_t* post_ids = nullptr;  // [nnz rounded up to 4, + 4]: ascending ids per list, zero padded
  uint32_t* chunk_pos = nullptr; // [vocab * (n_chunks + 1)]: first position of ids >= c << chunk_shift, relative to kw_off[v]
  // Keywords with a dense list also as object bitmaps: dense_slot[v] = the
  // bitmap of keyword v (kNoDense if it has none); bitmap s is
  // dense_bits[s * map_words ..], bit o set iff object o holds the keyword.
  uint32_t n_dense = 0;
  uint32_t dense_min_df = 0;     // lists of at least this many postings have a bitmap
  uint64_t map_words = 0;        // 32-bit words per bitmap (padded)
  uint64_t dense_postings = 0;   // postings of the keywords with a bitmap
  uint32_t* dense_slot = nullptr;  // [vocab] or NULL when n_dense = 0
  uint32_t* dense_bits = nullptr;  // [n_dense * map_words]
  uint64_t device_bytes = 0;
};

namespace genie {
constexpr uint32_t kNoDense = 0xFFFFFFFFu;
}  // namespace genie

// Compiled queries: every query is a list of keywords (relational items
// already expanded), with its count bound, scan volume and features.
struct genie_queries {
  const genie_index* index = nullptr;
  int device = 0;
  uint32_t n_queries = 0;
  uint32_t max_bound = 0;
  uint64_t n_keywords = 0;
  uint64_t n_entries = 0;
  uint64_t n_dense_entries = 0;  // of them, postings of keywords with an object bitmap
  uint32_t* q_off = nullptr;     // [n_queries + 1]
  uint32_t* q_kw = nullptr;      // [n_keywords]
  uint32_t* bound = nullptr;     // [n_queries]
  uint64_t* entries = nullptr;   // [n_queries]
  float* features = nullptr;     // [n_queries * 64]
  uint32_t* flags = nullptr;     // compile flags (64 bytes)
  void* base = nullptr;          // the one stream-ordered allocation holding all of the above
  cudaStream_t stream = nullptr; // the stream it was allocated (and is freed) on
};

namespace genie {
constexpr uint32_t kFeatures = 64;
constexpr float kFeatureScale = 1.0f / 32.0f;
}  // namespace genie
