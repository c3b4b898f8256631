// Multiple loadings (Sec. 3.4): an index split into parts by object id, held
// in pinned host memory, and searched one part at a time.
//
// The paper loads the parts of an index that does not fit in device memory
// one after the other, runs the whole query batch on each, and merges the
// per-part top-k lists on the CPU (Tables 3-4).  Here every part is a normal
// index whose arrays were copied to pinned host memory.  A search keeps two
// device slots: while the queries run against part p in one slot, a second
// stream copies part p + 1 into the other.  Each part's search is the usual
// one (compile, scan + c-PQ, per-range merge) and writes that part's top-k;
// the per-part lists then become result keys with global object ids and go
// through the same device merge as the object ranges of one index.  The merge
// is exact under (count desc, id asc): the batch's top-k is a subset of the
// union of the parts' top-k lists, and parts come in ascending id order, so
// ties at the k-th count are taken in ascending id.
//
// The List Array is most of a part's bytes, and with 32-bit ids its copy from
// host memory bounds a batch.  An id in range c is (c << chunk_shift) | place,
// and the sublist map already says where range c starts in each list, so with
// chunk_shift <= 16 a part keeps only the 16-bit places in host memory; the
// device rebuilds the ids from them before the part's search.
#include <algorithm>
#include <vector>

#include "cpq_device.cuh"
#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

struct HostPart {
  uint32_t base = 0;  // global id of the part's object 0
  uint32_t n_objects = 0, max_object_len = 0, chunk_shift = 0, n_chunks = 0;
  uint64_t nnz = 0, post_len = 0, chunk_len = 0;
  uint64_t* kw_off = nullptr;    // pinned host copies of the index arrays
  uint32_t* post_ids = nullptr;  // NULL when the part keeps 16-bit places
  uint16_t* post16 = nullptr;    // the ids' places in their ranges (chunk_shift <= 16)
  uint32_t* chunk_pos = nullptr;
  uint64_t post_bytes() const { return post_len * (post16 ? 2 : 4); }
};

// ids -> their places in their object ranges (the low chunk_shift bits)
__global__ void narrow_ids_kernel(const uint32_t* __restrict__ ids, uint64_t n, uint32_t mask,
                                  uint16_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint16_t)(ids[i] & mask);
}

// places -> ids.  The List Array is cut into segments of kWidenSeg
// positions, one block each: list lengths range from one posting to a large
// share of the part, so the work follows positions, not keywords.
constexpr uint32_t kWidenThreads = 256, kWidenPer = 8, kWidenSeg = kWidenThreads * kWidenPer;

// seg_kw[s] = the keyword whose list holds position min(s * kWidenSeg, nnz - 1),
// for s = 0 .. n_seg: the largest keyword whose list starts at or before it.
__global__ void segment_keywords_kernel(const uint64_t* __restrict__ kw_off, uint32_t vocab,
                                        uint64_t nnz, uint32_t n_seg, uint32_t* __restrict__ seg_kw) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= n_seg; s += gridDim.x * blockDim.x) {
    const uint64_t pos = min((uint64_t)s * kWidenSeg, nnz - 1);
    uint32_t kw = 0;  // kw_off[kw] <= pos, the answer in [kw, kw + n)
    for (uint32_t n = vocab; n > 1;) {
      const uint32_t half = n >> 1;
      if (kw_off[kw + half] <= pos) kw += half;
      n -= half;
    }
    seg_kw[s] = kw;
  }
}

// Each thread takes kWidenPer positions of its block's segment.  The block
// lists the start of every sublist of the segment's keywords (lo .. hi, each
// with nch ranges), as an offset from the segment's first position clamped to
// [0, kWidenSeg], in shared memory: the starts do not decrease in (keyword,
// range) order, and a position's sublist is the last one that starts at or
// before it.  One coalesced read fills the table and each position searches it
// on chip.  A segment with more than kWidenFlat sublists (many short lists)
// searches the keyword and then the range in global memory instead: binary
// searches with a fixed number of steps, the positions' searches interleaved
// so that their loads overlap.
constexpr uint32_t kWidenFlat = 4096;

__global__ void __launch_bounds__(kWidenThreads)
    widen_ids_kernel(const uint64_t* __restrict__ kw_off, const uint32_t* __restrict__ chunk_pos,
                     uint32_t nch, uint32_t shift, uint64_t nnz, const uint32_t* __restrict__ seg_kw,
                     const uint16_t* __restrict__ in, uint32_t* __restrict__ ids) {
  __shared__ uint32_t start[kWidenFlat];
  const uint64_t seg0 = (uint64_t)blockIdx.x * kWidenSeg;
  const uint64_t s0 = seg0 + threadIdx.x;
  const uint32_t lo = seg_kw[blockIdx.x], hi = seg_kw[blockIdx.x + 1];
  uint64_t pc[kWidenPer];  // the position, clamped into the List Array
  uint32_t place[kWidenPer], kw[kWidenPer], c[kWidenPer];
#pragma unroll
  for (uint32_t j = 0; j < kWidenPer; ++j) {
    pc[j] = min(s0 + j * kWidenThreads, nnz - 1);
    place[j] = in[pc[j]];
    kw[j] = lo;
    c[j] = 0;
  }
  const uint64_t n_flat = (uint64_t)(hi - lo + 1) * nch;  // the same for the whole block
  if (n_flat <= kWidenFlat) {
    for (uint32_t t = threadIdx.x; t < n_flat; t += kWidenThreads) {
      const uint32_t v = lo + t / nch, r = t % nch;
      const uint64_t a = kw_off[v] + chunk_pos[(uint64_t)v * (nch + 1) + r];
      start[t] = (uint32_t)(a <= seg0 ? 0 : min(a - seg0, (uint64_t)kWidenSeg));
    }
    __syncthreads();
    uint32_t f[kWidenPer], rel[kWidenPer];
#pragma unroll
    for (uint32_t j = 0; j < kWidenPer; ++j) {
      f[j] = 0;  // start[f[j]] <= rel[j]; the answer in [f[j], f[j] + n)
      rel[j] = (uint32_t)(pc[j] - seg0);
    }
    for (uint32_t n = (uint32_t)n_flat; n > 1;) {
      const uint32_t half = n >> 1;
#pragma unroll
      for (uint32_t j = 0; j < kWidenPer; ++j) f[j] += start[f[j] + half] <= rel[j] ? half : 0u;
      n -= half;
    }
#pragma unroll
    for (uint32_t j = 0; j < kWidenPer; ++j)
      if (s0 + j * kWidenThreads < nnz) ids[s0 + j * kWidenThreads] = ((f[j] % nch) << shift) | place[j];
    return;
  }
  for (uint32_t n = hi - lo + 1; n > 1;) {  // kw_off[kw[j]] <= pc[j]; the answer in [kw[j], kw[j] + n)
    const uint32_t half = n >> 1;
#pragma unroll
    for (uint32_t j = 0; j < kWidenPer; ++j) kw[j] += kw_off[kw[j] + half] <= pc[j] ? half : 0u;
    n -= half;
  }
#pragma unroll
  for (uint32_t j = 0; j < kWidenPer; ++j) pc[j] -= kw_off[kw[j]];  // the position in its list
  for (uint32_t n = nch; n > 1;) {  // row[c[j]] <= pc[j]; the answer in [c[j], c[j] + n)
    const uint32_t half = n >> 1;
#pragma unroll
    for (uint32_t j = 0; j < kWidenPer; ++j)
      c[j] += chunk_pos[(uint64_t)kw[j] * (nch + 1) + c[j] + half] <= pc[j] ? half : 0u;
    n -= half;
  }
#pragma unroll
  for (uint32_t j = 0; j < kWidenPer; ++j)
    if (s0 + j * kWidenThreads < nnz) ids[s0 + j * kWidenThreads] = (c[j] << shift) | place[j];
}

// part outputs [P][Q][k] -> result keys [Q][P][k] with global ids (0 past n_valid)
__global__ void part_keys_kernel(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ counts,
                                 const uint32_t* __restrict__ n_valid,
                                 const uint32_t* __restrict__ bases, uint32_t P, uint32_t Q,
                                 uint32_t k, unsigned long long* __restrict__ keys) {
  const uint64_t total = (uint64_t)P * Q * k;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)(i % k);
    const uint64_t pq = i / k;  // p * Q + q
    const uint32_t p = (uint32_t)(pq / Q), q = (uint32_t)(pq % Q);
    unsigned long long key = 0;
    if (j < n_valid[pq]) key = dev::result_key(counts[i], bases[p] + ids[i]);
    keys[((uint64_t)q * P + p) * k + j] = key;
  }
}

__global__ void max_bound_kernel(const uint32_t* __restrict__ b, uint32_t n,
                                 uint32_t* __restrict__ acc) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc[i] = max(acc[i], b[i]);
}

uint32_t grid_for(uint64_t n, uint32_t threads) {
  return (uint32_t)std::min<uint64_t>((n + threads - 1) / threads, 152ull * 32);
}

}  // namespace
}  // namespace genie

using namespace genie;

struct genie_parts {
  int device = 0;
  uint32_t vocab = 0;
  std::vector<HostPart> parts;
  // two device slots, each a complete index view sized for the largest part
  genie_index slot[2];
  uint16_t* stage16[2] = {nullptr, nullptr};  // a part's 16-bit places on their way in
  uint32_t* seg_kw = nullptr;                 // the first keyword of each segment (widening)
  int64_t slot_part[2] = {-1, -1};            // the part a slot holds (-1: none)
  bool slot_wide[2] = {false, false};         // its ids are rebuilt from the 16-bit places
  uint64_t slot_post_cap = 0, slot_chunk_cap = 0;
  cudaStream_t copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
};

namespace {

void free_slots(genie_parts* ps) {
  for (genie_index& s : ps->slot) {
    cudaFree(s.kw_off);
    cudaFree(s.post_ids);
    cudaFree(s.chunk_pos);
    s.kw_off = nullptr;
    s.post_ids = nullptr;
    s.chunk_pos = nullptr;
  }
  for (uint16_t*& b : ps->stage16) {
    cudaFree(b);
    b = nullptr;
  }
  cudaFree(ps->seg_kw);
  ps->seg_kw = nullptr;
  ps->slot_part[0] = ps->slot_part[1] = -1;
  ps->slot_post_cap = ps->slot_chunk_cap = 0;
}

// device slots large enough for every part
cudaError_t ensure_slots(genie_parts* ps) {
  uint64_t post = 0, chunk = 0;
  bool narrow = false;
  for (const HostPart& h : ps->parts) {
    post = std::max(post, h.post_len);
    chunk = std::max(chunk, h.chunk_len);
    narrow |= h.post16 != nullptr;
  }
  if (post <= ps->slot_post_cap && chunk <= ps->slot_chunk_cap && ps->slot[0].kw_off &&
      (!narrow || ps->stage16[0]))
    return cudaSuccess;
  free_slots(ps);
  cudaError_t e = cudaSuccess;
  for (genie_index& s : ps->slot) {
    if (e == cudaSuccess) e = cudaMalloc(&s.kw_off, ((uint64_t)ps->vocab + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s.post_ids, post * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.chunk_pos, chunk * 4);
    s.device = ps->device;
    s.vocab = ps->vocab;
  }
  for (uint16_t*& b : ps->stage16)
    if (e == cudaSuccess && narrow) e = cudaMalloc(&b, post * 2);
  if (e == cudaSuccess && narrow) e = cudaMalloc(&ps->seg_kw, (post / kWidenSeg + 2) * 4);
  if (e != cudaSuccess) {
    free_slots(ps);
    return e;
  }
  ps->slot_post_cap = post;
  ps->slot_chunk_cap = chunk;
  return cudaSuccess;
}

}  // namespace

extern "C" genie_status genie_parts_create(genie_parts** out) {
  if (!out) return fail(GENIE_ERR_INVALID_ARG, "genie_parts_create: out is NULL");
  genie_parts* ps = new genie_parts();
  cudaError_t e = cudaGetDevice(&ps->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps->copy, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&ps->copied[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ps->used[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    genie_parts_destroy(ps);
    return fail_cuda(e, "genie_parts_create");
  }
  *out = ps;
  return GENIE_OK;
}

extern "C" void genie_parts_destroy(genie_parts* ps) {
  if (!ps) return;
  if (ps->copy) cudaStreamSynchronize(ps->copy);
  cudaDeviceSynchronize();
  for (HostPart& h : ps->parts) {
    cudaFreeHost(h.kw_off);
    cudaFreeHost(h.post_ids);
    cudaFreeHost(h.post16);
    cudaFreeHost(h.chunk_pos);
  }
  free_slots(ps);
  for (int i = 0; i < 2; ++i) {
    if (ps->copied[i]) cudaEventDestroy(ps->copied[i]);
    if (ps->used[i]) cudaEventDestroy(ps->used[i]);
  }
  if (ps->copy) cudaStreamDestroy(ps->copy);
  delete ps;
}

extern "C" genie_status genie_parts_add(genie_parts* ps, const genie_index* index, uint32_t id_base,
                                        genie_stream stream) {
  if (!ps || !index) return fail(GENIE_ERR_INVALID_ARG, "genie_parts_add: NULL argument");
  if (!ps->parts.empty() && index->vocab != ps->vocab)
    return fail(GENIE_ERR_INVALID_ARG, "genie_parts_add: the parts must share one vocabulary");
  const HostPart* last = ps->parts.empty() ? nullptr : &ps->parts.back();
  if (last && (uint64_t)id_base < (uint64_t)last->base + last->n_objects)
    return fail(GENIE_ERR_INVALID_ARG,
                "genie_parts_add: parts must come in ascending, disjoint object-id ranges");
  if ((uint64_t)id_base + index->n_objects >= 0xFFFFFFFFull)
    return fail(GENIE_ERR_INVALID_ARG, "genie_parts_add: global object ids must stay below 2^32 - 1");
  HostPart h;
  h.base = id_base;
  h.n_objects = index->n_objects;
  h.max_object_len = index->max_object_len;
  h.chunk_shift = index->chunk_shift;
  h.n_chunks = index->n_chunks;
  h.nnz = index->nnz;
  h.post_len = ((index->nnz + 3) & ~3ull) + 4;  // the padded List Array
  h.chunk_len = (uint64_t)index->vocab * (index->n_chunks + 1);
  cudaStream_t s = as_stream(stream);
  const bool narrow = index->chunk_shift <= 16;  // the places fit in 16 bits
  uint16_t* d16 = nullptr;
  cudaError_t e = cudaMallocHost(&h.kw_off, ((uint64_t)index->vocab + 1) * 8);
  if (e == cudaSuccess && narrow) e = cudaMallocHost(&h.post16, h.post_len * 2);
  if (e == cudaSuccess && !narrow) e = cudaMallocHost(&h.post_ids, h.post_len * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&h.chunk_pos, h.chunk_len * 4);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.kw_off, index->kw_off, ((uint64_t)index->vocab + 1) * 8,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && narrow) {
    e = cudaMallocAsync((void**)&d16, h.post_len * 2, s);
    if (e == cudaSuccess) {
      narrow_ids_kernel<<<grid_for(h.post_len, 256), 256, 0, s>>>(
          index->post_ids, h.post_len, (1u << index->chunk_shift) - 1u, d16);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.post16, d16, h.post_len * 2, cudaMemcpyDeviceToHost, s);
    if (d16) {
      cudaError_t f = cudaFreeAsync(d16, s);
      if (e == cudaSuccess) e = f;
    }
  } else if (e == cudaSuccess) {
    e = cudaMemcpyAsync(h.post_ids, index->post_ids, h.post_len * 4, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.chunk_pos, index->chunk_pos, h.chunk_len * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeHost(h.kw_off);
    cudaFreeHost(h.post_ids);
    cudaFreeHost(h.post16);
    cudaFreeHost(h.chunk_pos);
    return fail_cuda(e, "genie_parts_add");
  }
  ps->vocab = index->vocab;
  ps->parts.push_back(h);
  return GENIE_OK;
}

extern "C" genie_status genie_parts_get_info(const genie_parts* ps, genie_parts_info* out) {
  if (!ps || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_parts_get_info: NULL argument");
  out->n_parts = (uint32_t)ps->parts.size();
  out->vocab = ps->vocab;
  out->n_objects = ps->parts.empty() ? 0 : ps->parts.back().base + ps->parts.back().n_objects;
  out->host_bytes = 0;
  out->max_part_bytes = 0;
  for (const HostPart& h : ps->parts) {
    const uint64_t b = ((uint64_t)ps->vocab + 1) * 8 + h.post_bytes() + h.chunk_len * 4;
    out->host_bytes += b;
    out->max_part_bytes = std::max(out->max_part_bytes, b);
  }
  return GENIE_OK;
}

extern "C" genie_status genie_parts_search(genie_parts* ps, const uint32_t* d_q_off,
                                           const uint32_t* d_q_kw, uint32_t n_queries, uint32_t k,
                                           const uint32_t* d_k, uint32_t* d_ids, uint32_t* d_counts,
                                           uint32_t* d_n_valid, genie_stream stream) {
  if (!ps || !d_q_off || !d_ids || !d_counts || !d_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_parts_search: NULL argument");
  if (ps->parts.empty()) return fail(GENIE_ERR_INVALID_ARG, "genie_parts_search: no parts");
  if (k == 0 || k > GENIE_MAX_K) return fail(GENIE_ERR_INVALID_ARG, "genie_parts_search: k must be in 1..GENIE_MAX_K");
  if (n_queries == 0) return GENIE_OK;
  cudaStream_t s = as_stream(stream);
  const uint32_t P = (uint32_t)ps->parts.size(), Q = n_queries;
  GENIE_CUDA_TRY(ensure_slots(ps));
  // scratch: per-part outputs, then keys, bounds and part bases
  const uint64_t out_words = (uint64_t)P * Q * k;
  const uint64_t bytes = out_words * 8 + (uint64_t)P * Q * 4 + out_words * 8 + (uint64_t)Q * 4 + P * 4 + 64;
  unsigned char* base = nullptr;
  GENIE_CUDA_TRY(cudaMallocAsync((void**)&base, bytes, s));
  uint32_t* p_ids = reinterpret_cast<uint32_t*>(base);
  uint32_t* p_counts = p_ids + out_words;
  uint32_t* p_nv = p_counts + out_words;
  unsigned long long* keys =
      reinterpret_cast<unsigned long long*>(((uintptr_t)(p_nv + (uint64_t)P * Q) + 15) & ~(uintptr_t)15);
  uint32_t* max_b = reinterpret_cast<uint32_t*>(keys + out_words);
  uint32_t* d_bases = max_b + Q;
  std::vector<uint32_t> bases(P);
  for (uint32_t p = 0; p < P; ++p) bases[p] = ps->parts[p].base;
  cudaError_t e = cudaMemsetAsync(max_b, 0, (size_t)Q * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_bases, bases.data(), P * 4, cudaMemcpyHostToDevice, s);
  // the slots are free once the work enqueued so far on `s` is done
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(ps->used[i], s);
  auto load = [&](uint32_t p) -> cudaError_t {
    const HostPart& h = ps->parts[p];
    genie_index& sl = ps->slot[p & 1];
    if (ps->slot_part[p & 1] == (int64_t)p) return cudaSuccess;  // still there from the call before
    ps->slot_part[p & 1] = p;
    ps->slot_wide[p & 1] = false;
    cudaError_t r = cudaStreamWaitEvent(ps->copy, ps->used[p & 1], 0);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(sl.kw_off, h.kw_off, ((uint64_t)ps->vocab + 1) * 8, cudaMemcpyHostToDevice,
                          ps->copy);
    if (r == cudaSuccess && h.post16)
      r = cudaMemcpyAsync(ps->stage16[p & 1], h.post16, h.post_len * 2, cudaMemcpyHostToDevice, ps->copy);
    else if (r == cudaSuccess)
      r = cudaMemcpyAsync(sl.post_ids, h.post_ids, h.post_len * 4, cudaMemcpyHostToDevice, ps->copy);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(sl.chunk_pos, h.chunk_pos, h.chunk_len * 4, cudaMemcpyHostToDevice, ps->copy);
    if (r == cudaSuccess) r = cudaEventRecord(ps->copied[p & 1], ps->copy);
    return r;
  };
  genie_status st = GENIE_OK;
  uint32_t za_len = 2;
  if (e == cudaSuccess) e = load(0);
  for (uint32_t p = 0; p < P && e == cudaSuccess && st == GENIE_OK; ++p) {
    if (p + 1 < P) e = load(p + 1);  // overlaps the search of part p
    // With an even number of parts, part 0's slot is free while the last one
    // is searched: load part 0 there for the next call.
    else if (P % 2 == 0) e = load(0);
    if (e != cudaSuccess) break;
    e = cudaStreamWaitEvent(s, ps->copied[p & 1], 0);
    if (e != cudaSuccess) break;
    const HostPart& h = ps->parts[p];
    genie_index& sl = ps->slot[p & 1];
    if (h.post16 && !ps->slot_wide[p & 1]) {
      // ids from their places (zero padding after the lists).  On `s`, not on
      // the copy stream, so that the next part's copy never waits for SMs
      // that this part's search holds.
      const uint32_t n_seg = (uint32_t)((h.nnz + kWidenSeg - 1) / kWidenSeg);
      if (n_seg) {
        segment_keywords_kernel<<<grid_for(n_seg + 1ull, 256), 256, 0, s>>>(sl.kw_off, ps->vocab, h.nnz,
                                                                          n_seg, ps->seg_kw);
        widen_ids_kernel<<<n_seg, kWidenThreads, 0, s>>>(sl.kw_off, sl.chunk_pos, h.n_chunks,
                                                         h.chunk_shift, h.nnz, ps->seg_kw,
                                                         ps->stage16[p & 1], sl.post_ids);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(sl.post_ids + h.nnz, 0, (h.post_len - h.nnz) * 4, s);
      if (e != cudaSuccess) break;
      ps->slot_wide[p & 1] = true;
    }
    sl.n_objects = h.n_objects;
    sl.nnz = h.nnz;
    sl.max_object_len = h.max_object_len;
    sl.chunk_shift = h.chunk_shift;
    sl.n_chunks = h.n_chunks;
    genie_queries* qs = nullptr;
    st = genie_make_queries(&sl, d_q_off, d_q_kw, Q, stream, &qs);
    if (st != GENIE_OK) break;
    st = genie_search(&sl, qs, k, d_k, nullptr, p_ids + (uint64_t)p * Q * k,
                      p_counts + (uint64_t)p * Q * k, p_nv + (uint64_t)p * Q, stream);
    if (st == GENIE_OK) {
      max_bound_kernel<<<grid_for(Q, 256), 256, 0, s>>>(qs->bound, Q, max_b);
      za_len = std::max(za_len, qs->max_bound + 2);
      e = cudaGetLastError();
    }
    genie_queries_destroy(qs);
    if (e == cudaSuccess && st == GENIE_OK) e = cudaEventRecord(ps->used[p & 1], s);
  }
  if (e == cudaSuccess && st == GENIE_OK) {
    part_keys_kernel<<<grid_for(out_words, 256), 256, 0, s>>>(p_ids, p_counts, p_nv, d_bases, P, Q,
                                                               k, keys);
    MergeArgs m;
    m.cand = keys;
    m.n_sel = Q;
    m.q_sel = nullptr;
    m.n_groups = P;
    m.k = k;
    m.k_arr = d_k;
    m.bound = max_b;
    m.za_len = za_len;
    m.ids = d_ids;
    m.counts = d_counts;
    m.n_valid = d_n_valid;
    const size_t msmem = dev::next_pow2(k) * 8 + (size_t)za_len * 4;
    e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
    if (e == cudaSuccess) {
      merge_kernel<<<std::min<uint32_t>(Q, 152u * 16u), kMergeThreads, msmem, s>>>(m);
      e = cudaGetLastError();
    }
  }
  // the copy stream must not write a slot after this call returns
  cudaError_t e2 = cudaStreamSynchronize(ps->copy);
  cudaFreeAsync(base, s);
  if (st != GENIE_OK || e != cudaSuccess || e2 != cudaSuccess)
    ps->slot_part[0] = ps->slot_part[1] = -1;  // a slot may hold part of a part
  if (st != GENIE_OK) return st;
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return fail_cuda(e, "genie_parts_search");
  return GENIE_OK;
}

// ---------------------------------------------------------------------------
// genie_merge_host: the result merge of the multiple-loading method on the host
// ---------------------------------------------------------------------------
//
// Sec. 3.4 merges the per-part top-k lists on the CPU (Table 4, "Result
// merge").  Every list is ranked by (count desc, id asc) and holds its part's
// exact top-k, ties at its k-th count taken in ascending id; an object a part
// left out is outranked by k objects of that part, so the union of the lists
// holds the whole batch's top-k, and a k-way merge of the lists under the same
// order yields it.  This is the exchange of an object-sharded search over
// several GPUs: each GPU searches its shard, the lists meet on one host.

extern "C" genie_status genie_merge_host(uint32_t n_parts, const uint32_t* const* h_ids,
                                         const uint32_t* const* h_counts, uint32_t n_queries,
                                         uint32_t k_part, uint32_t k, uint32_t* h_ids_out,
                                         uint32_t* h_counts_out, uint32_t* h_n_valid) {
  if (n_parts == 0 || !h_ids || !h_counts || !h_ids_out || !h_counts_out || !h_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_merge_host: NULL argument or no part");
  if (k == 0 || k > GENIE_MAX_K || k_part == 0 || k_part > GENIE_MAX_K)
    return fail(GENIE_ERR_INVALID_ARG, "genie_merge_host: k and k_part must be in 1..GENIE_MAX_K");
  for (uint32_t p = 0; p < n_parts; ++p)
    if (!h_ids[p] || !h_counts[p]) return fail(GENIE_ERR_INVALID_ARG, "genie_merge_host: NULL list");
  std::vector<uint32_t> cur(n_parts);
  for (uint64_t q = 0; q < n_queries; ++q) {
    std::fill(cur.begin(), cur.end(), 0u);
    uint32_t n = 0;
    uint32_t* out_i = h_ids_out + q * k;
    uint32_t* out_c = h_counts_out + q * k;
    while (n < k) {
      // the head of the list whose next entry ranks first: count desc, id asc
      int best = -1;
      uint32_t bc = 0, bi = 0;
      for (uint32_t p = 0; p < n_parts; ++p) {
        if (cur[p] >= k_part) continue;
        const uint32_t c = h_counts[p][q * k_part + cur[p]], id = h_ids[p][q * k_part + cur[p]];
        if (c == 0) continue;  // padding: the list has ended
        if (best < 0 || c > bc || (c == bc && id < bi)) {
          best = (int)p;
          bc = c;
          bi = id;
        }
      }
      if (best < 0) break;
      out_i[n] = bi;
      out_c[n] = bc;
      ++cur[best];
      ++n;
    }
    h_n_valid[q] = n;
    for (uint32_t j = n; j < k; ++j) {
      out_i[j] = 0xFFFFFFFFu;
      out_c[j] = 0;
    }
  }
  return GENIE_OK;
}
