// Device-side construction of the inverted index (Sec. 3.2, Fig. 3) and of
// the sublist map (Sec. 3.2.1).
//
// The paper builds its index on the CPU (Table 2, "Index-build").  Here the
// transposition object -> keywords into keyword -> objects is a stable LSD
// radix sort of the (keyword, object id) pairs by keyword, eight bits per pass
// (three passes for a vocabulary of up to 2^24): per tile a 256-bin digit
// histogram, one exclusive scan over the (digit, tile) counts, and a scatter
// that ranks each pair among the tile's pairs with the same digit in input
// order.  The pairs enter in ascending object id, so stability leaves every
// postings list in ascending id order, which the block-per-object-range scan
// depends on.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

// Radix tiles: 256 threads (one per digit value) x 16 pairs; each warp ranks
// a contiguous 512 pairs of the tile.
constexpr uint32_t kRadixBits = 8;
constexpr uint32_t kDigits = 1u << kRadixBits;
constexpr uint32_t kRadixThreads = kDigits;
constexpr uint32_t kRadixItems = 16;
constexpr uint32_t kRadixTile = kRadixThreads * kRadixItems;
constexpr uint32_t kRadixWarps = kRadixThreads / 32;
// Large exclusive scans: blocks of 256 threads x 16 values.
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kScanItems = 16;
constexpr uint32_t kScanChunk = kScanThreads * kScanItems;

enum BuildFlag { kBadOffsets = 0, kBadKeyword = 1, kMaxLen = 2, kDuplicate = 3, kNumFlags = 4 };

__global__ void validate_objects_kernel(const uint32_t* __restrict__ off, const uint32_t* __restrict__ kw,
                                        uint32_t n_obj, uint64_t nnz, uint32_t vocab,
                                        uint32_t* flags) {
  uint32_t max_len = 0;
  bool bad_off = false, bad_kw = false;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n_obj;
       o += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t a = off[o], b = off[o + 1];
    if (b < a || b > nnz) {
      bad_off = true;
      continue;
    }
    max_len = max(max_len, b - a);
    for (uint32_t e = a; e < b; ++e) bad_kw |= kw[e] >= vocab;
  }
  if (bad_off) atomicOr(&flags[kBadOffsets], 1u);
  if (bad_kw) atomicOr(&flags[kBadKeyword], 1u);
  atomicMax(&flags[kMaxLen], max_len);
}

// keys[e] = keyword, vals[e] = object id of posting e (object order).
__global__ void expand_pairs_kernel(const uint32_t* __restrict__ off, const uint32_t* __restrict__ kw,
                                    uint32_t n_obj, uint32_t* __restrict__ keys,
                                    uint32_t* __restrict__ vals) {
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < n_obj; o += warps) {
    uint32_t a = off[o], b = off[o + 1];
    for (uint32_t e = a + dev::lane_id(); e < b; e += 32) {
      keys[e] = kw[e];
      vals[e] = o;
    }
  }
}

// Digit histogram of each tile: tile_hist[d * n_tiles + tile] = pairs of the
// tile whose key has digit d at `shift` (d < nd; larger digits do not occur).
__global__ void radix_count_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint32_t shift,
                                   uint32_t nd, uint32_t n_tiles, uint32_t* __restrict__ tile_hist) {
  __shared__ uint32_t h[kDigits];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t start = (uint64_t)blockIdx.x * kRadixTile;
#pragma unroll
  for (uint32_t j = 0; j < kRadixItems; ++j) {
    const uint64_t i = start + j * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kDigits - 1)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < nd) tile_hist[(uint64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Sums of consecutive chunks of kScanChunk values (first phase of a scan).
__global__ void scan_partial_kernel(const uint32_t* __restrict__ v, uint64_t n,
                                    uint32_t* __restrict__ part) {
  __shared__ uint32_t scratch[33];
  const uint64_t start = (uint64_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
#pragma unroll
  for (uint32_t j = 0; j < kScanItems; ++j) {
    const uint64_t i = start + j * kScanThreads + threadIdx.x;
    if (i < n) s += v[i];
  }
  const uint32_t total = dev::block_sum(s, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Exclusive scan of each chunk in place, offset by the chunk's scanned sum.
__global__ void scan_apply_kernel(uint32_t* __restrict__ v, uint64_t n,
                                  const uint32_t* __restrict__ part) {
  __shared__ uint32_t scratch[33];
  const uint64_t mine = (uint64_t)blockIdx.x * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
  uint32_t x[kScanItems], s = 0;
#pragma unroll
  for (uint32_t j = 0; j < kScanItems; ++j) {
    x[j] = mine + j < n ? v[mine + j] : 0u;
    s += x[j];
  }
  uint32_t tot;
  uint32_t base = part[blockIdx.x] + dev::block_exclusive_scan(s, scratch, &tot);
#pragma unroll
  for (uint32_t j = 0; j < kScanItems; ++j) {
    if (mine + j < n) v[mine + j] = base;
    base += x[j];
  }
}

}  // namespace

// exclusive scan of n values in place, total into *total (one block)
__global__ void scan_small_kernel(uint32_t* __restrict__ v, uint32_t n, uint32_t* total) {
  __shared__ uint32_t scratch[33];
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t a = min(n, threadIdx.x * per), b = min(n, a + per);
  uint32_t s = 0;
  for (uint32_t i = a; i < b; ++i) s += v[i];
  uint32_t tot;
  uint32_t base = dev::block_exclusive_scan(s, scratch, &tot);
  for (uint32_t i = a; i < b; ++i) {
    uint32_t x = v[i];
    v[i] = base;
    base += x;
  }
  if (threadIdx.x == 0) *total = tot;
}

void launch_exclusive_scan(uint32_t* v, uint32_t n, uint32_t* total, cudaStream_t s) {
  scan_small_kernel<<<1, 1024, 0, s>>>(v, n, total);
}

namespace {

// Stable scatter of one tile by the digit at `shift`.  A pair's destination
// is tile_off[d * n_tiles + tile] (the pairs of digit d in earlier tiles and
// of smaller digits everywhere, from the scan of the histograms) plus its
// rank among the tile's pairs of digit d.  Warp w ranks the tile's pairs
// [512 w, 512 w + 512) in 16 rounds of 32 consecutive pairs: the lanes that
// share a digit in a round find each other with match.any, take their order
// from their lane numbers and their base from the warp's running count of the
// digit; the counts of the warps before it are added afterwards.  The tile is
// then laid out in shared memory in destination order and written from
// there, so that consecutive threads write consecutive addresses.
__global__ void __launch_bounds__(kRadixThreads)
    radix_scatter_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                         uint32_t n, uint32_t shift, uint32_t nd, uint32_t n_tiles,
                         const uint32_t* __restrict__ tile_off, uint32_t* __restrict__ keys_out,
                         uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t wh[kRadixWarps][kDigits];
  __shared__ uint32_t loc[kDigits];   // first tile position of each digit
  __shared__ uint32_t glob[kDigits];  // first destination of each digit's pairs of the tile
  __shared__ uint32_t sk[kRadixTile], sv[kRadixTile];
  __shared__ uint32_t scratch[33];
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (uint32_t w = 0; w < kRadixWarps; ++w) wh[w][tid] = 0;
  __syncthreads();
  const uint64_t tile_start = (uint64_t)blockIdx.x * kRadixTile;
  const uint64_t wbase = tile_start + warp * (32u * kRadixItems);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t k[kRadixItems], v[kRadixItems], r[kRadixItems];
#pragma unroll
  for (uint32_t j = 0; j < kRadixItems; ++j) {
    const uint64_t i = wbase + j * 32 + lane;
    const bool ok = i < n;
    k[j] = ok ? keys[i] : 0u;
    v[j] = ok ? vals[i] : 0u;
    const uint32_t d = ok ? (k[j] >> shift) & (kDigits - 1) : kDigits;  // kDigits: no pair
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (ok && lane == leader) {
      before = wh[warp][d];
      wh[warp][d] = before + __popc(peers);
    }
    r[j] = __shfl_sync(0xFFFFFFFFu, before, leader) + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  // thread d: the tile's pairs of digit d in the warps before each warp
  uint32_t cnt = 0;
#pragma unroll
  for (uint32_t w = 0; w < kRadixWarps; ++w) {
    const uint32_t c = wh[w][tid];
    wh[w][tid] = cnt;
    cnt += c;
  }
  uint32_t tot;
  const uint32_t first = dev::block_exclusive_scan(cnt, scratch, &tot);
  loc[tid] = first;
  glob[tid] = tid < nd ? tile_off[(uint64_t)tid * n_tiles + blockIdx.x] : 0u;
  __syncthreads();
#pragma unroll
  for (uint32_t j = 0; j < kRadixItems; ++j) {
    if (wbase + j * 32 + lane < n) {
      const uint32_t d = (k[j] >> shift) & (kDigits - 1);
      const uint32_t pos = loc[d] + wh[warp][d] + r[j];
      sk[pos] = k[j];
      sv[pos] = v[j];
    }
  }
  __syncthreads();
  const uint32_t tile_n = (uint32_t)min((uint64_t)kRadixTile, (uint64_t)n - tile_start);
  for (uint32_t i = tid; i < tile_n; i += kRadixThreads) {
    const uint32_t kk = sk[i];
    const uint32_t d = (kk >> shift) & (kDigits - 1);
    const uint32_t dst = glob[d] + (i - loc[d]);
    keys_out[dst] = kk;
    vals_out[dst] = sv[i];
  }
}

__global__ void check_duplicates_kernel(const uint32_t* __restrict__ keys,
                                        const uint32_t* __restrict__ vals, uint32_t n,
                                        uint32_t* flags) {
  bool dup = false;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    dup |= keys[i] == keys[i - 1] && vals[i] == vals[i - 1];
  if (dup) atomicOr(&flags[kDuplicate], 1u);
}

// kw_off[v] = first position whose key >= v (Position Map)
__global__ void list_offsets_kernel(const uint32_t* __restrict__ keys, uint32_t n, uint32_t vocab,
                                    uint64_t* __restrict__ kw_off) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v <= vocab;
       v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
      uint32_t mid = lo + ((hi - lo) >> 1);
      if (keys[mid] < v) lo = mid + 1; else hi = mid;
    }
    kw_off[v] = lo;
  }
}

// chunk_pos[v*(nch+1) + c] = first position in list v of an id >= c << shift
__global__ void sublist_map_kernel(const uint64_t* __restrict__ kw_off, const uint32_t* __restrict__ ids,
                                   uint32_t vocab, uint32_t nch, uint32_t shift,
                                   uint32_t* __restrict__ chunk_pos) {
  const uint64_t total = (uint64_t)vocab * (nch + 1);
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = (uint32_t)(t / (nch + 1));
    uint32_t c = (uint32_t)(t % (nch + 1));
    uint64_t a = kw_off[v], b = kw_off[v + 1];
    uint64_t want = (uint64_t)c << shift;
    uint64_t lo = a, hi = b;
    while (lo < hi) {
      uint64_t mid = lo + ((hi - lo) >> 1);
      if ((uint64_t)ids[mid] < want) lo = mid + 1; else hi = mid;
    }
    chunk_pos[t] = (uint32_t)(lo - a);
  }
}

// Object bitmaps of the dense keywords: one block per dense keyword; each
// thread folds a run of its (ascending) ids into one word at a time and sets
// it with one atomicOr when the word changes.
__global__ void dense_fill_kernel(const uint64_t* __restrict__ kw_off,
                                  const uint32_t* __restrict__ ids,
                                  const uint32_t* __restrict__ dense_kw, uint64_t map_words,
                                  uint32_t* __restrict__ bits) {
  const uint32_t kw = dense_kw[blockIdx.x];
  uint32_t* map = bits + (uint64_t)blockIdx.x * map_words;
  const uint64_t a = kw_off[kw], b = kw_off[kw + 1];
  const uint64_t per = (b - a + blockDim.x - 1) / blockDim.x;
  const uint64_t lo = a + per * threadIdx.x, hi = min(b, lo + per);
  uint32_t word = 0xFFFFFFFFu, acc = 0;
  for (uint64_t p = lo; p < hi; ++p) {
    const uint32_t id = ids[p];
    if ((id >> 5) != word) {
      if (acc) atomicOr(&map[word], acc);
      word = id >> 5;
      acc = 0;
    }
    acc |= 1u << (id & 31);
  }
  if (acc) atomicOr(&map[word], acc);
}

int grid_for(uint64_t n, int threads, int cap = 152 * 32) {
  uint64_t g = (n + threads - 1) / threads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)cap));
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_build_index_ex(const uint32_t* d_obj_off, const uint32_t* d_obj_kw,
                                             uint32_t n_objects, uint32_t vocab,
                                             const genie_index_opts* opts, genie_stream stream,
                                             genie_index** out) {
  uint32_t chunk_shift = opts ? opts->chunk_shift : 0u;
  if (!out) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: out is NULL");
  if (!d_obj_off) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: d_obj_off is NULL");
  if (n_objects == 0 || n_objects > (1u << 31))
    return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: n_objects must be in 1..2^31");
  if (vocab == 0 || vocab > (1u << 31))
    return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: vocab must be in 1..2^31");
  if (chunk_shift == 0) chunk_shift = 16;  // the object range of a 16-bit-counter block
  if (chunk_shift < 12 || chunk_shift > 20)
    return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: chunk_shift must be 0 or 12..20");
  cudaStream_t s = as_stream(stream);

  uint32_t ends[2];
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[0], d_obj_off, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaMemcpyAsync(&ends[1], d_obj_off + n_objects, 4, cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (ends[0] != 0) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: d_obj_off[0] != 0");
  const uint32_t nnz = ends[1];
  if (nnz > 0xFFFFFFF0u) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: too many postings");
  if (nnz > 0 && !d_obj_kw) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: d_obj_kw is NULL");

  DevBuf flags_b, keys_a, keys_b, vals_a, vals_b, tiles_b;
  GENIE_CUDA_TRY(cudaMalloc(&flags_b.p, 64));
  uint32_t* flags = (uint32_t*)flags_b.p;
  GENIE_CUDA_TRY(cudaMemsetAsync(flags, 0, 64, s));
  validate_objects_kernel<<<grid_for(n_objects, 256), 256, 0, s>>>(d_obj_off, d_obj_kw, n_objects,
                                                                    nnz, vocab, flags);
  GENIE_CUDA_TRY(cudaGetLastError());
  uint32_t hflags[kNumFlags];
  GENIE_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (hflags[kBadOffsets]) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: object offsets are not non-decreasing within [0, nnz]");
  if (hflags[kBadKeyword]) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: a keyword id is >= vocab");

  const uint64_t padded = ((uint64_t)nnz + 3) / 4 * 4 + 4;  // aligned 16-byte loads stay inside
  GENIE_CUDA_TRY(cudaMalloc(&keys_a.p, std::max<uint64_t>(nnz, 1) * 4));
  GENIE_CUDA_TRY(cudaMalloc(&keys_b.p, std::max<uint64_t>(nnz, 1) * 4));
  GENIE_CUDA_TRY(cudaMalloc(&vals_a.p, padded * 4));
  GENIE_CUDA_TRY(cudaMalloc(&vals_b.p, padded * 4));
  int bits = 0;
  while (bits < 32 && ((uint64_t)1 << bits) < vocab) ++bits;
  const uint32_t n_tiles = (uint32_t)((nnz + kRadixTile - 1) / kRadixTile);
  const uint32_t max_nd = (uint32_t)std::min<uint64_t>(kDigits, (uint64_t)1 << bits);
  const uint64_t hist_n = (uint64_t)max_nd * n_tiles;
  const uint32_t n_parts = (uint32_t)((hist_n + kScanChunk - 1) / kScanChunk);
  GENIE_CUDA_TRY(cudaMalloc(&tiles_b.p, (hist_n + n_parts + 2) * 4));
  uint32_t* tile_hist = (uint32_t*)tiles_b.p;
  uint32_t* parts = tile_hist + hist_n;
  uint32_t* parts_total = parts + n_parts + 1;

  uint32_t *ka = (uint32_t*)keys_a.p, *kb = (uint32_t*)keys_b.p;
  uint32_t *va = (uint32_t*)vals_a.p, *vb = (uint32_t*)vals_b.p;
  if (nnz > 0) {
    expand_pairs_kernel<<<grid_for((uint64_t)n_objects * 32, 256), 256, 0, s>>>(d_obj_off, d_obj_kw,
                                                                               n_objects, ka, va);
    GENIE_CUDA_TRY(cudaGetLastError());
    for (uint32_t shift = 0; shift < (uint32_t)bits; shift += kRadixBits) {
      const uint32_t nd = 1u << std::min<uint32_t>(kRadixBits, (uint32_t)bits - shift);
      const uint64_t hn = (uint64_t)nd * n_tiles;
      const uint32_t np = (uint32_t)((hn + kScanChunk - 1) / kScanChunk);
      radix_count_kernel<<<n_tiles, kRadixThreads, 0, s>>>(ka, nnz, shift, nd, n_tiles, tile_hist);
      scan_partial_kernel<<<np, kScanThreads, 0, s>>>(tile_hist, hn, parts);
      scan_small_kernel<<<1, 1024, 0, s>>>(parts, np, parts_total);
      scan_apply_kernel<<<np, kScanThreads, 0, s>>>(tile_hist, hn, parts);
      radix_scatter_kernel<<<n_tiles, kRadixThreads, 0, s>>>(ka, va, nnz, shift, nd, n_tiles,
                                                             tile_hist, kb, vb);
      GENIE_CUDA_TRY(cudaGetLastError());
      std::swap(ka, kb);
      std::swap(va, vb);
    }
    check_duplicates_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(ka, va, nnz, flags);
    GENIE_CUDA_TRY(cudaGetLastError());
  }
  GENIE_CUDA_TRY(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
  GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  if (hflags[kDuplicate]) return fail(GENIE_ERR_INVALID_ARG, "genie_build_index: an object repeats a keyword (objects are sets)");

  genie_index* idx = new (std::nothrow) genie_index();
  if (!idx) return fail(GENIE_ERR_OUT_OF_MEMORY, "genie_build_index: host allocation");
  cudaGetDevice(&idx->device);
  idx->n_objects = n_objects;
  idx->vocab = vocab;
  idx->nnz = nnz;
  idx->max_object_len = hflags[kMaxLen];
  idx->chunk_shift = chunk_shift;
  idx->n_chunks = (uint32_t)(((uint64_t)n_objects + (1u << chunk_shift) - 1) >> chunk_shift);
  auto cleanup = [&](genie_status st) {
    cudaFree(idx->kw_off);
    cudaFree(idx->chunk_pos);
    cudaFree(idx->dense_slot);
    cudaFree(idx->dense_bits);
    delete idx;
    return st;
  };
  cudaError_t e = cudaMalloc(&idx->kw_off, ((uint64_t)vocab + 1) * 8);
  if (e != cudaSuccess) return cleanup(fail_cuda(e, "cudaMalloc(kw_off)"));
  const uint64_t tab_n = (uint64_t)vocab * (idx->n_chunks + 1);
  e = cudaMalloc(&idx->chunk_pos, tab_n * 4);
  if (e != cudaSuccess) return cleanup(fail_cuda(e, "cudaMalloc(chunk_pos)"));

  list_offsets_kernel<<<grid_for((uint64_t)vocab + 1, 256), 256, 0, s>>>(ka, nnz, vocab, idx->kw_off);
  // the sorted object ids become the List Array; keep the buffer, zero its padding
  idx->post_ids = va;
  if (va == (uint32_t*)vals_a.p) vals_a.p = nullptr; else vals_b.p = nullptr;
  e = cudaMemsetAsync(idx->post_ids + nnz, 0, (padded - nnz) * 4, s);
  if (e == cudaSuccess) {
    sublist_map_kernel<<<grid_for(tab_n, 256), 256, 0, s>>>(idx->kw_off, idx->post_ids, vocab,
                                                            idx->n_chunks, chunk_shift, idx->chunk_pos);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(idx->post_ids);
    return cleanup(fail_cuda(e, "genie_build_index kernels"));
  }
  idx->device_bytes = ((uint64_t)vocab + 1) * 8 + padded * 4 + tab_n * 4;

  // Dense keywords: lists of at least dense_min_df postings also become
  // object bitmaps (n_objects bits, padded so that a search block's slice of
  // up to 2^18 objects, plus one word, stays inside).
  uint32_t min_df = opts ? opts->dense_min_df : 0u;
  // default: a bitmap (n_objects bits) no larger than the list (32 bits a posting)
  if (min_df == 0) min_df = std::max<uint32_t>(64u, (n_objects + 31) / 32);
  idx->dense_min_df = min_df;
  if (min_df != GENIE_NO_DENSE && nnz > 0) {
    std::vector<uint64_t> h_off((size_t)vocab + 1);
    e = cudaMemcpyAsync(h_off.data(), idx->kw_off, h_off.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(idx->post_ids);
      return cleanup(fail_cuda(e, "genie_build_index: list offsets"));
    }
    std::vector<uint32_t> slot(vocab, kNoDense), dense_kw;
    for (uint32_t v = 0; v < vocab; ++v)
      if (h_off[v + 1] - h_off[v] >= min_df) {
        slot[v] = (uint32_t)dense_kw.size();
        dense_kw.push_back(v);
        idx->dense_postings += h_off[v + 1] - h_off[v];
      }
    if (!dense_kw.empty()) {
      const uint64_t words = ((uint64_t)n_objects + 31) / 32 + 2;
      idx->map_words = (words + 8191) / 8192 * 8192;
      idx->n_dense = (uint32_t)dense_kw.size();
      uint32_t* d_kw = nullptr;
      e = cudaMalloc(&idx->dense_slot, (uint64_t)vocab * 4);
      if (e == cudaSuccess) e = cudaMalloc(&idx->dense_bits, idx->n_dense * idx->map_words * 4);
      if (e == cudaSuccess) e = cudaMalloc(&d_kw, dense_kw.size() * 4);
      if (e == cudaSuccess) e = cudaMemcpyAsync(idx->dense_slot, slot.data(), (uint64_t)vocab * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_kw, dense_kw.data(), dense_kw.size() * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(idx->dense_bits, 0, idx->n_dense * idx->map_words * 4, s);
      if (e == cudaSuccess) {
        dense_fill_kernel<<<idx->n_dense, 256, 0, s>>>(idx->kw_off, idx->post_ids, d_kw,
                                                       idx->map_words, idx->dense_bits);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(d_kw);
      if (e != cudaSuccess) {
        cudaFree(idx->post_ids);
        return cleanup(fail_cuda(e, "genie_build_index: dense bitmaps"));
      }
      idx->device_bytes += (uint64_t)vocab * 4 + idx->n_dense * idx->map_words * 4;
    }
  }
  *out = idx;
  return GENIE_OK;
}

extern "C" genie_status genie_build_index(const uint32_t* d_obj_off, const uint32_t* d_obj_kw,
                                          uint32_t n_objects, uint32_t vocab,
                                          uint32_t chunk_shift, genie_stream stream,
                                          genie_index** out) {
  genie_index_opts o;
  o.chunk_shift = chunk_shift;
  o.dense_min_df = 0;
  return genie_build_index_ex(d_obj_off, d_obj_kw, n_objects, vocab, &o, stream, out);
}

extern "C" void genie_index_destroy(genie_index* index) {
  if (!index) return;
  cudaDeviceSynchronize();
  cudaFree(index->kw_off);
  cudaFree(index->post_ids);
  cudaFree(index->chunk_pos);
  cudaFree(index->dense_slot);
  cudaFree(index->dense_bits);
  delete index;
}

extern "C" genie_status genie_index_get_info(const genie_index* index, genie_index_info* out) {
  if (!index || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_index_get_info: NULL argument");
  out->n_objects = index->n_objects;
  out->vocab = index->vocab;
  out->nnz = index->nnz;
  out->max_object_len = index->max_object_len;
  out->chunk_shift = index->chunk_shift;
  out->n_chunks = index->n_chunks;
  out->reserved = 0;
  out->device_bytes = index->device_bytes;
  out->dense_keywords = index->n_dense;
  out->dense_min_df = index->dense_min_df;
  out->dense_bytes = index->n_dense ? (uint64_t)index->vocab * 4 + index->n_dense * index->map_words * 4 : 0;
  return GENIE_OK;
}

extern "C" genie_status genie_index_export(const genie_index* index, uint64_t* d_kw_off,
                                           uint32_t* d_post_ids, genie_stream stream) {
  if (!index) return fail(GENIE_ERR_INVALID_ARG, "genie_index_export: index is NULL");
  cudaStream_t s = as_stream(stream);
  if (d_kw_off)
    GENIE_CUDA_TRY(cudaMemcpyAsync(d_kw_off, index->kw_off, ((uint64_t)index->vocab + 1) * 8,
                                   cudaMemcpyDeviceToDevice, s));
  if (d_post_ids && index->nnz)
    GENIE_CUDA_TRY(cudaMemcpyAsync(d_post_ids, index->post_ids, index->nnz * 4,
                                   cudaMemcpyDeviceToDevice, s));
  return GENIE_OK;
}
