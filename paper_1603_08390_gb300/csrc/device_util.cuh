// Small block-wide building blocks used by several kernels.
#pragma once

#include <cstdint>

namespace genie {
namespace dev {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t warp_id() { return threadIdx.x >> 5; }

// Inclusive prefix sum across a warp.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(0xFFFFFFFFu, v, d);
    if ((int)lane_id() >= d) v += o;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
  return v;
}

// Exclusive prefix sum over the block; `scratch` holds 33 T in shared memory.
// Every thread of the block must call it.  Returns the thread's exclusive
// prefix and writes the block total to *total.
template <typename T>
__device__ T block_exclusive_scan(T v, T* scratch, T* total) {
  const uint32_t nwarps = (blockDim.x + 31) >> 5;
  T inc = warp_inclusive_scan(v);
  __syncthreads();  // scratch may still be read by a previous call
  if (lane_id() == 31 || threadIdx.x == blockDim.x - 1) scratch[warp_id()] = inc;
  __syncthreads();
  if (warp_id() == 0) {
    T w = lane_id() < nwarps ? scratch[lane_id()] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane_id() < nwarps) scratch[lane_id()] = wi - w;
    if (lane_id() == 31) scratch[32] = wi;
  }
  __syncthreads();
  *total = scratch[32];
  return scratch[warp_id()] + inc - v;
}

template <typename T>
__device__ T block_sum(T v, T* scratch) {
  T total;
  block_exclusive_scan(v, scratch, &total);
  return total;
}

// Bitonic sort of n (a power of two) 64-bit keys in shared memory into
// DESCENDING order.  All threads of the block must call it.
__device__ inline void bitonic_sort_desc(unsigned long long* s, uint32_t n) {
  for (uint32_t size = 2; size <= n; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        uint32_t pos = 2 * i - (i & (stride - 1));
        uint32_t partner = pos + stride;
        bool desc = (pos & size) == 0;
        unsigned long long a = s[pos], b = s[partner];
        if ((a < b) == desc) {
          s[pos] = b;
          s[partner] = a;
        }
      }
      __syncthreads();
    }
  }
}

__host__ __device__ inline uint32_t next_pow2(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Result key of one (object, count): ordering keys descending gives count
// descending, then object id ascending.  Key 0 means "no object".
__device__ __forceinline__ unsigned long long result_key(uint32_t count, uint32_t id) {
  return ((unsigned long long)count << 32) | (unsigned long long)(0xFFFFFFFFu - id);
}
__device__ __forceinline__ uint32_t key_count(unsigned long long key) { return (uint32_t)(key >> 32); }
__device__ __forceinline__ uint32_t key_id(unsigned long long key) {
  return 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull);
}

}  // namespace dev
}  // namespace genie
