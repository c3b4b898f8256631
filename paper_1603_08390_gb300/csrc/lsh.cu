// LSH keywords of points (Sec. 4.1): the transformation of a point into an
// object of m keywords, one per hash function (Sec. 4.1.2, O = [r_1(h_1(p)),
// ..., r_m(h_m(p))]), for two families:
//   - p-stable hashing (Eqn. (plsh)): h_i(p) = floor((a_i . p + b_i) / w),
//     re-hashed by taking the residue modulo D;
//   - random binning for the Laplacian kernel (Sec. 4.1.3): the cell
//     (floor((p[d] - u_i[d]) / g_i[d]))_d of a randomly shifted grid,
//     re-hashed into D buckets by an integer mixing chain over the cell's
//     coordinates (the lowbias32 finalizer of Wellons' hash-prospector; the
//     paper uses MurmurHash3).
// Keyword = i * D + bucket.  Every floating-point step is one correctly
// rounded binary32 operation in a fixed order (the dot product accumulates by
// fused multiply-adds in dimension order), so the keywords do not depend on
// how the work is split.  A block computes a tile of points x hash functions
// with both tiles staged in shared memory, dimension chunk by chunk.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kTP = 16;      // points per block tile
constexpr uint32_t kTH = 64;      // hash functions per block tile
constexpr uint32_t kDC = 64;      // dimensions staged per chunk
constexpr uint32_t kPad = kDC + 1;
constexpr uint32_t kThreads = 256;
constexpr uint32_t kPerThread = kTP * kTH / kThreads;  // 4 outputs

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ int64_t sat_i64(float t) {
  if (!(t >= -4.611686e18f)) return -(int64_t(1) << 62);
  if (t >= 4.611686e18f) return int64_t(1) << 62;
  return (int64_t)t;
}

__device__ __forceinline__ int32_t sat_i32(float c) {
  if (!(c >= -2147483648.0f)) return INT32_MIN;
  if (c >= 2147483648.0f) return INT32_MAX;
  return (int32_t)c;
}

// RBH = false: p-stable (A = a, B = b); true: random binning (A = g, B = u).
template <bool RBH>
__global__ void __launch_bounds__(kThreads) lsh_kernel(const float* __restrict__ pts, uint64_t n,
                                                       uint32_t dim, const float* __restrict__ A,
                                                       const float* __restrict__ B,
                                                       const uint32_t* __restrict__ key,
                                                       uint32_t m, float w, uint32_t D,
                                                       uint32_t* __restrict__ kw) {
  __shared__ float sp[kTP * kPad];
  __shared__ float sa[kTH * kPad];
  __shared__ float sb[RBH ? kTH * kPad : 1];
  const uint32_t tid = threadIdx.x;
  const uint32_t th = tid % kTH, tp0 = tid / kTH;  // outputs (tp0 + 4 j, th)
  const uint64_t n_ptile = (n + kTP - 1) / kTP;
  const uint32_t n_htile = (m + kTH - 1) / kTH;
  for (uint64_t tile = blockIdx.x; tile < n_ptile * n_htile; tile += gridDim.x) {
    const uint64_t p0 = (tile / n_htile) * kTP;
    const uint32_t h0 = (uint32_t)(tile % n_htile) * kTH;
    const uint32_t hi = h0 + th;
    float acc[kPerThread];
    uint32_t x[kPerThread];
#pragma unroll
    for (uint32_t j = 0; j < kPerThread; ++j) {
      acc[j] = 0.0f;
      x[j] = (RBH && hi < m) ? key[hi] : 0u;
    }
    for (uint32_t d0 = 0; d0 < dim; d0 += kDC) {
      const uint32_t dc = min(kDC, dim - d0);
      __syncthreads();
      for (uint32_t e = tid; e < kTP * kDC; e += kThreads) {
        const uint32_t r = e / kDC, c = e % kDC;
        const uint64_t p = p0 + r;
        sp[r * kPad + c] = (p < n && c < dc) ? pts[p * dim + d0 + c] : 0.0f;
      }
      for (uint32_t e = tid; e < kTH * kDC; e += kThreads) {
        const uint32_t r = e / kDC, c = e % kDC;
        const uint32_t h = h0 + r;
        const bool in = h < m && c < dc;
        sa[r * kPad + c] = in ? A[(uint64_t)h * dim + d0 + c] : 1.0f;
        if (RBH) sb[r * kPad + c] = in ? B[(uint64_t)h * dim + d0 + c] : 0.0f;
      }
      __syncthreads();
      for (uint32_t c = 0; c < dc; ++c) {
        const float a = sa[th * kPad + c];
        const float b = RBH ? sb[th * kPad + c] : 0.0f;
#pragma unroll
        for (uint32_t j = 0; j < kPerThread; ++j) {
          const float v = sp[(tp0 + 4 * j) * kPad + c];
          if (RBH) {
            const float cell = floorf(__fdiv_rn(__fsub_rn(v, b), a));
            x[j] = mix32(x[j] ^ (uint32_t)sat_i32(cell));
          } else {
            acc[j] = __fmaf_rn(a, v, acc[j]);
          }
        }
      }
    }
    if (hi < m) {
#pragma unroll
      for (uint32_t j = 0; j < kPerThread; ++j) {
        const uint64_t p = p0 + tp0 + 4 * j;
        if (p >= n) continue;
        uint32_t bucket;
        if (RBH) {
          bucket = mix32(x[j]) % D;
        } else {
          const float t = __fdiv_rn(__fadd_rn(acc[j], B[hi]), w);
          const int64_t r = sat_i64(floorf(t)) % (int64_t)D;
          bucket = (uint32_t)(r < 0 ? r + D : r);
        }
        kw[p * m + hi] = hi * D + bucket;
      }
    }
  }
}

genie_status check_lsh(const char* who, const float* pts, uint64_t n, uint32_t dim, uint32_t m,
                       uint32_t D, const uint32_t* kw) {
  if ((n && (!pts || !kw)) || dim == 0 || m == 0 || D == 0)
    return fail(GENIE_ERR_INVALID_ARG, std::string(who) + ": NULL argument or zero size");
  if ((uint64_t)m * D > 0x100000000ull)
    return fail(GENIE_ERR_INVALID_ARG, std::string(who) + ": m * D must be at most 2^32");
  return GENIE_OK;
}

uint32_t lsh_grid(uint64_t n, uint32_t m) {
  const uint64_t tiles = ((n + kTP - 1) / kTP) * ((m + kTH - 1) / kTH);
  return (uint32_t)std::min<uint64_t>(tiles, 152ull * 16);
}

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_lsh_pstable(const float* d_points, uint64_t n_points, uint32_t dim,
                                          const float* d_a, const float* d_b, uint32_t m, float w,
                                          uint32_t D, uint32_t* d_kw, genie_stream stream) {
  genie_status st = check_lsh("genie_lsh_pstable", d_points, n_points, dim, m, D, d_kw);
  if (st != GENIE_OK) return st;
  if (!d_a || !d_b || !(w > 0.0f))
    return fail(GENIE_ERR_INVALID_ARG, "genie_lsh_pstable: a, b must be given and w > 0");
  if (n_points == 0) return GENIE_OK;
  lsh_kernel<false><<<lsh_grid(n_points, m), kThreads, 0, as_stream(stream)>>>(
      d_points, n_points, dim, d_a, d_b, nullptr, m, w, D, d_kw);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}

extern "C" genie_status genie_lsh_rbh(const float* d_points, uint64_t n_points, uint32_t dim,
                                      const float* d_g, const float* d_u, const uint32_t* d_key,
                                      uint32_t m, uint32_t D, uint32_t* d_kw, genie_stream stream) {
  genie_status st = check_lsh("genie_lsh_rbh", d_points, n_points, dim, m, D, d_kw);
  if (st != GENIE_OK) return st;
  if (!d_g || !d_u || !d_key)
    return fail(GENIE_ERR_INVALID_ARG, "genie_lsh_rbh: g, u and key must be given");
  if (n_points == 0) return GENIE_OK;
  lsh_kernel<true><<<lsh_grid(n_points, m), kThreads, 0, as_stream(stream)>>>(
      d_points, n_points, dim, d_g, d_u, d_key, m, 0.0f, D, d_kw);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}
