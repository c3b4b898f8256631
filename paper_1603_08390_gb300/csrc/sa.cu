// Sequence similarity search by the shotgun-and-assembly scheme (Sec. 5.1).
//
// Shotgun: a sequence S becomes its set of ordered n-grams G(S), the pairs
// (n-gram, i) where i numbers the equal windows before it in S (Sec. 5.1.1).
// Here a window is read as a base-sigma number g (first character most
// significant) and (g, i) becomes the keyword g * R + i; R bounds the
// occurrences of one n-gram in one sequence.  The data sequences' keyword
// sets are indexed by genie_build_index and the queries' by
// genie_make_queries; the match count of a query and a sequence is then
// |G(Q) n G(S)|, the number of shared n-grams counted with multiplicity
// (Lemma 5.1).
//
// Assembly: a search returns the K sequences with the largest counts, and the
// verification of Algorithm 2 computes edit distances in count order until
// the n-gram bound of Theorem 5.1 shows that no later candidate can be
// closer.  genie_sa_verify computes the edit distances of all K candidates
// of a query in parallel (one thread per candidate, the bit-parallel
// Levenshtein recurrence of Myers (JACM 1999) in 64-bit blocks), then one
// thread runs the algorithm over them in count order, keeping the k best
// (distance asc, candidate order), and tests the certificate of Theorem 5.2.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kMaxQueryLen = 512;   // query characters (8 blocks of 64)
constexpr uint32_t kMaxBlocks = kMaxQueryLen / 64;
constexpr uint32_t kVerifyThreads = 256;

enum SaFlag { kBadChar = 0, kTooManyRepeats = 1, kNumSaFlags = 2 };

__global__ void gram_count_kernel(const uint32_t* __restrict__ off, uint32_t n_seqs, uint32_t n,
                                  uint32_t* __restrict__ cnt) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_seqs; s += gridDim.x * blockDim.x) {
    const uint32_t len = off[s + 1] - off[s];
    cnt[s] = len >= n ? len - n + 1 : 0;
  }
}

// One warp per sequence: the window codes go to `code`, then each window's
// occurrence number is the count of equal codes before it.
__global__ void gram_kernel(const uint32_t* __restrict__ off, const uint8_t* __restrict__ chars,
                            uint32_t n_seqs, uint32_t n, uint32_t sigma, uint32_t R,
                            const uint32_t* __restrict__ kw_off, uint32_t* __restrict__ code,
                            uint32_t* __restrict__ kw, uint32_t* __restrict__ flags) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_seqs; s += warps) {
    const uint8_t* c = chars + off[s];
    const uint32_t base = kw_off[s], m = kw_off[s + 1] - base;
    bool bad = false;
    for (uint32_t p = lane; p < m; p += 32) {
      uint32_t g = 0;
      for (uint32_t j = 0; j < n; ++j) {
        const uint32_t x = c[p + j];
        bad |= x >= sigma;
        g = g * sigma + x;
      }
      code[base + p] = g;
    }
    __syncwarp();
    bool over = false;
    for (uint32_t p = lane; p < m; p += 32) {
      const uint32_t g = code[base + p];
      uint32_t occ = 0;
      for (uint32_t q = 0; q < p; ++q) occ += code[base + q] == g;
      over |= occ >= R;
      kw[base + p] = g * R + occ;
    }
    if (bad) atomicOr(&flags[kBadChar], 1u);
    if (over) atomicOr(&flags[kTooManyRepeats], 1u);
    __syncwarp();
  }
}

// Levenshtein distance between the query (W blocks of its character masks
// peq[c * kMaxBlocks + b], length m) and the text t[0 .. len), by the
// bit-parallel recurrence over the columns of the dynamic-programming table:
// per block, bit i of Pv / Mv marks a vertical difference of +1 / -1 between
// rows i and i - 1 of the current column; a column step propagates the
// horizontal difference of the block's top row (hin) to its bottom (hout).
// The top row of the table is 0, 1, 2, ..., so every column enters the first
// block with hin = +1.
// W: blocks the routine can hold (1, 2, 4 or 8); only the first
// ceil(m / 64) are used, and the score is read at row m - 1 of the last.
template <uint32_t W>
__device__ uint32_t myers_ed(const unsigned long long* __restrict__ peq, uint32_t m,
                             const uint8_t* __restrict__ t, uint32_t len) {
  unsigned long long Pv[W], Mv[W];
#pragma unroll
  for (uint32_t b = 0; b < W; ++b) {
    Pv[b] = ~0ull;
    Mv[b] = 0ull;
  }
  const uint32_t nb = (m + 63) / 64;
  const unsigned long long last = 1ull << ((m - 1) & 63);
  int score = (int)m;
  for (uint32_t j = 0; j < len; ++j) {
    const unsigned long long* eq = peq + (uint32_t)t[j] * kMaxBlocks;
    int hin = 1;
#pragma unroll
    for (uint32_t b = 0; b < W; ++b) {
      if (b >= nb) break;
      unsigned long long Eq = eq[b];
      const unsigned long long Xv = Eq | Mv[b];
      if (hin < 0) Eq |= 1ull;
      const unsigned long long Xh = (((Eq & Pv[b]) + Pv[b]) ^ Pv[b]) | Eq;
      unsigned long long Ph = Mv[b] | ~(Xh | Pv[b]);
      unsigned long long Mh = Pv[b] & Xh;
      const unsigned long long top = b + 1 == nb ? last : (1ull << 63);
      const int hout = (Ph & top) ? 1 : ((Mh & top) ? -1 : 0);
      Ph <<= 1;
      Mh <<= 1;
      if (hin < 0) Mh |= 1ull;
      else if (hin > 0) Ph |= 1ull;
      Pv[b] = Mh | ~(Xv | Ph);
      Mv[b] = Ph & Xv;
      hin = hout;
    }
    score += hin;
  }
  return (uint32_t)score;
}

struct VerifyArgs {
  const uint32_t* q_off;
  const uint8_t* q_chars;
  const uint32_t* s_off;
  const uint8_t* s_chars;
  const uint32_t* cand_ids;     // [Q][K], count order
  const uint32_t* cand_counts;  // [Q][K]
  const uint32_t* cand_n;       // [Q]
  uint32_t n_queries, K, k, n;
  uint32_t* out_ids;            // [Q][k]
  uint32_t* out_ed;             // [Q][k]
  uint32_t* out_n;              // [Q]
  uint32_t* certified;          // [Q]
  uint32_t* examined;           // [Q]
};

__global__ void __launch_bounds__(kVerifyThreads) verify_kernel(const VerifyArgs A) {
  __shared__ unsigned long long peq[256 * kMaxBlocks];
  extern __shared__ uint32_t dyn[];
  uint32_t* ed = dyn;               // [K]
  uint32_t* best_ed = dyn + A.K;    // [k]
  uint32_t* best_j = best_ed + A.k; // [k]
  for (uint32_t q = blockIdx.x; q < A.n_queries; q += gridDim.x) {
    const uint32_t m = A.q_off[q + 1] - A.q_off[q];
    const uint8_t* qc = A.q_chars + A.q_off[q];
    // a query longer than the character masks hold gets no result
    const uint32_t nc = m <= kMaxQueryLen ? min(A.cand_n[q], A.K) : 0u;
    const uint32_t W = (m + 63) / 64;
    for (uint32_t i = threadIdx.x; i < 256 * kMaxBlocks; i += blockDim.x) peq[i] = 0ull;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m && i < kMaxQueryLen; i += blockDim.x)
      atomicOr(&peq[(uint32_t)qc[i] * kMaxBlocks + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
    const uint32_t* ids = A.cand_ids + (uint64_t)q * A.K;
    for (uint32_t j = threadIdx.x; j < nc; j += blockDim.x) {
      const uint32_t id = ids[j];
      const uint8_t* t = A.s_chars + A.s_off[id];
      const uint32_t len = A.s_off[id + 1] - A.s_off[id];
      uint32_t d;
      if (m == 0) d = len;
      else if (W <= 1) d = myers_ed<1>(peq, m, t, len);
      else if (W <= 2) d = myers_ed<2>(peq, m, t, len);
      else if (W <= 4) d = myers_ed<4>(peq, m, t, len);
      else d = myers_ed<8>(peq, m, t, len);
      ed[j] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // Algorithm 2 over the candidates in count order, keeping the k best
      const uint32_t* cnt = A.cand_counts + (uint64_t)q * A.K;
      const int64_t qlen = (int64_t)m, n = (int64_t)A.n;
      uint32_t nb = 0, examined = 0;
      for (uint32_t j = 0; j < nc; ++j) {
        if (nb == A.k) {
          const int64_t tau = best_ed[nb - 1];
          const int64_t theta = qlen - n + 1 - n * (tau - 1);
          if (theta > (int64_t)cnt[j]) break;  // no later candidate is closer (Theorem 5.1)
          const uint32_t id = ids[j];
          const int64_t slen = A.s_off[id + 1] - A.s_off[id];
          if ((qlen > slen ? qlen - slen : slen - qlen) > tau) continue;  // length filter
        }
        ++examined;
        const uint32_t e = ed[j];
        if (nb == A.k && e >= best_ed[nb - 1]) continue;
        uint32_t p = nb < A.k ? nb++ : nb - 1;  // insert (e, j): ties keep count order
        while (p > 0 && best_ed[p - 1] > e) {
          best_ed[p] = best_ed[p - 1];
          best_j[p] = best_j[p - 1];
          --p;
        }
        best_ed[p] = e;
        best_j[p] = j;
      }
      uint32_t* oid = A.out_ids + (uint64_t)q * A.k;
      uint32_t* oed = A.out_ed + (uint64_t)q * A.k;
      for (uint32_t i = 0; i < A.k; ++i) {
        oid[i] = i < nb ? ids[best_j[i]] : 0xFFFFFFFFu;
        oed[i] = i < nb ? best_ed[i] : 0xFFFFFFFFu;
      }
      // Theorem 5.2: c_K is the K-th candidate's count (0 when fewer than K
      // sequences share an n-gram with the query)
      const int64_t cK = nc >= A.K ? (int64_t)cnt[A.K - 1] : 0;
      const bool cert = nb == A.k && cK < qlen - n + 1 - (int64_t)best_ed[A.k - 1] * n;
      A.out_n[q] = nb;
      A.certified[q] = cert ? 1u : 0u;
      A.examined[q] = examined;
    }
    __syncthreads();
  }
}

uint32_t grid_for(uint64_t n, uint32_t threads) {
  return (uint32_t)std::min<uint64_t>((n + threads - 1) / threads, 152ull * 64);
}

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_sa_grams(const uint32_t* d_off, const uint8_t* d_chars,
                                       uint32_t n_seqs, uint32_t n, uint32_t sigma, uint32_t R,
                                       uint32_t* d_kw_off, uint32_t* d_kw, uint64_t kw_capacity,
                                       uint64_t* total, genie_stream stream) {
  if (!d_off || !d_kw_off || !total || (n_seqs && !d_chars))
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: NULL argument");
  if (n == 0 || sigma < 2 || sigma > 256 || R == 0)
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: need n >= 1, 2 <= sigma <= 256, R >= 1");
  uint64_t space = R;  // keyword ids g * R + i < sigma^n * R
  for (uint32_t j = 0; j < n; ++j) {
    space *= sigma;
    if (space > 0x80000000ull)
      return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: sigma^n * R must be at most 2^31");
  }
  cudaStream_t s = as_stream(stream);
  uint32_t tot = 0;
  if (n_seqs) {
    gram_count_kernel<<<grid_for(n_seqs, 256), 256, 0, s>>>(d_off, n_seqs, n, d_kw_off);
    GENIE_CUDA_TRY(cudaGetLastError());
    launch_exclusive_scan(d_kw_off, n_seqs, d_kw_off + n_seqs, s);
    GENIE_CUDA_TRY(cudaGetLastError());
    GENIE_CUDA_TRY(cudaMemcpyAsync(&tot, d_kw_off + n_seqs, 4, cudaMemcpyDeviceToHost, s));
    GENIE_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    GENIE_CUDA_TRY(cudaMemsetAsync(d_kw_off, 0, 4, s));
  }
  *total = tot;
  if (tot > kw_capacity)
    return fail(GENIE_ERR_CAPACITY, "genie_sa_grams: d_kw holds fewer entries than the n-grams");
  if (tot == 0) return GENIE_OK;
  if (!d_kw) return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: d_kw is NULL");
  uint32_t* code = nullptr;
  GENIE_CUDA_TRY(cudaMallocAsync((void**)&code, (uint64_t)tot * 4 + 64, s));
  uint32_t* flags = code + tot;  // kNumSaFlags words after the codes (64 bytes reserved)
  cudaError_t e = cudaMemsetAsync(flags, 0, 64, s);
  if (e == cudaSuccess) {
    gram_kernel<<<grid_for((uint64_t)n_seqs * 32, 256), 256, 0, s>>>(d_off, d_chars, n_seqs, n, sigma,
                                                                     R, d_kw_off, code, d_kw, flags);
    e = cudaGetLastError();
  }
  uint32_t h[kNumSaFlags] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(code, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "genie_sa_grams");
  if (h[kBadChar]) return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: a character is >= sigma");
  if (h[kTooManyRepeats])
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_grams: an n-gram occurs R or more times in a sequence");
  return GENIE_OK;
}

extern "C" genie_status genie_sa_verify(const uint32_t* d_q_off, const uint8_t* d_q_chars,
                                        uint32_t n_queries, const uint32_t* d_s_off,
                                        const uint8_t* d_s_chars, const uint32_t* d_cand_ids,
                                        const uint32_t* d_cand_counts, const uint32_t* d_cand_n,
                                        uint32_t K, uint32_t k, uint32_t n, uint32_t max_query_len,
                                        uint32_t* d_ids, uint32_t* d_ed, uint32_t* d_n_out,
                                        uint32_t* d_certified, uint32_t* d_examined,
                                        genie_stream stream) {
  if (!d_q_off || !d_s_off || !d_cand_ids || !d_cand_counts || !d_cand_n || !d_ids || !d_ed ||
      !d_n_out || !d_certified || !d_examined)
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_verify: NULL argument");
  if (K == 0 || K > GENIE_MAX_K || k == 0 || k > K || n == 0)
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_verify: need 1 <= k <= K <= GENIE_MAX_K and n >= 1");
  if (max_query_len > kMaxQueryLen)
    return fail(GENIE_ERR_INVALID_ARG, "genie_sa_verify: queries longer than 512 characters");
  if (n_queries == 0) return GENIE_OK;
  VerifyArgs a{d_q_off, d_q_chars, d_s_off, d_s_chars, d_cand_ids, d_cand_counts, d_cand_n,
               n_queries, K, k, n, d_ids, d_ed, d_n_out, d_certified, d_examined};
  cudaStream_t s = as_stream(stream);
  const size_t smem = ((size_t)K + 2 * (size_t)k) * 4;
  verify_kernel<<<std::min<uint32_t>(n_queries, 152u * 8u), kVerifyThreads, smem, s>>>(a);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}
