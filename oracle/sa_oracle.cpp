/*
 * CPU oracle for sequence similarity search by the shotgun-and-assembly
 * scheme (Sec. 5.1).  TEST INFRASTRUCTURE ONLY: only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It
 * shares no code, header or table with the CUDA path.
 *
 * What it computes, straight from the definitions:
 *   - ed(a, b): the Levenshtein distance (unit-cost insertion, deletion and
 *     substitution), by the textbook dynamic programme over the
 *     (|a|+1) x (|b|+1) table, one row at a time.
 *   - sa_grams: the ordered n-grams G(S) of Sec. 5.1.1, as keyword ids: the
 *     window S[p .. p+n-1] read as a base-sigma number g (first character
 *     most significant), its occurrence number i among the equal windows
 *     before it in S, keyword = g * R + i.  R bounds the occurrences; a
 *     larger i is reported as an error.
 *   - sa_topk_ed: the true top-k of a query under edit distance over all
 *     data sequences, ordered by (distance asc, sequence id asc).
 *
 * Returns 0 on success, 1 on an invalid argument.
 */
#include <algorithm>
#include <cstdint>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

uint32_t ed_dp(const uint8_t* a, uint32_t na, const uint8_t* b, uint32_t nb, std::vector<uint32_t>& row) {
  // row[j] = ed(a[0..i), b[0..j)) for the current i
  row.resize(nb + 1);
  for (uint32_t j = 0; j <= nb; ++j) row[j] = j;
  for (uint32_t i = 1; i <= na; ++i) {
    uint32_t diag = row[0];  // ed(a[0..i-1), b[0..j-1)) for j = 1
    row[0] = i;
    for (uint32_t j = 1; j <= nb; ++j) {
      const uint32_t up = row[j];  // ed(a[0..i-1), b[0..j))
      const uint32_t sub = diag + (a[i - 1] == b[j - 1] ? 0u : 1u);
      const uint32_t ins = row[j - 1] + 1;
      const uint32_t del = up + 1;
      row[j] = std::min(sub, std::min(ins, del));
      diag = up;
    }
  }
  return row[nb];
}

}  // namespace

extern "C" {

uint32_t oracle_ed(const uint8_t* a, uint32_t na, const uint8_t* b, uint32_t nb) {
  std::vector<uint32_t> row;
  return ed_dp(a, na, b, nb, row);
}

// ed of n (query, sequence) pairs: q[pq[2i]] against s[pq[2i+1]]
int oracle_ed_pairs(const uint32_t* q_off, const uint8_t* q_chars, const uint32_t* s_off,
                    const uint8_t* s_chars, uint64_t n, const uint32_t* pq, uint32_t* out) {
#pragma omp parallel
  {
    std::vector<uint32_t> row;
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
      const uint32_t q = pq[2 * i], s = pq[2 * i + 1];
      out[i] = ed_dp(q_chars + q_off[q], q_off[q + 1] - q_off[q], s_chars + s_off[s],
                     s_off[s + 1] - s_off[s], row);
    }
  }
  return 0;
}

// ordered n-gram keywords of n_seq sequences; kw_off[n_seq+1] is filled here
int oracle_sa_grams(uint32_t n_seq, const uint32_t* off, const uint8_t* chars, uint32_t n,
                    uint32_t sigma, uint32_t R, uint32_t* kw_off, uint32_t* kw) {
  if (n == 0 || sigma < 2 || R == 0) return 1;
  kw_off[0] = 0;
  for (uint32_t s = 0; s < n_seq; ++s) {
    const uint32_t len = off[s + 1] - off[s];
    kw_off[s + 1] = kw_off[s] + (len >= n ? len - n + 1 : 0);
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
  for (int64_t s = 0; s < (int64_t)n_seq; ++s) {
    const uint8_t* c = chars + off[s];
    const uint32_t m = kw_off[s + 1] - kw_off[s];
    std::vector<uint64_t> g(m);
    for (uint32_t p = 0; p < m; ++p) {
      uint64_t v = 0;
      for (uint32_t j = 0; j < n; ++j) {
        if (c[p + j] >= sigma) bad = 1;
        v = v * sigma + c[p + j];
      }
      g[p] = v;
    }
    for (uint32_t p = 0; p < m; ++p) {
      uint32_t occ = 0;
      for (uint32_t q = 0; q < p; ++q) occ += g[q] == g[p];
      if (occ >= R) bad = 1;
      kw[kw_off[s] + p] = (uint32_t)(g[p] * R + occ);
    }
  }
  return bad;
}

// true top-k under edit distance: (distance asc, id asc); out_* [n_q * k]
int oracle_sa_topk_ed(uint32_t n_seq, const uint32_t* s_off, const uint8_t* s_chars, uint32_t n_q,
                      const uint32_t* q_off, const uint8_t* q_chars, uint32_t k, uint32_t* out_ids,
                      uint32_t* out_ed) {
  if (k == 0) return 1;
#pragma omp parallel
  {
    std::vector<uint32_t> row;
    std::vector<std::pair<uint32_t, uint32_t>> all(n_seq);
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < (int64_t)n_q; ++q) {
      for (uint32_t s = 0; s < n_seq; ++s)
        all[s] = {ed_dp(q_chars + q_off[q], q_off[q + 1] - q_off[q], s_chars + s_off[s],
                        s_off[s + 1] - s_off[s], row),
                  s};
      const uint32_t kk = std::min<uint32_t>(k, n_seq);
      std::partial_sort(all.begin(), all.begin() + kk, all.end());
      for (uint32_t j = 0; j < k; ++j) {
        out_ids[q * k + j] = j < kk ? all[j].second : 0xFFFFFFFFu;
        out_ed[q * k + j] = j < kk ? all[j].first : 0xFFFFFFFFu;
      }
    }
  }
  return 0;
}

}  // extern "C"
