/*
 * CPU oracle for match-count top-k search.  TEST INFRASTRUCTURE ONLY: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code, header or table with the CUDA path.
 *
 * What it computes, straight from the definitions:
 *   - Definition 2.1 (match-count model): MC(Q,O) = sum over items r of Q of
 *     C(r,O), where C(r,O) = |{e in O : e in r}|.
 *       * keyword queries: every item is one keyword, so
 *         MC(Q,O) = sum over e in O of (number of items of Q equal to e);
 *       * relational queries (Example 2.1): item (d,[lo,hi]) contains the
 *         element (d,v) of O iff lo <= v <= hi, and O has one value per d.
 *   - The ranking of Sec. 2.1 ("rank all the objects ... to obtain the
 *     top-k"): sort the objects by (MC desc, object id asc) and keep the first
 *     min(k, #{O : MC >= 1}).  The paper breaks ties at the k-th count
 *     randomly (Sec. 3.3.1, after Theorem 3.1); this build fixes the order to
 *     ascending id.  Objects with MC = 0 are never returned (the gate starts at
 *     AuditThreshold 1, Example 3.2).
 *   - Per query it also reports t_k (the k-th largest count, 0 when fewer than
 *     k objects have MC >= 1; Theorem 3.1 says MC_k = AT - 1) and the sum of
 *     MC over all objects.
 *   - cpuidx_*: a second, independent CPU computation in the manner of the
 *     CPU-Idx competitor (Sec. 6.1.2): an inverted index scanned into a dense
 *     count array, then a partial sort.
 *
 * Every routine processes queries independently (OpenMP over queries).
 * Returns 0 on success, 1 on an invalid argument.
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Ranked {
  uint32_t count;
  uint32_t id;
};

/* the total order of the output: count descending, then id ascending */
inline bool before(const Ranked& a, const Ranked& b) {
  if (a.count != b.count) return a.count > b.count;
  return a.id < b.id;
}

/* sort the objects with MC >= 1 and emit the first k of them */
void emit_topk(const uint32_t* mc, uint32_t obj_lo, uint32_t obj_hi, uint32_t k,
               uint32_t* ids, uint32_t* counts, uint32_t* n_valid, uint32_t* tk,
               uint64_t* mcsum) {
  std::vector<Ranked> all;
  uint64_t sum = 0;
  for (uint32_t o = obj_lo; o < obj_hi; ++o) {
    sum += mc[o];
    if (mc[o] >= 1) all.push_back({mc[o], o});
  }
  std::sort(all.begin(), all.end(), before);
  uint32_t n = (uint32_t)std::min<size_t>(k, all.size());
  for (uint32_t j = 0; j < k; ++j) {
    ids[j] = j < n ? all[j].id : 0xFFFFFFFFu;
    counts[j] = j < n ? all[j].count : 0u;
  }
  *n_valid = n;
  *tk = all.size() >= k ? all[k - 1].count : 0u;
  *mcsum = sum;
}

int set_threads(int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
  return omp_get_max_threads();
#else
  (void)n_threads;
  return 1;
#endif
}

}  // namespace

extern "C" {

int oracle_max_threads(int n_threads) { return set_threads(n_threads); }

/*
 * Keyword objects (CSR obj_off[n_obj+1], obj_kw) and keyword-multiset queries
 * (CSR q_off[n_q+1], q_kw).  Only objects with id in [obj_lo, obj_hi) are
 * ranked (the whole set when obj_lo = 0 and obj_hi = n_obj).  Query q writes
 * k_arr[q] slots at ids[q*stride], counts[q*stride].
 */
int oracle_topk_keywords(uint32_t n_obj, const uint32_t* obj_off, const uint32_t* obj_kw,
                         uint32_t vocab, uint32_t n_q, const uint32_t* q_off,
                         const uint32_t* q_kw, const uint32_t* k_arr, uint32_t stride,
                         uint32_t obj_lo, uint32_t obj_hi, uint32_t* ids, uint32_t* counts,
                         uint32_t* n_valid, uint32_t* tk, uint64_t* mcsum, int n_threads) {
  if (obj_lo > obj_hi || obj_hi > n_obj) return 1;
  for (uint32_t q = 0; q < n_q; ++q) {
    if (k_arr[q] == 0 || k_arr[q] > stride) return 1;
    for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i)
      if (q_kw[i] >= vocab) return 1;
  }
  for (uint64_t i = 0; i < obj_off[n_obj]; ++i)
    if (obj_kw[i] >= vocab) return 1;
  set_threads(n_threads);
#pragma omp parallel
  {
    std::vector<uint32_t> mult(vocab, 0u);  /* items of Q equal to each keyword */
    std::vector<uint32_t> mc(n_obj, 0u);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qq = 0; qq < (int64_t)n_q; ++qq) {
      uint32_t q = (uint32_t)qq;
      for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i) mult[q_kw[i]] += 1;
      for (uint32_t o = obj_lo; o < obj_hi; ++o) {
        uint32_t c = 0;
        for (uint32_t e = obj_off[o]; e < obj_off[o + 1]; ++e) c += mult[obj_kw[e]];
        mc[o] = c;
      }
      emit_topk(mc.data(), obj_lo, obj_hi, k_arr[q], ids + (size_t)q * stride,
                counts + (size_t)q * stride, n_valid + q, tk + q, mcsum + q);
      for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i) mult[q_kw[i]] = 0;
    }
  }
  return 0;
}

/*
 * Relational objects values[n_obj * n_dim] and range queries: query q has
 * items item_off[q] .. item_off[q+1]-1, item i being (item_dim[i],
 * [item_lo[i], item_hi[i]]).  C(item, O) = 1 iff lo <= O[d] <= hi.
 */
int oracle_topk_relational(uint32_t n_obj, uint32_t n_dim, const uint32_t* values, uint32_t n_q,
                           const uint32_t* item_off, const uint32_t* item_dim,
                           const int32_t* item_lo, const int32_t* item_hi,
                           const uint32_t* k_arr, uint32_t stride, uint32_t obj_lo,
                           uint32_t obj_hi, uint32_t* ids, uint32_t* counts, uint32_t* n_valid,
                           uint32_t* tk, uint64_t* mcsum, int n_threads) {
  if (obj_lo > obj_hi || obj_hi > n_obj) return 1;
  for (uint32_t q = 0; q < n_q; ++q) {
    if (k_arr[q] == 0 || k_arr[q] > stride) return 1;
    for (uint32_t i = item_off[q]; i < item_off[q + 1]; ++i)
      if (item_dim[i] >= n_dim) return 1;
  }
  set_threads(n_threads);
#pragma omp parallel
  {
    std::vector<uint32_t> mc(n_obj, 0u);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qq = 0; qq < (int64_t)n_q; ++qq) {
      uint32_t q = (uint32_t)qq;
      for (uint32_t o = obj_lo; o < obj_hi; ++o) {
        uint32_t c = 0;
        for (uint32_t i = item_off[q]; i < item_off[q + 1]; ++i) {
          int64_t v = values[(size_t)o * n_dim + item_dim[i]];
          if ((int64_t)item_lo[i] <= v && v <= (int64_t)item_hi[i]) c += 1;
        }
        mc[o] = c;
      }
      emit_topk(mc.data(), obj_lo, obj_hi, k_arr[q], ids + (size_t)q * stride,
                counts + (size_t)q * stride, n_valid + q, tk + q, mcsum + q);
    }
  }
  return 0;
}

/* Full match-count matrix mc[q * n_obj + o] for keyword queries (small cases). */
int oracle_counts_keywords(uint32_t n_obj, const uint32_t* obj_off, const uint32_t* obj_kw,
                           uint32_t vocab, uint32_t n_q, const uint32_t* q_off,
                           const uint32_t* q_kw, uint32_t* mc) {
  std::vector<uint32_t> mult(vocab, 0u);
  for (uint32_t q = 0; q < n_q; ++q) {
    for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i) {
      if (q_kw[i] >= vocab) return 1;
      mult[q_kw[i]] += 1;
    }
    for (uint32_t o = 0; o < n_obj; ++o) {
      uint32_t c = 0;
      for (uint32_t e = obj_off[o]; e < obj_off[o + 1]; ++e) {
        if (obj_kw[e] >= vocab) return 1;
        c += mult[obj_kw[e]];
      }
      mc[(size_t)q * n_obj + o] = c;
    }
    for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i) mult[q_kw[i]] = 0;
  }
  return 0;
}

/*
 * CPU-Idx (Sec. 6.1.2): build an inverted index (keyword -> ascending object
 * ids) by counting sort, scan the lists of each query keyword into a dense
 * count array, then std::partial_sort the touched objects.
 */
int cpuidx_topk_keywords(uint32_t n_obj, const uint32_t* obj_off, const uint32_t* obj_kw,
                         uint32_t vocab, uint32_t n_q, const uint32_t* q_off,
                         const uint32_t* q_kw, const uint32_t* k_arr, uint32_t stride,
                         uint32_t* ids, uint32_t* counts, uint32_t* n_valid, uint32_t* tk,
                         uint64_t* mcsum, int n_threads) {
  const uint64_t nnz = obj_off[n_obj];
  std::vector<uint64_t> head(vocab + 1, 0);
  for (uint64_t i = 0; i < nnz; ++i) {
    if (obj_kw[i] >= vocab) return 1;
    head[obj_kw[i] + 1] += 1;
  }
  for (uint32_t v = 0; v < vocab; ++v) head[v + 1] += head[v];
  std::vector<uint32_t> lists(nnz);
  {
    std::vector<uint64_t> fill(head.begin(), head.end() - 1);
    for (uint32_t o = 0; o < n_obj; ++o)
      for (uint32_t e = obj_off[o]; e < obj_off[o + 1]; ++e) lists[fill[obj_kw[e]]++] = o;
  }
  for (uint32_t q = 0; q < n_q; ++q) {
    if (k_arr[q] == 0 || k_arr[q] > stride) return 1;
    for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i)
      if (q_kw[i] >= vocab) return 1;
  }
  set_threads(n_threads);
#pragma omp parallel
  {
    std::vector<uint32_t> cnt(n_obj, 0u);
    std::vector<uint32_t> touched;
#pragma omp for schedule(dynamic, 1)
    for (int64_t qq = 0; qq < (int64_t)n_q; ++qq) {
      uint32_t q = (uint32_t)qq;
      touched.clear();
      uint64_t sum = 0;
      for (uint32_t i = q_off[q]; i < q_off[q + 1]; ++i) {
        uint32_t kw = q_kw[i];
        for (uint64_t p = head[kw]; p < head[kw + 1]; ++p) {
          uint32_t o = lists[p];
          if (cnt[o]++ == 0) touched.push_back(o);
          sum += 1;
        }
      }
      std::vector<Ranked> cand;
      cand.reserve(touched.size());
      for (uint32_t o : touched) cand.push_back({cnt[o], o});
      uint32_t k = k_arr[q];
      uint32_t n = (uint32_t)std::min<size_t>(k, cand.size());
      std::partial_sort(cand.begin(), cand.begin() + n, cand.end(), before);
      uint32_t* oi = ids + (size_t)q * stride;
      uint32_t* oc = counts + (size_t)q * stride;
      for (uint32_t j = 0; j < k; ++j) {
        oi[j] = j < n ? cand[j].id : 0xFFFFFFFFu;
        oc[j] = j < n ? cand[j].count : 0u;
      }
      n_valid[q] = n;
      tk[q] = cand.size() >= k ? cand[k - 1].count : 0u;
      mcsum[q] = sum;
      for (uint32_t o : touched) cnt[o] = 0;
    }
  }
  return 0;
}

}  // extern "C"
