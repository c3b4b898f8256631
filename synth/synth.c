/*
 * Seeded synthetic inputs for the match-count workloads.
 *
 * This file only draws inputs: vectors and their p-stable LSH keywords (the
 * data transformation of Sec. 4.1, Eqn. (plsh), with the bucket re-hash of
 * Sec. 4.1.2 reduced to "bucket mod D"), and Zipf-distributed keyword sets
 * (a stand-in for word / n-gram sets of Sec. 5.1-5.2).  It holds none of the
 * match-count arithmetic: no counting, no top-k, no c-PQ.  Both the CUDA path
 * and the CPU oracle take its output as their input.
 *
 * Randomness: every draw is a pure function of (seed, stream, index) through
 * the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), so results do not depend on
 * the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* counter-based draw: value number `i` of stream (seed, stream, item) */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t item, uint64_t i) {
  uint64_t h = mix64(seed ^ mix64(stream * 0xD1B54A32D192ED03ull));
  h = mix64(h ^ mix64(item));
  return mix64(h + i * 0x9E3779B97F4A7C15ull);
}

/* uniform in [0,1) with 53 random bits */
static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* one standard normal from two uniforms (Box-Muller) */
static inline double normal(uint64_t seed, uint64_t stream, uint64_t item, uint64_t i) {
  double u1 = unif(draw(seed, stream, item, 2 * i));
  double u2 = unif(draw(seed, stream, item, 2 * i + 1));
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* uniform integer in [0, n) (multiply-shift on the top 32 bits; n < 2^32) */
static inline uint32_t below(uint64_t r, uint32_t n) {
  return (uint32_t)(((r >> 32) * (uint64_t)n) >> 32);
}

enum { ST_MEANS = 1, ST_PROJ = 2, ST_OFFSET = 3, ST_COMP = 4, ST_NOISE = 5,
       ST_LEN = 6, ST_KW = 7, ST_PERM = 8 };

/*
 * Gaussian-mixture vectors and their LSH keywords.
 *   means  mu_c ~ N(0, comp_sd^2 I), c < n_comp           (stream seed_model)
 *   a_i ~ N(0, I), b_i ~ U[0, width)                      (stream seed_model)
 *   x = mu_c + N(0, within_sd^2 I), c uniform, stored as float32 (seed_data)
 *   h_i(x) = floor((a_i . x + b_i) / width) in float64
 *   keyword_i(x) = i * n_buckets + (h_i(x) mod n_buckets), mod non-negative
 * out_vec (optional) receives the float32 vectors, out_kw the keywords.
 */
int synth_lsh(uint64_t seed_model, uint64_t seed_data, uint64_t n_vec, uint32_t dim,
              uint32_t n_comp, double comp_sd, double within_sd, uint32_t n_hash,
              double width, uint32_t n_buckets, float* out_vec, uint32_t* out_kw,
              uint32_t* out_comp) {
  double* mu = (double*)malloc(sizeof(double) * (size_t)n_comp * dim);
  double* a = (double*)malloc(sizeof(double) * (size_t)n_hash * dim);
  double* b = (double*)malloc(sizeof(double) * n_hash);
  if (!mu || !a || !b) { free(mu); free(a); free(b); return 1; }
  for (uint32_t c = 0; c < n_comp; ++c)
    for (uint32_t d = 0; d < dim; ++d)
      mu[(size_t)c * dim + d] = comp_sd * normal(seed_model, ST_MEANS, c, d);
  for (uint32_t i = 0; i < n_hash; ++i) {
    for (uint32_t d = 0; d < dim; ++d) a[(size_t)i * dim + d] = normal(seed_model, ST_PROJ, i, d);
    b[i] = width * unif(draw(seed_model, ST_OFFSET, i, 0));
  }
#pragma omp parallel
  {
    float* xf = (float*)malloc(sizeof(float) * dim);
    double* x = (double*)malloc(sizeof(double) * dim);
#pragma omp for schedule(static, 1024)
    for (int64_t v = 0; v < (int64_t)n_vec; ++v) {
      uint32_t c = below(draw(seed_data, ST_COMP, (uint64_t)v, 0), n_comp);
      if (out_comp) out_comp[v] = c;
      for (uint32_t d = 0; d < dim; ++d) {
        xf[d] = (float)(mu[(size_t)c * dim + d] + within_sd * normal(seed_data, ST_NOISE, (uint64_t)v, d));
        x[d] = (double)xf[d];
      }
      if (out_vec) memcpy(out_vec + (size_t)v * dim, xf, sizeof(float) * dim);
      for (uint32_t i = 0; i < n_hash; ++i) {
        const double* ai = a + (size_t)i * dim;
        double s = 0.0;
        for (uint32_t d = 0; d < dim; ++d) s += ai[d] * x[d];
        int64_t h = (int64_t)floor((s + b[i]) / width);
        int64_t bucket = h % (int64_t)n_buckets;
        if (bucket < 0) bucket += n_buckets;
        out_kw[(size_t)v * n_hash + i] = i * n_buckets + (uint32_t)bucket;
      }
    }
    free(xf);
    free(x);
  }
  free(mu); free(a); free(b);
  return 0;
}

/* set lengths, uniform in [len_lo, len_hi] */
void synth_set_lengths(uint64_t seed, uint64_t n_sets, uint32_t len_lo, uint32_t len_hi,
                       uint32_t* out_len) {
#pragma omp parallel for schedule(static, 4096)
  for (int64_t s = 0; s < (int64_t)n_sets; ++s)
    out_len[s] = len_lo + below(draw(seed, ST_LEN, (uint64_t)s, 0), len_hi - len_lo + 1);
}

/* seeded random permutation of [0, n): rank -> keyword id (Fisher-Yates) */
void synth_permutation(uint64_t seed, uint32_t n, uint32_t* out_perm) {
  for (uint32_t i = 0; i < n; ++i) out_perm[i] = i;
  for (uint32_t i = n - 1; i > 0; --i) {
    uint32_t j = below(draw(seed, ST_PERM, 0, i), i + 1);
    uint32_t t = out_perm[i]; out_perm[i] = out_perm[j]; out_perm[j] = t;
  }
}

/*
 * Zipf keyword sets.  Rank r (0-based) has probability (r+1)^-s / H.  Set number
 * t draws ranks with replacement until it holds len[t] distinct ones, and
 * stores keyword perm[rank] for each, in draw order.  off[] is the exclusive
 * prefix sum of len[] (off[n_sets] = total), out_kw has off[n_sets] entries.
 * Requires len[t] <= vocab and len[t] <= 4096.
 */
int synth_zipf_sets(uint64_t seed, uint64_t n_sets, uint32_t vocab, double s,
                    const uint32_t* perm, const uint64_t* off, uint32_t* out_kw) {
  double* cdf = (double*)malloc(sizeof(double) * vocab);
  if (!cdf) return 1;
  double acc = 0.0;
  for (uint32_t r = 0; r < vocab; ++r) { acc += pow((double)r + 1.0, -s); cdf[r] = acc; }
  for (uint32_t r = 0; r < vocab; ++r) cdf[r] /= acc;
  cdf[vocab - 1] = 1.0;
  int bad = 0;
#pragma omp parallel
  {
    uint32_t table[8192];
#pragma omp for schedule(dynamic, 256)
    for (int64_t t = 0; t < (int64_t)n_sets; ++t) {
      uint64_t begin = off[t];
      uint32_t want = (uint32_t)(off[t + 1] - begin);
      if (want > 4096 || want > vocab) { bad = 1; continue; }
      memset(table, 0xFF, sizeof(table));
      uint32_t have = 0;
      for (uint64_t i = 0; have < want; ++i) {
        double u = unif(draw(seed, ST_KW, (uint64_t)t, i));
        uint32_t lo = 0, hi = vocab - 1; /* first r with cdf[r] > u */
        while (lo < hi) {
          uint32_t mid = lo + (hi - lo) / 2;
          if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        uint32_t h = (lo * 2654435761u) & 8191u;
        int dup = 0;
        while (table[h] != 0xFFFFFFFFu) {
          if (table[h] == lo) { dup = 1; break; }
          h = (h + 1) & 8191u;
        }
        if (dup) continue;
        table[h] = lo;
        out_kw[begin + have++] = perm[lo];
      }
    }
  }
  free(cdf);
  return bad ? 2 : 0;
}

/*
 * Characters of sequences: sequence t holds off[t+1] - off[t] characters, each
 * drawn independently from the alphabet 0 .. sigma-1 with probability
 * proportional to (c+1)^-s (inverse transform over the cumulative weights).
 */
void synth_chars(uint64_t seed, uint64_t n_seqs, uint32_t sigma, double s, const uint64_t* off,
                 uint8_t* out) {
  double cdf[256];
  double total = 0.0;
  for (uint32_t c = 0; c < sigma && c < 256; ++c) {
    total += pow((double)(c + 1), -s);
    cdf[c] = total;
  }
#pragma omp parallel for schedule(static, 1024)
  for (int64_t t = 0; t < (int64_t)n_seqs; ++t) {
    for (uint64_t i = off[t]; i < off[t + 1]; ++i) {
      const double u = unif(draw(seed, ST_KW, (uint64_t)t, i - off[t])) * total;
      uint32_t lo = 0, hi = sigma - 1;
      while (lo < hi) {  /* first c with cdf[c] > u */
        const uint32_t mid = (lo + hi) >> 1;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
      }
      out[i] = (uint8_t)lo;
    }
  }
}
