/*
 * CPU oracle for LSH keyword generation (Sec. 4.1).  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or table with the CUDA path.
 * Built with -ffp-contract=off: every floating-point operation below is one
 * correctly rounded IEEE binary32 operation, in the order written.
 *
 * Point p (dim floats) and hash function i (of m) give keyword i * D + b:
 *   - p-stable (Eqn. (plsh)): s = a_i . p, accumulated as
 *     s = fma(a_i[d], p[d], s) for d = 0, 1, ..., dim - 1 from s = 0; then
 *     h = floor((s + b_i) / w) and b = h mod D (the non-negative residue).
 *   - random binning (the Laplacian-kernel case study, Sec. 4.1.3): the grid
 *     cell of p, c_d = floor((p[d] - u_i[d]) / g_i[d]) for every d; the
 *     re-hash of Sec. 4.1.2 maps the cell to a bucket: starting from
 *     x = key_i, for each d, x = mix(x ^ (uint32) c_d); b = mix(x) mod D, with
 *     mix(x) = the 32-bit integer finalizer "lowbias32" published with
 *     Wellons' hash-prospector: x ^= x >> 16; x *= 0x7feb352d; x ^= x >> 15;
 *     x *= 0x846ca68b; x ^= x >> 16.
 *   Float-to-integer conversions saturate: h to [-2^62, 2^62], c_d to the
 *   int32 range.
 * Returns 0 on success, 1 on an invalid argument.
 */
#include <climits>
#include <cmath>
#include <cstdint>

namespace {

uint32_t mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

int64_t to_i64(float t) {
  if (!(t >= -4.611686e18f)) return -(int64_t(1) << 62);
  if (t >= 4.611686e18f) return int64_t(1) << 62;
  return (int64_t)t;
}

int32_t to_i32(float c) {
  if (!(c >= -2147483648.0f)) return INT32_MIN;
  if (c >= 2147483648.0f) return INT32_MAX;
  return (int32_t)c;
}

uint32_t residue(int64_t h, uint32_t D) {
  int64_t r = h % (int64_t)D;
  return (uint32_t)(r < 0 ? r + D : r);
}

}  // namespace

extern "C" {

int oracle_lsh_pstable(uint64_t n, uint32_t dim, const float* pts, uint32_t m, const float* a,
                       const float* b, float w, uint32_t D, uint32_t* kw) {
  if (dim == 0 || m == 0 || D == 0 || !(w > 0.0f)) return 1;
#pragma omp parallel for schedule(static, 256)
  for (int64_t o = 0; o < (int64_t)n; ++o) {
    const float* p = pts + (uint64_t)o * dim;
    for (uint32_t i = 0; i < m; ++i) {
      const float* ai = a + (uint64_t)i * dim;
      float s = 0.0f;
      for (uint32_t d = 0; d < dim; ++d) s = std::fma(ai[d], p[d], s);
      const float t = (s + b[i]) / w;
      kw[(uint64_t)o * m + i] = i * D + residue(to_i64(std::floor(t)), D);
    }
  }
  return 0;
}

int oracle_lsh_rbh(uint64_t n, uint32_t dim, const float* pts, uint32_t m, const float* g,
                   const float* u, const uint32_t* key, uint32_t D, uint32_t* kw) {
  if (dim == 0 || m == 0 || D == 0) return 1;
#pragma omp parallel for schedule(static, 256)
  for (int64_t o = 0; o < (int64_t)n; ++o) {
    const float* p = pts + (uint64_t)o * dim;
    for (uint32_t i = 0; i < m; ++i) {
      uint32_t x = key[i];
      for (uint32_t d = 0; d < dim; ++d) {
        const float c = std::floor((p[d] - u[(uint64_t)i * dim + d]) / g[(uint64_t)i * dim + d]);
        x = mix(x ^ (uint32_t)to_i32(c));
      }
      kw[(uint64_t)o * m + i] = i * D + mix(x) % D;
    }
  }
  return 0;
}

}  // extern "C"
