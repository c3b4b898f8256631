// Device code of the search: the per-(query, object range) c-PQ work item
// and the per-query merge, shared by the one-launch-per-batch kernels
// (search.cu) and the persistent batched kernel (batch.cu).  The design and
// the readings of the paper it relies on are described at the top of
// search.cu.
#pragma once

#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kKwBatch = 512;  // query keywords staged in shared memory per round

struct ScanArgs {
  const uint64_t* kw_off;
  const uint32_t* post_ids;
  const uint32_t* chunk_pos;
  uint32_t n_chunks;
  uint32_t chunk_shift;
  uint32_t n_objects;
  const uint32_t* q_off;
  const uint32_t* q_kw;
  const uint32_t* bound;
  const uint32_t* q_sel;  // NULL: block query index = query id
  uint32_t n_sel;
  uint32_t k;             // row stride of the candidate lists
  const uint32_t* k_arr;  // per-query k or NULL
  const uint32_t* seed;   // per-query AuditThreshold seed or NULL
  uint32_t block_shift;
  uint32_t chunks_per_block;
  uint32_t n_groups;
  uint32_t ht_slots;
  uint32_t za_len;
  unsigned long long* cand;  // [n_sel][n_groups][k]
  uint32_t* chunk_at;        // [n_sel][n_groups] or NULL
  unsigned long long* stats;
  // [n_sel] or NULL: the largest k-th count of the query's ranges finished so
  // far.  The k-th count of a range is at most the query's k-th count (the
  // k-th largest of a subset never exceeds that of the whole set), so a range
  // may start its AuditThreshold there without losing any top-k object.
  uint32_t* at_hint;
  // [n_sel][hint_stride] or NULL: per query, how many objects its finished
  // ranges reported at each count.  They are distinct objects with exact
  // counts, so the k-th largest count among them is also at most the query's
  // k-th count; it replaces the single largest range k-th count in at_hint.
  uint32_t* hint_hist;
  uint32_t hint_stride;
  // 1: count only, then select from the Bitmap Counter (the Gate and the
  // hash table stay idle) -- the GEN-SPQ-style ablation of Sec. 6.1.2
  uint32_t no_gate;
  // dense keywords (NULL: none): dense_slot[kw] = the keyword's object bitmap
  // or kNoDense; bitmap s = dense_bits[s * map_words ..]
  const uint32_t* dense_slot;
  const uint32_t* dense_bits;
  uint64_t map_words;
};

constexpr uint32_t kMaxProbe = 32;   // hash-table probes before an insert gives up
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kTilePrePad = 36;  // tile prefix sums: sentinels read by a warp-wide step
// the tile prefix sums' room holds 255 bitmap pointers (8-byte aligned) in the dense phase
static_assert((kKwBatch + kTilePrePad) * 4 >= 255 * 8 + 4, "room for the dense pointers");
constexpr uint32_t kRun = 8;         // consecutive tiles a warp claims as one run

size_t scan_smem_bytes(uint32_t log2w, uint32_t block_shift, uint32_t ht_slots, uint32_t za_len,
                       uint32_t k) {
  size_t words = ((size_t)1 << block_shift) >> (5 - log2w);
  size_t present = ((size_t)1 << block_shift) >> 5;
  return words * 4 + present * 4 + (size_t)ht_slots * 4 + (size_t)dev::next_pow2(k) * 8 +
         (size_t)za_len * 4 + (3 * kKwBatch + kTilePrePad) * 4;
}

__device__ __forceinline__ uint32_t vld(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// Counter lanes addressed by the object id itself.  A range starts at a
// multiple of the lanes per word, so the word of object id is
// byte_off(id) - byte_off(range start) bytes into the range's counters, and
// the lane inside the word is the low bits of the id.  inc: the word-sized
// increment of that lane; sel: a selector for the lane, pick: the lane's value
// in a counter word given its selector (0 for a zero word whatever the
// selector).  kHigh: the top bit of every lane; kOnes: 1 in every lane.
template <int LOG2W>
struct Lane;
template <>
struct Lane<4> {  // 16-bit counters, two per word
  static constexpr uint32_t kHigh = 0x80008000u, kOnes = 0x00010001u;
  static __device__ __forceinline__ uint32_t byte_off(uint32_t id) { return (id & ~1u) << 1; }
  static __device__ __forceinline__ uint32_t inc(uint32_t id) { return (id & 1u) * 0xFFFFu + 1u; }
  static __device__ __forceinline__ uint32_t sel(uint32_t id) { return 0x4410u + (id & 1u) * 0x22u; }
  static __device__ __forceinline__ uint32_t pick(uint32_t w, uint32_t s) {
    return __byte_perm(w, 0u, s);  // bytes 2l, 2l+1, then zeros
  }
};
template <>
struct Lane<3> {  // 8-bit counters, four per word
  static constexpr uint32_t kHigh = 0x80808080u, kOnes = 0x01010101u;
  static __device__ __forceinline__ uint32_t byte_off(uint32_t id) { return id & ~3u; }
  static __device__ __forceinline__ uint32_t inc(uint32_t id) { return 1u << ((id & 3u) << 3); }
  static __device__ __forceinline__ uint32_t sel(uint32_t id) { return 0x4440u | (id & 3u); }
  static __device__ __forceinline__ uint32_t pick(uint32_t w, uint32_t s) {
    return __byte_perm(w, 0u, s);  // byte l, then zeros
  }
};
template <>
struct Lane<2> {  // 4-bit counters, eight per word
  static constexpr uint32_t kHigh = 0x88888888u, kOnes = 0x11111111u;
  static __device__ __forceinline__ uint32_t byte_off(uint32_t id) { return (id >> 1) & ~3u; }
  static __device__ __forceinline__ uint32_t inc(uint32_t id) { return 1u << ((id & 7u) << 2); }
  static __device__ __forceinline__ uint32_t sel(uint32_t id) { return (id & 7u) << 2; }
  static __device__ __forceinline__ uint32_t pick(uint32_t w, uint32_t s) { return (w >> s) & 0xFu; }
};

// atomicAdd on a 32-bit shared-memory address, returning the old word
__device__ __forceinline__ uint32_t atom_add_shared(uint32_t saddr, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(saddr), "r"(v) : "memory");
  return old;
}

// Shared-memory adds with no value returned (red), for counting without the
// Gate; the second only where slot < len (unsigned).
__device__ __forceinline__ void red_add_shared(uint32_t saddr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared_in(uint32_t slot, uint32_t len, uint32_t saddr,
                                                  uint32_t v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %0, %1;\n\t@q red.shared.add.u32 [%2], %3;\n\t}"
      ::"r"(slot), "r"(len), "r"(saddr), "r"(v)
      : "memory");
}

// The same, done only where slot < len (unsigned; the address is not touched
// otherwise); returns 0 where it is not done.
__device__ __forceinline__ uint32_t atom_add_shared_in(uint32_t slot, uint32_t len, uint32_t saddr,
                                                       uint32_t v) {
  uint32_t old = 0;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q atom.shared.add.u32 %0, [%3], %4;\n\t}"
      : "+r"(old)
      : "r"(slot), "r"(len), "r"(saddr), "r"(v)
      : "memory");
  return old;
}

// First `limit` lanes (ascending id) whose count equals `value` (or is at
// least `value` when AT_LEAST; value >= 1) become result keys dst[0..);
// returns how many.  Each thread reads four counter words per round; the
// rounds stop once `limit` lanes are found.  Words between nwords and the next
// multiple of four must exist and be zero.  All threads of the block call it.
template <int LOG2W, bool AT_LEAST>
__device__ uint32_t collect_lanes(const uint32_t* bc, uint32_t nwords, uint32_t value,
                                  uint32_t limit, uint32_t obj_base, unsigned long long* dst,
                                  uint32_t* scratch) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, MASK = (1u << W) - 1u;
  const uint32_t nw4 = (nwords + 3) & ~3u;
  uint32_t found = 0;
  for (uint32_t r0 = 0; r0 < nw4 && found < limit; r0 += 4 * blockDim.x) {
    const uint32_t w0 = r0 + 4 * threadIdx.x;
    const uint4 q = w0 < nw4 ? *reinterpret_cast<const uint4*>(bc + w0) : make_uint4(0, 0, 0, 0);
    const uint32_t words[4] = {q.x, q.y, q.z, q.w};
    uint32_t m = 0;
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) {
#pragma unroll
      for (uint32_t l = 0; l < PER; ++l) {
        const uint32_t v = (words[e] >> (l * W)) & MASK;
        m += AT_LEAST ? (v >= value) : (v == value);
      }
    }
    uint32_t total;
    uint32_t pos = found + dev::block_exclusive_scan(m, scratch, &total);
    if (m && pos < limit) {
#pragma unroll
      for (uint32_t e = 0; e < 4; ++e) {
#pragma unroll
        for (uint32_t l = 0; l < PER; ++l) {
          const uint32_t v = (words[e] >> (l * W)) & MASK;
          if ((AT_LEAST ? (v >= value) : (v == value)) && pos < limit)
            dst[pos++] = dev::result_key(v, obj_base + (w0 + e) * PER + l);
        }
      }
    }
    found += total;
  }
  return min(found, limit);
}

// Largest count of the range (all threads of the block call it).
template <int LOG2W>
__device__ uint32_t max_count(const uint32_t* bc, uint32_t nwords, uint32_t* scratch) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, MASK = (1u << W) - 1u;
  uint32_t m = 0;
  for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) {
    const uint32_t word = bc[w];
    if (word) {
#pragma unroll
      for (uint32_t l = 0; l < PER; ++l) m = max(m, (word >> (l * W)) & MASK);
    }
  }
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  __syncthreads();  // scratch may still be read by a previous call
  if (dev::lane_id() == 0) scratch[dev::warp_id()] = m;
  __syncthreads();
  if (dev::warp_id() == 0) {
    uint32_t v = dev::lane_id() < (blockDim.x >> 5) ? scratch[dev::lane_id()] : 0u;
    v = __reduce_max_sync(0xFFFFFFFFu, v);
    if (dev::lane_id() == 0) scratch[32] = v;
  }
  __syncthreads();
  return scratch[32];
}

// How many counters of the range are at least x1, x2 and x3, in one pass
// over the words (all threads of the block call it).
template <int LOG2W>
__device__ void count_at_least3(const uint32_t* bc, uint32_t nwords, uint32_t x1, uint32_t x2,
                                uint32_t x3, unsigned long long* scratch, uint32_t out[3]) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, MASK = (1u << W) - 1u;
  uint32_t m1 = 0, m2 = 0, m3 = 0;
  for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) {
    const uint32_t word = bc[w];
    if (word) {
#pragma unroll
      for (uint32_t l = 0; l < PER; ++l) {
        const uint32_t v = (word >> (l * W)) & MASK;
        m1 += v >= x1;
        m2 += v >= x2;
        m3 += v >= x3;
      }
    }
  }
  // at most 2^18 counters per range: three 21-bit fields
  const unsigned long long s = dev::block_sum<unsigned long long>(
      m1 | ((unsigned long long)m2 << 21) | ((unsigned long long)m3 << 42), scratch);
  out[0] = (uint32_t)(s & 0x1FFFFFu);
  out[1] = (uint32_t)((s >> 21) & 0x1FFFFFu);
  out[2] = (uint32_t)(s >> 42);
}

// The k-th largest count t of the range (0 when fewer than k counters are
// >= 1): the largest x with #{count >= x} >= k.  One pass for the maximum M,
// then a four-way search of [1, M] with three thresholds counted per pass
// (a binary search of [1, B] would take log2 B passes).  All threads call it.
template <int LOG2W>
__device__ uint32_t kth_count(const uint32_t* bc, uint32_t nwords, uint32_t k, uint32_t* scratch,
                              unsigned long long* scratch64) {
  const uint32_t M = max_count<LOG2W>(bc, nwords, scratch);
  uint32_t lo = 0, hi = M;  // #{>= lo} >= k (or lo = 0) and #{>= hi + 1} < k
  while (lo < hi) {
    const uint32_t span = hi - lo;  // candidates lo + 1 .. hi
    const uint32_t y1 = lo + (span + 3) / 4;
    const uint32_t y2 = max(y1, lo + (span + 1) / 2);
    const uint32_t y3 = max(y2, lo + (3 * span + 3) / 4);
    uint32_t c[3];
    count_at_least3<LOG2W>(bc, nwords, y1, y2, y3, scratch64, c);
    if (c[2] >= k) lo = y3;
    else if (c[1] >= k) { lo = y2; hi = y3 - 1; }
    else if (c[0] >= k) { lo = y1; hi = y2 - 1; }
    else hi = y1 - 1;
  }
  return lo;
}

template <int LOG2W>
__device__ __forceinline__ uint32_t lane_count(const uint32_t* bc, uint32_t local) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, LPW = 5 - LOG2W, MASK = (1u << W) - 1u;
  return (vld(&bc[local >> LPW]) >> ((local & (PER - 1)) << LOG2W)) & MASK;
}

// ---------------------------------------------------------------------------
// Dense keywords: their object bitmaps are added whole
// ---------------------------------------------------------------------------
//
// A keyword whose list holds a large share of the objects is also stored as
// an object bitmap.  A block adds the bitmaps of its query's dense keywords to
// the Bitmap Counter before it scans the sparse keywords' lists: each thread
// sums its 32-object bitmap words over the keywords in bit-sliced counters
// (slice j holds bit j of 32 counts; full adders on whole words, three
// inputs per two bitwise operations), then turns the slices into counts with
// an 8 x 8 bit transpose and adds them to the counter words it owns.  The
// counts are those the lists would give, one per (keyword, object) pair.

// Full adder on 32 bit positions at once: l = a ^ b ^ c (weight 1), h =
// majority(a, b, c) (weight 2).
__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

// s[0..7] (bit-sliced counts, weights 1, 2, ..., 128) += x.
__device__ __forceinline__ void slices_add1(uint32_t (&s)[8], uint32_t x) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t t = s[j] & x;
    s[j] ^= x;
    x = t;
  }
}

// s += x[0] + ... + x[7]: a carry-save tree for the low three weights, the
// weight-8 carry rippled into the rest.
__device__ __forceinline__ void slices_add8(uint32_t (&s)[8], const uint32_t* x) {
  uint32_t t2a, t2b, t4a, t4b, t8;
  csa(t2a, s[0], s[0], x[0], x[1]);
  csa(t2b, s[0], s[0], x[2], x[3]);
  csa(t4a, s[1], s[1], t2a, t2b);
  csa(t2a, s[0], s[0], x[4], x[5]);
  csa(t2b, s[0], s[0], x[6], x[7]);
  csa(t4b, s[1], s[1], t2a, t2b);
  csa(t8, s[2], s[2], t4a, t4b);
#pragma unroll
  for (int j = 3; j < 8; ++j) {
    const uint32_t t = s[j] & t8;
    s[j] ^= t8;
    t8 = t;
  }
}

// Counts of objects 8q .. 8q+7 of a bitmap word from its slices, one byte
// each (byte c = count of object 8q + c): the 8 x 8 bit matrix with row j =
// byte q of slice j, transposed (three delta swaps).
__device__ __forceinline__ unsigned long long slice_bytes(const uint32_t (&s)[8], uint32_t q) {
  const uint32_t sel = q | ((q + 4) << 4);
  const uint32_t lo = __byte_perm(__byte_perm(s[0], s[1], sel), __byte_perm(s[2], s[3], sel), 0x5410);
  const uint32_t hi = __byte_perm(__byte_perm(s[4], s[5], sel), __byte_perm(s[6], s[7], sel), 0x5410);
  unsigned long long x = ((unsigned long long)hi << 32) | lo, t;
  t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x ^= t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x ^= t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x ^= t ^ (t << 28);
  return x;
}

// 8 object counts (bytes, object c in byte c) as counter words: 8-bit lanes
// (x, y of a uint2 as the words' values; z, w unused) or 16-bit lanes (a
// uint4: objects 2i, 2i+1 in the low and high halves of word i).
template <int LOG2W>
__device__ __forceinline__ uint4 lane_words(unsigned long long b) {
  const uint32_t lo = (uint32_t)b, hi = (uint32_t)(b >> 32);
  if (LOG2W == 3) return make_uint4(lo, hi, 0u, 0u);
  return make_uint4(__byte_perm(lo, 0u, 0x4140), __byte_perm(lo, 0u, 0x4342),
                    __byte_perm(hi, 0u, 0x4140), __byte_perm(hi, 0u, 0x4342));
}

// Adds the counter words of 8 objects to those at word index i: a uint2
// (8-bit lanes) or uint4 (16-bit lanes) in shared memory.
template <int LOG2W>
__device__ __forceinline__ void lane_words_add(uint32_t* bc, uint32_t i, uint4 x) {
  if (LOG2W == 3) {
    uint2* p = reinterpret_cast<uint2*>(bc + i);
    uint2 v = *p;
    v.x += x.x;
    v.y += x.y;
    *p = v;
  } else {
    uint4* p = reinterpret_cast<uint4*>(bc + i);
    uint4 v = *p;
    v.x += x.x;
    v.y += x.y;
    v.z += x.z;
    v.w += x.w;
    *p = v;
  }
}

// Adds the counts of bitmap word w (local objects 32w .. 32w+31) to the
// counter words that hold them (8-bit lanes: four objects per word; 16-bit:
// two).  The calling thread owns those words.  With
// 16-bit lanes a word's four groups of 8 objects (16 bytes of counters each)
// go in an order that starts at a group set by the thread's index, so that
// the threads of a warp, which own words 128 bytes apart, spread their
// accesses over the shared-memory banks.
template <int LOG2W>
__device__ __forceinline__ void slices_emit(uint32_t* bc, uint32_t w, const uint32_t (&s)[8]) {
  if (!(s[0] | s[1] | s[2] | s[3] | s[4] | s[5] | s[6] | s[7])) return;
  constexpr uint32_t WPG = 8u >> (5 - LOG2W);  // counter words per group of 8 objects
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j) {
    const uint32_t q = LOG2W == 4 ? (j + threadIdx.x) & 3u : j;
    lane_words_add<LOG2W>(bc, (4 * w + q) * WPG, lane_words<LOG2W>(slice_bytes(s, q)));
  }
}

// Adds n <= 255 object bitmaps to the Bitmap Counter of range g: ptrs[i] =
// the range's slice of bitmap i, as 8-byte words (in shared memory, set once
// per block).  Each thread takes two adjacent 32-object words at a time (one
// 8-byte load per bitmap) and reads eight bitmaps per step; all threads call
// it.
template <int LOG2W>
__device__ void dense_add(const ScanArgs& A, uint32_t g, uint32_t* bc, const uint2* const* ptrs,
                          uint32_t n) {
  const uint32_t nwr = (1u << A.block_shift) >> 5;  // bitmap words of the range (even)
  for (uint32_t p = threadIdx.x; p < (nwr >> 1); p += blockDim.x) {
    uint32_t s0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, s1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t d = 0;
    for (; d + 8 <= n; d += 8) {
      uint32_t x0[8], x1[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint2 v = __ldg(ptrs[d + e] + p);
        x0[e] = v.x;
        x1[e] = v.y;
      }
      slices_add8(s0, x0);
      slices_add8(s1, x1);
    }
    for (; d < n; ++d) {
      const uint2 v = __ldg(ptrs[d] + p);
      slices_add1(s0, v.x);
      slices_add1(s1, v.y);
    }
    slices_emit<LOG2W>(bc, 2 * p, s0);
    slices_emit<LOG2W>(bc, 2 * p + 1, s1);
  }
}

// State the Gate touches, all in shared memory of one block.
struct GateState {
  uint32_t* za;       // ZipperArray, 1-based
  uint32_t* present;  // one bit per object of the range: has a hash-table entry
  uint32_t* ht;       // hash table of candidate ids
  const uint32_t* bc; // Bitmap Counter
  uint32_t* at;       // AuditThreshold
  uint32_t* flags;    // [0] an insert found no slot, [1] a count above the bound
};

// What the Gate of one block needs besides a posting, kept in shared memory so
// that the scan loop does not hold it in registers.
struct GateCtx {
  GateState g;
  uint32_t kq;        // k of the query
  uint32_t B;         // count bound of the query
  uint32_t obj_base;  // first object id of the range
  uint32_t ht_mask;   // hash-table slots - 1
  uint32_t ht_bits;   // log2 of the hash-table slots
  uint32_t n_gate;    // Gate passes of the block (statistics)
  uint32_t n_ins;     // hash-table inserts of the block (statistics)
};

// Hash-table insert of a candidate id (once per object while it is flagged
// present).  A slot is free when empty or when its object's exact count has
// fallen below AT - 1 (Sec. 3.3.2); the evicted object loses its flag.
template <int LOG2W>
__device__ __noinline__ void ht_insert(const GateState g, uint32_t id, uint32_t obj_base,
                                       uint32_t ht_mask, uint32_t ht_bits) {
  uint32_t slot = ht_bits ? (id * 2654435761u) >> (32 - ht_bits) : 0u;
  for (uint32_t probe = 0; probe < kMaxProbe; ++probe, slot = (slot + 1) & ht_mask) {
    uint32_t e = vld(&g.ht[slot]);
    for (;;) {
      bool free_slot = e == kEmpty;
      if (!free_slot) free_slot = lane_count<LOG2W>(g.bc, e - obj_base) + 1 < vld(g.at);
      if (!free_slot) break;
      uint32_t prev = atomicCAS(&g.ht[slot], e, id);
      if (prev == e) {
        if (e != kEmpty) {
          uint32_t le = e - obj_base;
          atomicAnd(&g.present[le >> 5], ~(1u << (le & 31)));
        }
        return;
      }
      e = prev;
    }
  }
  g.flags[0] = 1;  // not placed: the read-out falls back to the Bitmap Counter
}

// AT advance of Algorithm 1: while ZA[AT] >= k, AT grows by one.
// AT is read without locking and raised by atomicMax, so concurrent callers
// only ever move it up to a level whose ZipperArray entry has reached k.
__device__ __noinline__ void advance_at(const GateState g, uint32_t kq, uint32_t B) {
  uint32_t a = vld(g.at);
  while (a <= B && vld(&g.za[a]) >= kq) {
    atomicMax(g.at, a + 1);
    ++a;
  }
}

// The Gate of Algorithm 1 for one posting that made object id's
// count c >= AT: the pass is numbered z at its level by the ZipperArray
// increment; the first k passes of a level are hash-table candidates (each
// object inserted once while it holds its presence bit); the pass that fills
// a level to k advances AT.  AT may lag behind a full level for a while (a
// stale AT only admits more passes); the read-out recomputes AT_f.
template <int LOG2W>
__device__ __forceinline__ void gate_pass(const GateState& g, uint32_t id, uint32_t c,
                                          uint32_t kq, uint32_t B, uint32_t obj_base,
                                          uint32_t ht_mask, uint32_t ht_bits, uint32_t& n_gate,
                                          uint32_t& n_ins) {
  if (c > B) {  // cannot happen with a valid bound
    g.flags[1] = 1;
    return;
  }
  const uint32_t z = atomicAdd(&g.za[c], 1u);
  ++n_gate;
  if (z < kq) {
    const uint32_t local = id - obj_base;
    const uint32_t w = local >> 5, b = 1u << (local & 31);
    if (!(vld(&g.present[w]) & b) && !(atomicOr(&g.present[w], b) & b)) {
      ++n_ins;
      ht_insert<LOG2W>(g, id, obj_base, ht_mask, ht_bits);
    }
  }
  if (z + 1 == kq) advance_at(g, kq, B);
}

// Largest x in 1..B with h[x] + ... + h[B] >= k (0 if there is none): the
// k-th largest count of the objects the histogram h counts.  h is read
// through L2 (other blocks add to it).  All threads of the block call it.
__device__ __forceinline__ uint32_t hist_kth(const uint32_t* h, uint32_t B, uint32_t k,
                                             uint32_t* scratch, uint32_t& s_res) {
  if (threadIdx.x == 0) s_res = 0;
  uint32_t carry = 0;
  for (uint32_t top = B; top >= 1;) {  // levels top, top - 1, ... from the highest
    const uint32_t n = min(top, blockDim.x);
    const uint32_t c = threadIdx.x < n ? top - threadIdx.x : 0u;
    const uint32_t v = c ? __ldcg(&h[c]) : 0u;
    uint32_t total;
    const uint32_t incl = carry + dev::block_exclusive_scan(v, scratch, &total) + v;
    if (c && incl >= k && incl - v < k) s_res = c;  // the level where the sum reaches k
    __syncthreads();
    const uint32_t r = s_res;
    if (r || carry + total >= k) return r;
    carry += total;
    top -= n;
  }
  return 0;
}

// Adds the counts a finished range reports (cand[0..n_hi) and n_tie ties at
// at_f - 1) that lie above the query's current seed to the query's histogram
// hh, then raises the seed to the k-th largest count the histogram holds.
// h0: the seed as read a little earlier; it only grows, so an early read
// lets in some counts at or below the current seed, which are still reported
// counts of distinct objects.
// The histogram counts a subset of the reported objects, so that k-th
// largest is still at most the query's k-th count; counts at or below the
// current seed cannot raise it and are left out.  All threads of the block
// call it.
__device__ __noinline__ void publish_seed(uint32_t* hh, uint32_t* seed, uint32_t h0,
                                          const unsigned long long* cand, uint32_t n_hi,
                                          uint32_t n_tie, uint32_t at_f, uint32_t B, uint32_t k,
                                          uint32_t* scratch, uint32_t* s_res) {
  int added = 0;
  for (uint32_t i = threadIdx.x; i < n_hi; i += blockDim.x) {
    const uint32_t c = dev::key_count(cand[i]);
    if (c > h0) {
      atomicAdd(&hh[c], 1u);
      added = 1;
    }
  }
  if (threadIdx.x == 0 && n_tie && at_f - 1 > h0) {
    atomicAdd(&hh[at_f - 1], n_tie);
    added = 1;
  }
  // No fence: the barrier orders the block's additions before its reads, and
  // a seed taken from any part of the histogram is still a valid one.
  if (!__syncthreads_or(added)) return;
  const uint32_t x = hist_kth(hh, B, k, scratch, *s_res);
  if (threadIdx.x == 0 && x) atomicMax(seed, x);
}

// Old counter words of one lane's 4 * U postings in a tile.
template <int U>
struct TileWords {
  uint32_t w[4 * U];
};

// The exact Gate test of a tile whose word test may have passed, kept out of
// line so that the scan loop's registers and code stay those of the common
// case.  Slot i of the lane is posting c_start + (i / 4 * 32 + lane) * 4 +
// i % 4 of the List Array; it passes when it lies in [c_lo, c_hi) and its own
// lane of val.w[i], plus one, reaches at_c.  The passing slots run the Gate in
// ascending slot order (ids reloaded from L1) and are counted into
// ctx.n_gate and ctx.n_ins.  All lanes of the warp call it.
template <int LOG2W, int U>
__device__ __noinline__ void gate_tile(GateCtx& ctx, const uint32_t* __restrict__ post_ids,
                                        uint32_t c_start, uint32_t c_lo, uint32_t c_hi,
                                        const TileWords<U> val, uint32_t at_c) {
  const GateState g = ctx.g;
  const uint32_t kq = ctx.kq, B = ctx.B, obj_base = ctx.obj_base, ht_mask = ctx.ht_mask,
                 ht_bits = ctx.ht_bits;
  const uint32_t lane = dev::lane_id();
  const uint32_t d0 = c_start + lane * 4 - c_lo, len = c_hi - c_lo;
  uint32_t pm = 0;  // this lane's passing slots
#pragma unroll
  for (uint32_t u = 0; u < U; ++u) {
    const uint32_t idx = c_start + (u * 32 + lane) * 4;
    const uint4 w = idx < c_hi ? __ldg(reinterpret_cast<const uint4*>(post_ids + idx))
                               : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (uint32_t e = 0; e < 4; ++e) {
      const uint32_t i = u * 4 + e;
      const uint32_t id = e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w;
      pm |= (uint32_t)(d0 + u * 128 + e < len &&
                       Lane<LOG2W>::pick(val.w[i], Lane<LOG2W>::sel(id)) + 1 >= at_c)
            << i;
    }
  }
  uint32_t n_gate = 0, n_ins = 0;
  for (uint32_t m = pm; m; m &= m - 1) {
    const uint32_t i = __ffs(m) - 1;
    uint32_t word = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4 * U; ++j) word = j == i ? val.w[j] : word;
    const uint32_t id = __ldg(post_ids + c_start + ((i >> 2) * 32 + lane) * 4 + (i & 3));
    gate_pass<LOG2W>(g, id, Lane<LOG2W>::pick(word, Lane<LOG2W>::sel(id)) + 1, kq, B, obj_base,
                     ht_mask, ht_bits, n_gate, n_ins);
  }
  if (n_gate) atomicAdd(&ctx.n_gate, n_gate);
  if (n_ins) atomicAdd(&ctx.n_ins, n_ins);
}

// Static shared state of one block.
struct BlockShared {
  uint32_t at;        // AuditThreshold
  uint32_t n;         // read-out counter
  uint32_t item;      // persistent blocks: current work item
  uint32_t flags[2];  // [0] hash table incomplete, [1] inconsistent input
  uint32_t kth;       // hist_kth result
  uint32_t at0;       // AuditThreshold the range started with
  uint32_t gateless;  // count only, then select from the Bitmap Counter
  uint32_t tie_floor; // ties below it are left out of the read-out
  uint32_t hint_now;  // the query's seed as the read-out began
  uint32_t next_run;  // next run of tiles to be claimed
  uint32_t n_dense;   // dense keywords whose bitmaps the range added
  uint32_t n_found;   // objects the dense phase found at or above AT
  GateCtx gate;       // the Gate's pointers and query constants
  uint32_t scratch[33];
  unsigned long long scratch64[33];
};

// The dense keywords of query keywords q_kw[qa..qb) for range g: their
// bitmaps are added to the Bitmap Counter (the lists are not scanned).  Then,
// for a range that runs the Gate (gated), the ZipperArray is set to what the
// Gate would hold after these counts -- ZA[i] = #objects with count >= i for
// i >= AT (each object passes every level up to its count) -- AT advances
// past the full levels, and the objects at or above the new AT (fewer than
// k) enter the hash table.  pre_slot: dense_slot of keyword qa + threadIdx.x
// (loaded by the caller; kNoDense past qb).  list: 2 * kKwBatch words of
// shared memory; ptrs:
// room for 255 pointers, 8-byte aligned, in shared memory.
// Returns the number of dense keywords added.  All threads call it.
template <int LOG2W>
__device__ __noinline__ uint32_t dense_phase(const ScanArgs& A, uint32_t g, uint32_t qa, uint32_t qb,
                                             uint32_t pre_slot, uint32_t* bc, uint32_t nwords,
                                             uint32_t* list,
                                             const uint2** ptrs, bool gated, BlockShared& S) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, MASK = (1u << W) - 1u;
  const uint32_t tid = threadIdx.x, cap = 2 * kKwBatch;
  uint32_t total = 0;
  const uint32_t nwr = (1u << A.block_shift) >> 5;
  const uint2* base = reinterpret_cast<const uint2*>(A.dense_bits + (uint64_t)g * nwr);
  const uint64_t mw2 = A.map_words >> 1;
  for (uint32_t kb = qa; kb < qb; kb += cap) {
    const uint32_t nk = min(cap, qb - kb);
    if (kb != qa) {  // S.n starts at 0 (the reset of the work item)
      if (tid == 0) S.n = 0;
      __syncthreads();
    }
    // the list of slots, and the pointers of its first 255 bitmaps
    for (uint32_t i = tid; i < nk; i += blockDim.x) {
      const uint32_t sl = (kb == qa && i == tid) ? pre_slot : A.dense_slot[A.q_kw[kb + i]];
      if (sl != kNoDense) {
        const uint32_t j = atomicAdd(&S.n, 1u);
        list[j] = sl;
        if (j < 255) ptrs[j] = base + sl * mw2;
      }
    }
    __syncthreads();
    const uint32_t nd = S.n;
    for (uint32_t d0 = 0; d0 < nd; d0 += 255) {
      const uint32_t m = min(255u, nd - d0);
      if (d0) {  // the next group's pointers, once the last group's are read
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ptrs[i] = base + list[d0 + i] * mw2;
        __syncthreads();
      }
      dense_add<LOG2W>(A, g, bc, ptrs, m);
    }
    total += nd;
    __syncthreads();  // the list is refilled, the counters are read next
  }
  if (!gated || total == 0) return total;
  GateCtx& G = S.gate;
  uint32_t* za = G.g.za;
  const uint32_t at0 = S.at, B = G.B;
  // ZA[c] = #objects with count c (c >= at0) ...  With lane headroom a word's
  // lanes are looked at only when the word-wide test (as in the Gate: adding
  // 2^(W-1) - at0 to every lane sets a lane's top bit exactly when the lane
  // holds at0 or more) says one of them reaches at0.  The objects found are
  // also listed (up to `cap`; the dense slots are added, so `list` is free)
  // for the hash-table pass below.
  const bool headroom = B < (1u << (W - 1));
  const uint32_t add = Lane<LOG2W>::kHigh - at0 * Lane<LOG2W>::kOnes;
  for (uint32_t w = tid; w < nwords; w += blockDim.x) {
    const uint32_t word = bc[w];
    if (headroom ? !((word + add) & Lane<LOG2W>::kHigh) : !word) continue;
#pragma unroll
    for (uint32_t l = 0; l < PER; ++l) {
      const uint32_t c = (word >> (l * W)) & MASK;
      if (c >= at0 && c <= B) {
        atomicAdd(&za[c], 1u);
        const uint32_t i = atomicAdd(&S.n_found, 1u);  // zero since the reset
        if (i < cap) list[i] = w * PER + l;
      }
    }
  }
  __syncthreads();
  // ... then suffix sums over [at0, B] by warp 0, 32 levels per step from the top
  if (tid < 32) {
    uint32_t carry = 0;
    for (int top = (int)B; top >= (int)at0; top -= 32) {
      const int c = top - (int)tid;
      uint32_t v = c >= (int)at0 ? za[c] : 0u;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if ((int)tid >= d) v += o;
      }
      if (c >= (int)at0) za[c] = v + carry;
      carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t a = at0;
    while (a <= B && za[a] >= G.kq) ++a;
    S.at = a;
  }
  __syncthreads();
  const uint32_t a = S.at, n_found = S.n_found;
  if (a <= B && za[a] > 0 && n_found <= cap) {  // the listed objects at or above a
    for (uint32_t i = tid; i < n_found; i += blockDim.x) {
      const uint32_t local = list[i];
      if (lane_count<LOG2W>(bc, local) >= a) {
        atomicOr(&G.g.present[local >> 5], 1u << (local & 31));
        ht_insert<LOG2W>(G.g, G.obj_base + local, G.obj_base, G.ht_mask, G.ht_bits);
      }
    }
  } else if (a <= B && za[a] > 0) {  // fewer than k objects: presence bits and hash-table entries
    for (uint32_t w = tid; w < nwords; w += blockDim.x) {
      const uint32_t word = bc[w];
      if (word) {
#pragma unroll
        for (uint32_t l = 0; l < PER; ++l) {
          if (((word >> (l * W)) & MASK) >= a) {
            const uint32_t local = w * PER + l;
            atomicOr(&G.g.present[local >> 5], 1u << (local & 31));
            ht_insert<LOG2W>(G.g, G.obj_base + local, G.obj_base, G.ht_mask, G.ht_bits);
          }
        }
      }
    }
  }
  __syncthreads();
  return total;
}

// One (query, object range) work item: reset the range's c-PQ in shared
// memory, scan the postings of the query's keywords inside the range through
// the Bitmap Counter and the Gate, then write the range's exact top-k
// (Theorem 3.1) as result keys to A.cand.  All threads of the block call it.
// LOG2W: log2 of the counter width; U: 16-byte loads in flight per lane (a
// warp tile is 128 * U postings); DENSE: the range adds the bitmaps of the
// query's dense keywords and scans only the other lists (a separate
// instantiation, so that the plain scan's code is untouched by the dense one).
// The tile loop's Gate mode, fixed per block (the loop is compiled once per
// mode, so it holds no per-tile branch on it): 0 counting only (gateless), 1
// the word-wide Gate test (lane headroom), 2 the per-lane Gate test.
template <int M>
struct GateMode {
  static constexpr int value = M;
};

template <int LOG2W, int U, bool DENSE>
__device__ __forceinline__ void cpq_item(const ScanArgs& A, uint32_t qi, uint32_t g,
                                         uint4* smem_raw, BlockShared& S) {
  constexpr uint32_t W = 1u << LOG2W, PER = 32u / W, LPW = 5 - LOG2W;
  constexpr uint32_t kUnroll = U, kTile = 32 * 4 * U;
  uint32_t& s_at = S.at;
  uint32_t& s_n = S.n;
  uint32_t* s_flags = S.flags;
  uint32_t* scratch = S.scratch;

  // shared-memory layout: Bitmap Counter | presence bits | Hash Table | read-out
  // buffer | ZipperArray | staged keyword segments
  const uint32_t nwords = (1u << A.block_shift) >> LPW;
  const uint32_t npresent = (1u << A.block_shift) >> 5;
  const uint32_t kpad = dev::next_pow2(A.k);
  uint32_t* bc = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* present = bc + nwords;
  uint32_t* ht = present + npresent;
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(ht + A.ht_slots);
  uint2* seg = reinterpret_cast<uint2*>(cand + kpad);  // [keyword] (lo, hi) in the List Array
  uint32_t* za = reinterpret_cast<uint32_t*>(seg + kKwBatch);
  uint32_t* tile_pre = za + A.za_len;  // [keyword] first tile, then the tile count

  const uint32_t tid = threadIdx.x, lane = dev::lane_id(), warp = dev::warp_id();
  const uint32_t nwarps = blockDim.x >> 5;
  const uint32_t q = A.q_sel ? A.q_sel[qi] : qi;
  const uint32_t c0 = g * A.chunks_per_block, c1 = min(c0 + A.chunks_per_block, A.n_chunks);
  const uint32_t qa = A.q_off[q], qb = A.q_off[q + 1];
  // The first keyword batch's sublist bounds, loaded before the reset so that
  // their chain of loads overlaps it (not in the dense instantiation, whose
  // bitmap phase comes in between).
  uint32_t pre_lo = 0, pre_hi = 0;
  if (!DENSE && tid < min(kKwBatch, qb - qa)) {
    const uint32_t kw = A.q_kw[qa + tid];
    const uint64_t base = A.kw_off[kw];
    const uint32_t* row = A.chunk_pos + (uint64_t)kw * (A.n_chunks + 1);
    pre_lo = (uint32_t)(base + row[c0]);
    pre_hi = (uint32_t)(base + row[c1]);
  }
  // In the dense instantiation, the bitmap slot of the thread's first keyword
  uint32_t pre_slot = kNoDense;
  if (DENSE && LOG2W >= 3 && tid < min(2 * kKwBatch, qb - qa))
    pre_slot = A.dense_slot[A.q_kw[qa + tid]];

  // ---- reset this block's c-PQ ------------------------------------------
  // The query's k and bound and the range's first id live in S.gate from
  // here on (the scan loop keeps none of them in registers).
  {
    const uint32_t kq = A.k_arr ? A.k_arr[q] : A.k;
    const uint32_t B = A.bound[q];
    const uint32_t obj_base = g << A.block_shift;
    const uint32_t ht_mask = A.ht_slots - 1, ht_bits = 31 - __clz(A.ht_slots);
    // the seed's loads go out before the zeroing and are used after it (a
    // hint read a little early is still a valid seed: hints only grow)
    uint32_t seed0 = 1u, hint0 = 0u;
    if (tid == 0) {
      if (A.seed) seed0 = A.seed[q];
      if (A.at_hint) hint0 = vld(&A.at_hint[qi]);
    }
    uint4* b4 = reinterpret_cast<uint4*>(bc);
    const uint4 z4 = make_uint4(0, 0, 0, 0);
    for (uint32_t i = tid; i < ((nwords + npresent) >> 2); i += blockDim.x) b4[i] = z4;
    for (uint32_t i = tid; i < A.ht_slots; i += blockDim.x) ht[i] = kEmpty;
    for (uint32_t i = tid; i < B + 2; i += blockDim.x) za[i] = 0;
    if (tid == 0) {
      const uint32_t s0 = max(seed0, hint0);
      s_at = max(1u, min(s0, B + 1));
      S.at0 = s_at;
      // A range that starts before any range of its query has finished (no
      // seed yet) would run the Gate from AT = 1 through every level; its
      // k-th count is selected from the Bitmap Counter after counting
      // instead, and the ranges after it run the Gate from its seed.
      S.gateless = A.no_gate || (A.at_hint && s_at == 1);
      s_flags[0] = 0;
      s_flags[1] = 0;
      s_n = 0;  // the dense phase's counters
      S.n_found = 0;
      S.gate = GateCtx{GateState{za, present, ht, bc, &s_at, s_flags}, kq, B, obj_base, ht_mask,
                       ht_bits, 0u, 0u};
    }
  }
  __syncthreads();
  const bool gateless = S.gateless;
  // every count of the range stays below the top bit of its lane
  const bool swar = S.gate.B < (1u << ((1u << LOG2W) - 1));
  // dense keywords first: their bitmaps are added whole, their lists skipped
  // (the count stays in shared memory: the scan loop has no register to spare)
  if (DENSE && LOG2W >= 3) {
    // the tile prefix sums are not in use yet: room for the bitmap pointers
    const uint2** ptrs = reinterpret_cast<const uint2**>(
        (reinterpret_cast<uintptr_t>(tile_pre) + 7) & ~(uintptr_t)7);
    const uint32_t nd = dense_phase<LOG2W>(A, g, qa, qb, pre_slot, bc, nwords,
                                           reinterpret_cast<uint32_t*>(seg), ptrs, !gateless, S);
    if (tid == 0) S.n_dense = nd;
  } else if (tid == 0) {
    S.n_dense = 0;
  }

  // ---- scan: all postings of the query's keywords inside this id range ---
  const uint32_t stride = A.n_chunks + 1;
  // a register copy: A may live in shared memory (persistent blocks), which
  // the counter atomics' memory clobbers would make the loop reload
  const uint32_t* __restrict__ post_ids = A.post_ids;
  // shared address of the counter word of object id: bc_adj + byte_off(id)
  const uint32_t bc_adj =
      (uint32_t)__cvta_generic_to_shared(bc) - Lane<LOG2W>::byte_off(S.gate.obj_base);
  for (uint32_t kb = qa; kb < qb; kb += kKwBatch) {
    const uint32_t nk = min(kKwBatch, qb - kb);
    uint32_t ntiles = 0;
    if (tid < nk) {
      uint32_t lo = pre_lo, hi = pre_hi;
      if (DENSE || kb != qa) {
        const uint32_t kw = A.q_kw[kb + tid];
        lo = hi = 0;
        if (!DENSE || LOG2W < 3 || A.dense_slot[kw] == kNoDense) {  // a dense keyword's list is skipped
          const uint64_t base = A.kw_off[kw];
          const uint32_t* row = A.chunk_pos + (uint64_t)kw * stride;
          lo = (uint32_t)(base + row[c0]);
          hi = (uint32_t)(base + row[c1]);
        }
      }
      seg[tid] = make_uint2(lo, hi);
      ntiles = hi > lo ? (hi - (lo & ~3u) + kTile - 1) / kTile : 0;
    }
    uint32_t total_tiles;
    uint32_t pre = dev::block_exclusive_scan(ntiles, scratch, &total_tiles);
    if (tid < nk) tile_pre[tid] = pre;
    // after the last keyword: the tile count, then entries no tile reaches
    if (tid <= 32) tile_pre[nk + tid] = tid == 0 ? total_tiles : 0xFFFFFFFFu;
    if (tid == 0) S.next_run = nwarps;
    __syncthreads();

    // Warp w starts with run w of kRun consecutive tiles, then claims the
    // next unclaimed run from a shared counter (one atomic per run), so warps
    // that meet Gate passes hold the block back less.  A warp's tile numbers
    // only grow, so its segment cursor j only moves forward: by one test
    // inside a run, by 32 segments per warp-wide step when it jumps to its
    // next run.
    uint32_t j = 0;
    auto locate = [&](uint32_t tt, uint32_t& lo_, uint32_t& hi_) -> uint32_t {
      if (tile_pre[j + 1] <= tt) {
        for (;;) {
          const uint32_t ball = __ballot_sync(0xFFFFFFFFu, tile_pre[j + 1 + lane] <= tt);
          j += __popc(ball);  // tile_pre is non-decreasing: the ballot is a prefix
          if (ball != 0xFFFFFFFFu) break;
        }
      }
      const uint2 sg = seg[j];
      lo_ = sg.x;
      hi_ = sg.y;
      return (lo_ & ~3u) + (tt - tile_pre[j]) * kTile;
    };
    // the tile's 16-byte vectors that start before hi_; the others keep what
    // they held (their slots lie outside the list and are never counted)
    auto load = [&](uint32_t st_, uint32_t hi_, uint4 (&vv)[U]) {
#pragma unroll
      for (uint32_t u = 0; u < kUnroll; ++u) {
        const uint32_t idx = st_ + (u * 32 + lane) * 4;
        if (idx < hi_) vv[u] = __ldg(reinterpret_cast<const uint4*>(post_ids + idx));
      }
    };
    // One id buffer: the counter updates of a tile take its ids, then the
    // next tile is located and loaded into the same registers while the
    // updates are in flight.  The Gate test needs the counts only, not the
    // ids; the rare tile that passes it reloads its ids (from L1).
    // Runs of kRun tiles, except the last 4 x nwarps tiles of the round,
    // which are runs of one tile: the warps finish the round more evenly.
    const uint32_t n_big = total_tiles > 4 * nwarps ? (total_tiles - 4 * nwarps) / kRun : 0u;
    auto run_first = [&](uint32_t r) { return r < n_big ? r * kRun : n_big * kRun + (r - n_big); };
    auto run_last = [&](uint32_t r, uint32_t f) { return min(f + (r < n_big ? kRun : 1u), total_tiles); };
    uint32_t run = warp, t = run_first(run), t_end = run_last(run, t);
    uint32_t lo = 0, hi = 0, start = 0;
    uint4 v[kUnroll];
#pragma unroll
    for (uint32_t u = 0; u < kUnroll; ++u) v[u] = make_uint4(0, 0, 0, 0);
    if (t < total_tiles) {
      start = locate(t, lo, hi);
      load(start, hi, v);
    }
    auto tile_loop = [&](auto mode) {
      constexpr int M = decltype(mode)::value;  // GateMode
      while (t < total_tiles) {
        // the tile after t: the next of this run, else the first of the warp's next run
        const bool run_ends = t + 1 >= t_end;
        if (run_ends) {
          uint32_t r = 0;
          if (lane == 0) r = atomicAdd(&S.next_run, 1u);
          run = __shfl_sync(0xFFFFFFFFu, r, 0);
        }
        const uint32_t tn = run_ends ? run_first(run) : t + 1;
        const uint32_t tn_end = run_ends ? run_last(run, tn) : t_end;
        // Bitmap Counter: one sub-word atomic add per posting (the count update
        // of Algorithm 1); val = the counter word before the add (0 for slots
        // outside the list).  Every id of a sublist lies in this block's range.
        uint32_t val[4 * kUnroll];
        if constexpr (M == 0) {  // counting only: no old value is needed
          const uint32_t d0 = start + lane * 4 - lo, len = hi - lo;
          const bool inside = start >= lo && start + kTile <= hi;
#pragma unroll
          for (uint32_t i = 0; i < 4 * kUnroll; ++i) {
            const uint32_t u = i >> 2, e = i & 3;
            const uint32_t id = e == 0 ? v[u].x : e == 1 ? v[u].y : e == 2 ? v[u].z : v[u].w;
            const uint32_t saddr = bc_adj + Lane<LOG2W>::byte_off(id);
            if (inside) red_add_shared(saddr, Lane<LOG2W>::inc(id));
            else red_add_shared_in(d0 + u * 128 + e, len, saddr, Lane<LOG2W>::inc(id));
          }
        } else if (start >= lo && start + kTile <= hi) {
#pragma unroll
          for (uint32_t i = 0; i < 4 * kUnroll; ++i) {
            const uint32_t u = i >> 2, e = i & 3;
            const uint32_t id = e == 0 ? v[u].x : e == 1 ? v[u].y : e == 2 ? v[u].z : v[u].w;
            val[i] = atom_add_shared(bc_adj + Lane<LOG2W>::byte_off(id), Lane<LOG2W>::inc(id));
          }
        } else {  // a tile at either end of its list: slot positions checked one by one
          const uint32_t d0 = start + lane * 4 - lo, len = hi - lo;
#pragma unroll
          for (uint32_t i = 0; i < 4 * kUnroll; ++i) {
            const uint32_t u = i >> 2, e = i & 3;
            const uint32_t id = e == 0 ? v[u].x : e == 1 ? v[u].y : e == 2 ? v[u].z : v[u].w;
            val[i] = atom_add_shared_in(d0 + u * 128 + e, len, bc_adj + Lane<LOG2W>::byte_off(id),
                                        Lane<LOG2W>::inc(id));
          }
        }
        // Gate (Algorithm 1) for the postings whose new count reaches
        // the (possibly stale) AuditThreshold: rare, so a tile is tested once.
        // With headroom (every count below the lanes' top bit) the test runs
        // on whole words: adding 2^(W-1) - (AT - 1) to every lane sets a lane's
        // top bit exactly when the lane holds AT - 1 or more, without carries
        // between lanes.  It also looks at the other lanes of each word: a
        // false alarm costs only the exact test below.  Without headroom each
        // posting's own lane is taken, before the ids are overwritten.
        uint32_t at_c = 0;
        bool hit = false;
        if constexpr (M == 2) {
          at_c = vld(&s_at);
          uint32_t vmax = 0;
#pragma unroll
          for (uint32_t i = 0; i < 4 * kUnroll; ++i) {
            const uint32_t u = i >> 2, e = i & 3;
            const uint32_t id = e == 0 ? v[u].x : e == 1 ? v[u].y : e == 2 ? v[u].z : v[u].w;
            vmax = max(vmax, Lane<LOG2W>::pick(val[i], Lane<LOG2W>::sel(id)));
          }
          hit = vmax + 1 >= at_c;
        }
        const uint32_t c_lo = lo, c_hi = hi, c_start = start;
        if (tn < total_tiles) {
          if (!run_ends && start + kTile < hi) start += kTile;  // same segment
          else start = locate(tn, lo, hi);
          load(start, hi, v);
        }
        if constexpr (M != 0) {
          if constexpr (M == 1) {
            at_c = vld(&s_at);
            const uint32_t add = Lane<LOG2W>::kHigh - (at_c - 1) * Lane<LOG2W>::kOnes;
            uint32_t acc = 0;
#pragma unroll
            for (uint32_t i = 0; i < 4 * kUnroll; ++i) acc |= val[i] + add;
            hit = (acc & Lane<LOG2W>::kHigh) != 0;
          }
          if (__any_sync(0xFFFFFFFFu, hit)) {
            TileWords<U> tw;
#pragma unroll
            for (uint32_t i = 0; i < 4 * kUnroll; ++i) tw.w[i] = val[i];
            gate_tile<LOG2W, U>(S.gate, post_ids, c_start, c_lo, c_hi, tw, at_c);
          }
        }
        t = tn;
        t_end = tn_end;
      }
    };
    // 16-bit counters always have headroom (count bounds are at most
    // GENIE_MAX_BOUND), so their kernels carry no per-lane mode
    static_assert(GENIE_MAX_BOUND < (1u << 15), "16-bit counters need lane headroom");
    if (gateless) tile_loop(GateMode<0>{});
    else if (LOG2W == 4 || swar) tile_loop(GateMode<1>{});
    else tile_loop(GateMode<2>{});
    __syncthreads();
  }

  // ---- finalise AT (Lemma 3.1) and read out this range's top-k ----------
  const uint32_t kq = S.gate.kq, B = S.gate.B, obj_base = S.gate.obj_base;
  const uint32_t n_local = min(1u << A.block_shift, A.n_objects - obj_base);
  const uint32_t nwords_local = (n_local + PER - 1) / PER;
  // the query's current seed, read by one thread while AT_f is settled
  uint32_t hint_now = 0;
  if (tid == 0 && A.at_hint) hint_now = vld(&A.at_hint[qi]);
  if (gateless) {
    // the k-th count of the range: largest x with #{count >= x} >= k
    const uint32_t t = kth_count<LOG2W>(bc, nwords_local, kq, scratch, S.scratch64);
    if (tid == 0) {
      s_at = t + 1;
      s_n = 0;
    }
  } else if (tid == 0) {
    uint32_t a = s_at;
    while (a <= B && za[a] >= kq) ++a;
    s_at = a;
    s_n = 0;
  }
  // A seed (the starting AT, or the query's current one, which other blocks
  // may be raising) is at most the query's k-th count, so ties below it
  // cannot reach the query's top-k.  One thread reads it: every thread must
  // take the same branch around the block-wide tie collection.
  if (tid == 0) {
    S.tie_floor = max(S.at0, hint_now);
    S.hint_now = hint_now;
  }
  __syncthreads();
  const uint32_t at_f = s_at;
  unsigned long long* out = A.cand + ((unsigned long long)qi * A.n_groups + g) * A.k;
  // Theorem 3.1: the objects with count >= AT_f are candidates in the HT; their
  // number is exactly ZA[AT_f] (every object at or above AT_f passed that level
  // through the Gate), which certifies the read-out.
  const uint32_t want = za[at_f];
  for (uint32_t i = tid; i < A.ht_slots; i += blockDim.x) {
    uint32_t id = ht[i];
    if (id == kEmpty) continue;
    uint32_t c = lane_count<LOG2W>(bc, id - obj_base);
    if (c >= at_f) {
      uint32_t p = atomicAdd(&s_n, 1u);
      if (p < kpad) cand[p] = dev::result_key(c, id);
    }
  }
  __syncthreads();
  uint32_t n_hi = s_n;
  const bool certified = !gateless && !s_flags[0] && n_hi == want && n_hi < kq;
  if (!certified)  // Bitmap-Counter selection of the same set
    n_hi = collect_lanes<LOG2W, true>(bc, nwords_local, at_f, kq, obj_base, cand, scratch);
  __syncthreads();
  // the keys are distinct (one per object): each goes straight to its rank in
  // (count desc, id asc) order
  for (uint32_t i = tid; i < n_hi; i += blockDim.x) {
    const unsigned long long key = cand[i];
    uint32_t r = 0;
    for (uint32_t j = 0; j < n_hi; ++j) r += cand[j] > key;
    out[r] = key;
  }
  // ties at the k-th count, ascending id, from the Bitmap Counter; below the
  // tie floor they are left out (the range then reports only its objects at
  // or above AT_f)
  uint32_t n_tie = 0;
  if (at_f >= 2 && n_hi < kq && at_f - 1 >= S.tie_floor)
    n_tie = collect_lanes<LOG2W, false>(bc, nwords_local, at_f - 1, kq - n_hi, obj_base,
                                        out + n_hi, scratch);
  for (uint32_t i = n_hi + n_tie + tid; i < kq; i += blockDim.x) out[i] = 0ull;

  if (A.chunk_at && tid == 0) A.chunk_at[(unsigned long long)qi * A.n_groups + g] = at_f;
  if (A.at_hint && A.hint_hist) {
    publish_seed(A.hint_hist + (size_t)qi * A.hint_stride, &A.at_hint[qi], S.hint_now, cand, n_hi,
                 n_tie, at_f, B, kq, scratch, &S.kth);
  } else if (A.at_hint && tid == 0 && at_f >= 2) {
    atomicMax(&A.at_hint[qi], at_f - 1);
  }
  if (A.stats && tid == 0) {
    atomicAdd(&A.stats[0], (unsigned long long)S.gate.n_gate);
    atomicAdd(&A.stats[1], (unsigned long long)S.gate.n_ins);
    if (!certified && !gateless) atomicAdd(&A.stats[2], 1ull);
    if (gateless) atomicAdd(&A.stats[6], 1ull);
    if (S.n_dense) atomicAdd(&A.stats[7], (unsigned long long)S.n_dense);
    atomicAdd(&A.stats[4], 1ull);
    if (s_flags[1]) atomicAdd(&A.stats[5], 1ull);
  }
}

// One block per (query, object range).  LOG2W: log2 of the counter width; U:
// 16-byte loads in flight per lane (a warp tile is 128 * U postings);
// THREADS: the block size (512 threads with two loads per lane: two blocks
// per SM); DENSE: dense keywords are added as bitmaps.
template <int LOG2W, int U, int THREADS, bool DENSE>
__global__ void __launch_bounds__(THREADS, (THREADS == 512 && U == 2) ? 2 : 1)
    scan_cpq_kernel(const __grid_constant__ ScanArgs A) {
  extern __shared__ uint4 smem_raw[];
  __shared__ BlockShared S;
  cpq_item<LOG2W, U, DENSE>(A, blockIdx.x % A.n_sel, blockIdx.x / A.n_sel, smem_raw, S);
}

// ---------------------------------------------------------------------------
// Merge of the per-range top-k lists of each query (Sec. 3.4 merge, on device)
// ---------------------------------------------------------------------------

struct MergeArgs {
  const unsigned long long* cand;
  uint32_t n_sel;
  const uint32_t* q_sel;
  uint32_t n_groups;
  uint32_t k;
  const uint32_t* k_arr;
  const uint32_t* bound;
  uint32_t za_len;
  uint32_t* ids;
  uint32_t* counts;
  uint32_t* n_valid;
};

constexpr uint32_t kMergeThreads = 256;

// Static shared state of a merging block.
struct MergeShared {
  uint32_t t, ngt, r, n;
  uint32_t scratch[33];
};

// Top-k of query qi from its per-range lists: count threshold by histogram,
// everything above it sorted by (count desc, id asc), then the ties at the
// threshold in range order (= ascending id).  buf: next_pow2(k) keys, hist:
// za_len counters, both in shared memory.  With L2_ONLY the candidate lists
// are read past L1 (they were written by other blocks of the same launch).
template <bool L2_ONLY>
__device__ void merge_query(const MergeArgs& M, uint32_t qi, unsigned long long* buf,
                            uint32_t* hist, MergeShared& S) {
  uint32_t& s_t = S.t;
  uint32_t& s_ngt = S.ngt;
  uint32_t& s_r = S.r;
  uint32_t& s_n = S.n;
  uint32_t* scratch = S.scratch;
  const uint32_t tid = threadIdx.x;
  auto load = [](const unsigned long long* p) -> unsigned long long {
    return L2_ONLY ? __ldcg(p) : *p;
  };
  {
    const uint32_t q = M.q_sel ? M.q_sel[qi] : qi;
    const uint32_t kq = M.k_arr ? M.k_arr[q] : M.k;
    const uint32_t B = M.bound[q];
    const unsigned long long* lists = M.cand + (unsigned long long)qi * M.n_groups * M.k;
    for (uint32_t i = tid; i < B + 2; i += blockDim.x) hist[i] = 0;
    if (tid == 0) s_n = 0;
    __syncthreads();
    const uint32_t total_c = M.n_groups * kq;
    for (uint32_t i = tid; i < total_c; i += blockDim.x) {
      unsigned long long key = load(&lists[(i / kq) * M.k + (i % kq)]);
      if (key) atomicAdd(&hist[min(dev::key_count(key), B + 1)], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t cum = 0, t = 1;
      for (uint32_t v = B + 1; v >= 1; --v) {
        if (cum + hist[v] >= kq) { t = v; break; }
        cum += hist[v];
      }
      uint32_t ngt = 0;
      for (uint32_t v = t + 1; v <= B + 1; ++v) ngt += hist[v];
      s_t = t;
      s_ngt = ngt;
      s_r = min(kq - ngt, hist[t]);
    }
    __syncthreads();
    const uint32_t t = s_t, ngt = s_ngt, r = s_r;
    // every candidate above the k-th count
    for (uint32_t i = tid; i < total_c; i += blockDim.x) {
      unsigned long long key = load(&lists[(i / kq) * M.k + (i % kq)]);
      if (key && dev::key_count(key) > t) buf[atomicAdd(&s_n, 1u)] = key;
    }
    __syncthreads();
    const uint32_t n2 = dev::next_pow2(max(ngt, 1u));
    for (uint32_t i = ngt + tid; i < n2; i += blockDim.x) buf[i] = 0ull;
    __syncthreads();
    dev::bitonic_sort_desc(buf, n2);
    uint32_t* ids = M.ids + (unsigned long long)q * M.k;
    uint32_t* cnt = M.counts + (unsigned long long)q * M.k;
    for (uint32_t i = tid; i < ngt; i += blockDim.x) {
      ids[i] = dev::key_id(buf[i]);
      cnt[i] = dev::key_count(buf[i]);
    }
    // ties at the k-th count: range order = id order, each run ascending
    const uint32_t per = (M.n_groups + blockDim.x - 1) / blockDim.x;
    const uint32_t ga = min(M.n_groups, tid * per), gb = min(M.n_groups, ga + per);
    uint32_t m = 0;
    for (uint32_t gg = ga; gg < gb; ++gg)
      for (uint32_t j = 0; j < kq; ++j) {
        unsigned long long key = load(&lists[(unsigned long long)gg * M.k + j]);
        m += key && dev::key_count(key) == t;
      }
    uint32_t tot;
    uint32_t pos = dev::block_exclusive_scan(m, scratch, &tot);
    for (uint32_t gg = ga; gg < gb && pos < r; ++gg)
      for (uint32_t j = 0; j < kq && pos < r; ++j) {
        unsigned long long key = load(&lists[(unsigned long long)gg * M.k + j]);
        if (key && dev::key_count(key) == t) {
          ids[ngt + pos] = dev::key_id(key);
          cnt[ngt + pos] = t;
          ++pos;
        }
      }
    for (uint32_t i = ngt + r + tid; i < M.k; i += blockDim.x) {
      ids[i] = 0xFFFFFFFFu;
      cnt[i] = 0;
    }
    if (tid == 0) M.n_valid[q] = ngt + r;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMergeThreads) merge_kernel(const MergeArgs M) {
  extern __shared__ uint4 smem_raw[];
  __shared__ MergeShared S;
  unsigned long long* buf = reinterpret_cast<unsigned long long*>(smem_raw);  // [next_pow2(k)]
  uint32_t* hist = reinterpret_cast<uint32_t*>(buf + dev::next_pow2(M.k));    // [za_len]
  for (uint32_t qi = blockIdx.x; qi < M.n_sel; qi += gridDim.x) merge_query<false>(M, qi, buf, hist, S);
}

// ---------------------------------------------------------------------------
// Launch planning shared by the search entry points
// ---------------------------------------------------------------------------

__global__ void check_k_kernel(uint32_t n_queries, uint32_t k, const uint32_t* __restrict__ k_arr,
                               uint32_t* bad) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_queries; q += gridDim.x * blockDim.x)
    if (k_arr[q] == 0 || k_arr[q] > k) atomicOr(bad, 1u);
}

// Mean postings per (keyword, object range) from which a search defaults to
// 512 threads with eight loads per lane instead of 1024 (or 768) with two.
constexpr double kLongSublist = 4096.0;

struct Plan {
  bool dense;  // the scan adds dense keywords' bitmaps
  uint32_t log2w;
  uint32_t unroll;
  uint32_t block_shift;
  uint32_t n_groups;
  uint32_t ht_slots;
  uint32_t threads;
  uint32_t za_len;
  size_t smem;
};

genie_status make_plan(const genie_index* idx, const genie_queries* qs, uint32_t k,
                       const genie_search_opts* o, Plan* p) {
  const uint32_t B = qs->max_bound;
  p->log2w = B <= 15 ? 2u : (B <= 255 ? 3u : 4u);
  uint32_t need = 0;
  while (need < 31 && ((uint64_t)1 << need) < idx->n_objects) ++need;
  uint32_t shift = 20 - p->log2w;  // 128 KB of Bitmap Counter
  if (o && o->block_shift) shift = o->block_shift;
  shift = std::min(shift, std::max(need, idx->chunk_shift));
  shift = std::max(shift, idx->chunk_shift);
  p->block_shift = shift;
  p->n_groups = (uint32_t)(((uint64_t)idx->n_objects + (1ull << shift) - 1) >> shift);
  uint32_t slots = (o && o->ht_slots) ? o->ht_slots : std::max(256u, dev::next_pow2(8 * k));
  if (slots & (slots - 1)) return fail(GENIE_ERR_INVALID_ARG, "genie_search: ht_slots must be a power of two");
  if (slots < 32) return fail(GENIE_ERR_INVALID_ARG, "genie_search: ht_slots must be >= 32");
  p->ht_slots = slots;
  // Dense keywords' bitmaps pay when they carry most of the batch's postings
  // (their instantiation of the scan is slower on the lists it still scans).
  p->dense = idx->n_dense && p->log2w >= 3 && !(o && (o->flags & GENIE_SEARCH_NO_DENSE)) &&
             ((o && (o->flags & GENIE_SEARCH_DENSE)) ||
              (2 * qs->n_dense_entries >= qs->n_entries && qs->n_dense_entries > 0));
  // Default shape from the mean sublist a block scans per keyword: long
  // sublists go faster with fewer, wider warps (eight 16-byte loads per lane
  // in flight, less tile bookkeeping per posting), short ones with more warps
  // and smaller tiles (less waste at the sublist ends): 1024 threads, whose
  // 64 registers the loop fits, except with 4-bit counters, whose lane
  // arithmetic needs the registers of 768.
  // (postings of dense keywords are not scanned when their bitmaps are added)
  const uint64_t scanned = qs->n_entries - (p->dense ? qs->n_dense_entries : 0);
  const double seg = qs->n_keywords ? (double)scanned / ((double)qs->n_keywords * p->n_groups) : 0.0;
  const uint32_t short_threads = p->log2w >= 3 ? 1024u : 768u;
  p->za_len = B + 2;
  int dev = 0, max_smem = 0, sm_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // Dense searches with 8-bit counters run two 512-thread blocks per SM, each
  // over half the object range, so that one block's bitmap phase overlaps the
  // other's list scan (a Zipf serving batch of 1024 queries: 21.5 -> 20.2 ms).
  bool two_per_sm = false;
  if (!(o && (o->threads || o->unroll || o->block_shift)) && p->dense && p->log2w == 3 &&
      shift > idx->chunk_shift && seg < kLongSublist) {
    const size_t half = scan_smem_bytes(p->log2w, shift - 1, slots, p->za_len, k);
    if (2 * (half + 1024) <= (size_t)sm_smem) {
      two_per_sm = true;
      shift -= 1;
      p->block_shift = shift;
      p->n_groups = (uint32_t)(((uint64_t)idx->n_objects + (1ull << shift) - 1) >> shift);
    }
  }
  p->threads = (o && o->threads) ? o->threads
             : two_per_sm        ? 512u
                                 : (seg >= kLongSublist ? 512u : short_threads);
  if (p->threads != 512 && p->threads != 768 && p->threads != 896 && p->threads != 1024)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: threads must be 512, 768, 896 or 1024");
  p->unroll = (o && o->unroll) ? o->unroll : two_per_sm ? 2u : (p->threads == 512 ? 8u : 2u);
  if (p->threads == 896 && p->unroll != 2)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: 896 threads run two loads per lane");
  if (p->threads == 512 ? (p->unroll != 2 && p->unroll != 4 && p->unroll != 8) : (p->unroll != 2 && p->unroll != 4))
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: unroll must be 2 or 4 (768 or 1024 threads), 2, 4 or 8 (512)");
  p->smem = scan_smem_bytes(p->log2w, shift, slots, p->za_len, k);
  if (p->smem + 1024 > (size_t)max_smem)
    return fail(GENIE_ERR_INVALID_ARG, "genie_search: block_shift / ht_slots need more shared memory than a block has");
  return GENIE_OK;
}

}  // namespace
}  // namespace genie
