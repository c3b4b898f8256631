/*
 * genie.h -- C ABI of the GB300 match-count top-k search library.
 *
 * The library answers batches of match-count queries (Definition 2.1, Sec.
 * 2.1) against an inverted index resident in GPU memory (Sec. 3.2) and returns
 * the top-k objects of every query, ranked by match count descending and then
 * object id ascending.  Counting and top-k selection run in CUDA kernels for
 * sm_103a through the count priority queue c-PQ (Sec. 3.3: Bitmap Counter,
 * Hash Table, ZipperArray, AuditThreshold; Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc'd or any memory the
 *     current device can address); h_* are HOST pointers.  Inputs are owned by
 *     the caller and only read.  Handles (genie_index, genie_queries,
 *     genie_server) are owned by the library and released by *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; entry points that must read a value
 *     back from the device (sizes, validation flags) synchronise that stream
 *     and say so.
 *   - Object id = row index of the object in the object CSR (uint32).
 *     Objects are SETS of keywords (Sec. 2.1): a keyword repeated inside one
 *     object is rejected.  Queries are MULTISETS of items: MC sums over items
 *     (Definition 2.1), so a keyword given twice counts twice.
 *   - Result layout: d_ids[q*k + j], d_counts[q*k + j] for rank j of query q;
 *     ranks past the number of matching objects hold id 0xFFFFFFFF and count
 *     0; d_n_valid[q] = min(k_q, #objects with MC >= 1).  Objects with MC = 0
 *     are never returned.
 *   - Every failure is reported by the returned status; no entry point traps
 *     or aborts.  genie_last_error() gives the message of the calling thread's
 *     last failure.
 *   - The device must be a compute capability 10.3 GPU (sm_103a).  Calls use
 *     the CUDA device that is current on the calling thread.
 */
#ifndef GENIE_H
#define GENIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int genie_status;
#define GENIE_OK 0
#define GENIE_ERR_INVALID_ARG 1   /* bad sizes, ids, ranges, k; nothing enqueued */
#define GENIE_ERR_OUT_OF_MEMORY 2 /* a device or host allocation failed */
#define GENIE_ERR_CUDA 3          /* a CUDA call failed (message has the CUDA error) */
#define GENIE_ERR_CAPACITY 4      /* a fixed capacity was exceeded (server slots) */
#define GENIE_ERR_TIMEOUT 5       /* a bounded device or host wait ran out */

typedef void* genie_stream; /* cudaStream_t */

typedef struct genie_index genie_index;
typedef struct genie_queries genie_queries;

/* Largest supported values (checked; larger -> GENIE_ERR_INVALID_ARG). */
#define GENIE_MAX_K 1024u          /* results per query */
#define GENIE_MAX_BOUND 4095u      /* count bound of one query (see genie_make_queries) */

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* genie_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int genie_version(void);

/* ------------------------------------------------------------------------ */
/* Index (Sec. 3.2, List Array + Position Map; Fig. 3)                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t n_objects;
  uint32_t vocab;          /* keyword ids are < vocab */
  uint64_t nnz;            /* postings = sum of object sizes */
  uint32_t max_object_len; /* largest object (keywords) */
  uint32_t chunk_shift;    /* the object-range split: 2^chunk_shift ids per chunk */
  uint32_t n_chunks;       /* ceil(n_objects / 2^chunk_shift) */
  uint32_t reserved;
  uint64_t device_bytes;   /* device memory held by the index */
  uint32_t dense_keywords; /* keywords that also have an object bitmap */
  uint32_t dense_min_df;   /* the list length from which a keyword has one */
  uint64_t dense_bytes;    /* device memory of the bitmaps and their map */
} genie_index_info;

/* Build options (genie_build_index_ex). */
typedef struct {
  uint32_t chunk_shift;    /* as for genie_build_index (0 = default) */
  uint32_t dense_min_df;   /* keywords whose list holds at least this many objects are also
                              stored as object bitmaps (n_objects bits each), which the search
                              adds whole instead of scanning the list: 0 = the default,
                              max(64, ceil(n_objects / 32)), from which a bitmap is no larger
                              than the list; GENIE_NO_DENSE = none */
} genie_index_opts;
#define GENIE_NO_DENSE 0xFFFFFFFFu

/*
 * Build the inverted index on the device from objects given as keyword sets.
 * Paper: Sec. 2.1 (objects, keywords, postings lists), Sec. 3.2 (List Array
 * holding all postings lists, Position Map from keyword to its list), Sec.
 * 3.2.1 (one-to-many position map of sublists).
 *
 *   d_obj_off  [n_objects+1] uint32, device: object o holds keywords
 *              d_obj_kw[d_obj_off[o] .. d_obj_off[o+1]-1]; d_obj_off[0] = 0,
 *              non-decreasing.
 *   d_obj_kw   [nnz] uint32, device: keyword ids < vocab, distinct within an
 *              object, any order.
 *   n_objects  1 .. 2^31; vocab 1 .. 2^31.
 *   chunk_shift  log2 of the object-id range of one sublist (the unit a
 *              search block counts on chip): 12..20, or 0 for the default 16
 *              (the 64K-object range of a block with 16-bit counters; a
 *              search's object range is at least one chunk).
 *   out        receives the index handle (library-owned; free it with
 *              genie_index_destroy).  Unchanged on failure.
 *
 * The index holds: per keyword its postings list of object ids in ascending
 * order (List Array), the list offsets (Position Map), and per keyword the
 * positions where each chunk of 2^chunk_shift object ids starts in its list
 * (sublist map).  The inputs are not referenced after the call.
 * Synchronises `stream` (sizes and validation).  Errors: INVALID_ARG for
 * malformed offsets, keyword >= vocab or a repeated keyword in an object;
 * OUT_OF_MEMORY; CUDA.
 */
genie_status genie_build_index(const uint32_t* d_obj_off, const uint32_t* d_obj_kw,
                               uint32_t n_objects, uint32_t vocab, uint32_t chunk_shift,
                               genie_stream stream, genie_index** out);

/*
 * genie_build_index with options.  Besides the List Array, keywords with
 * dense lists (opts->dense_min_df) get an object bitmap: a search adds a
 * dense keyword's bitmap to the query's counters with bitwise adders (32
 * objects per operation) instead of one counter update per posting, then
 * scans only the sparse keywords' lists.  The counts, and so every result,
 * are those of the plain scan.  opts may be NULL (the defaults of
 * genie_build_index).
 */
genie_status genie_build_index_ex(const uint32_t* d_obj_off, const uint32_t* d_obj_kw,
                                  uint32_t n_objects, uint32_t vocab, const genie_index_opts* opts,
                                  genie_stream stream, genie_index** out);

/* Release an index (NULL is ignored).  Synchronises the device. */
void genie_index_destroy(genie_index* index);

/* Sizes of an index. */
genie_status genie_index_get_info(const genie_index* index, genie_index_info* out);

/*
 * Copy the CSR of the index out (for inspection and tests).
 *   d_kw_off   [vocab+1] uint64, device: list of keyword v is
 *              d_post_ids[d_kw_off[v] .. d_kw_off[v+1]-1].
 *   d_post_ids [nnz] uint32, device: object ids, ascending within each list.
 * Either pointer may be NULL.  Asynchronous on `stream`.
 */
genie_status genie_index_export(const genie_index* index, uint64_t* d_kw_off,
                                uint32_t* d_post_ids, genie_stream stream);

/* ------------------------------------------------------------------------ */
/* Query compiler (Sec. 2.1 items -> keywords; Sec. 3.2 list look-up)        */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t n_queries;
  uint32_t max_bound;      /* largest count bound B_q over the batch */
  uint64_t n_keywords;     /* keywords after expansion, with multiplicity */
  uint64_t n_entries;      /* postings the batch scans: sum over queries of sum of df */
  uint64_t n_dense_entries; /* of them, postings of keywords with an object bitmap */
} genie_queries_info;

/*
 * Keyword queries (LSH signatures, Sec. 4.1.1; n-gram or word sets, Sec.
 * 5.1-5.2): each item is one keyword.
 *   d_q_off [n_queries+1] uint32, device; d_q_kw keywords < vocab.
 *   n_queries  1 .. 2^24.
 * The count bound of query q is B_q = min(|Q|, max_object_len * max
 * multiplicity of a keyword in Q); queries with B_q > GENIE_MAX_BOUND are
 * rejected.  The handle copies what it needs; inputs are not referenced
 * after the call.  Synchronises `stream`.  Errors: INVALID_ARG (malformed
 * offsets, keyword >= vocab, bound too large), OUT_OF_MEMORY, CUDA.
 */
genie_status genie_make_queries(const genie_index* index, const uint32_t* d_q_off,
                                const uint32_t* d_q_kw, uint32_t n_queries, genie_stream stream,
                                genie_queries** out);

/*
 * Relational range queries (Example 2.1, Sec. 5.3).  The index must hold
 * keyword d*values_per_dim + v for value v of attribute d (the encoded pair of
 * Sec. 2.1).  Query q has items d_item_off[q] .. d_item_off[q+1]-1; item i is
 * (d_dim[i], [d_lo[i], d_hi[i]]) and expands to the keywords d*values_per_dim
 * + v for every v in [lo, hi] clipped to [0, values_per_dim).  A range that
 * lies outside the value domain contributes nothing; lo > hi is INVALID_ARG.
 * B_q = min(number of expanded keywords, max_object_len * items of q).
 * Synchronises `stream`.
 */
genie_status genie_compile_ranges(const genie_index* index, uint32_t values_per_dim,
                                  const uint32_t* d_item_off, const uint32_t* d_dim,
                                  const int32_t* d_lo, const int32_t* d_hi, uint32_t n_queries,
                                  genie_stream stream, genie_queries** out);

/* Release compiled queries (NULL is ignored).  The memory is freed in order
 * on the stream the queries were compiled on (stream-ordered, no device-wide
 * synchronisation): work on that stream that uses them completes first; work
 * on other streams must be finished or ordered before it by the caller. */
void genie_queries_destroy(genie_queries* queries);

genie_status genie_queries_get_info(const genie_queries* queries, genie_queries_info* out);

/*
 * Per-query facts computed by the compiler (device outputs, any may be NULL):
 *   d_bound   [n_queries] uint32: B_q;
 *   d_entries [n_queries] uint64: postings scanned = sum of df over its keywords;
 *   d_features [n_queries * 64] float: the histogram features of the
 *             k-th-count predictor (bin 0: keywords with df = 0; bin b >= 1:
 *             keywords with floor(log2 df) = b-1, clipped to 63), each count
 *             scaled by 1/32.
 * Asynchronous on `stream`.
 */
genie_status genie_queries_export(const genie_queries* queries, uint32_t* d_bound,
                                  uint64_t* d_entries, float* d_features, genie_stream stream);

/* ------------------------------------------------------------------------ */
/* Search (Sec. 3.2 scan + Sec. 3.3 c-PQ, Algorithm 1, Theorem 3.1)          */
/* ------------------------------------------------------------------------ */

typedef struct {
  /* Per-query seed of the AuditThreshold (device, [n_queries] uint32, or
   * NULL for the paper's start value 1).  A seed s_q > 1 closes the Gate below
   * s_q; results stay exact when s_q <= the true k-th count.  With seeds the
   * search verifies every query and reruns the ones it cannot certify with
   * s = 1 (this synchronises `stream` once to read the rerun count). */
  const uint32_t* d_seed;
  /* Tuning (0 = automatic): log2 of object ids counted by one block, threads
   * per block (512, 768, 896 or 1024), hash-table slots per block (power of
   * two >= 32), 16-byte loads in flight per thread (2 or 4 with 768 or 1024
   * threads, 2 with 896, 2, 4 or 8 with 512; 512 threads with 2 run two
   * blocks per SM where two blocks' shared memory fits an SM).
   * genie_search_shape reports what the automatic choice is. */
  uint32_t block_shift;
  uint32_t threads;
  uint32_t ht_slots;
  uint32_t unroll;
  /* Optional diagnostics (device, NULL = skip):
   *   d_chunk_at    [n_queries * n_blocks_per_query] uint32: final
   *                 AuditThreshold of each (query, object range) block;
   *   d_stats       [8] uint64 accumulated: 0 gate passes, 1 hash-table
   *                 inserts, 2 blocks whose hash-table read-out was not
   *                 certified and fell back to a Bitmap-Counter selection,
   *                 3 seeded queries rerun, 4 blocks launched, 5 blocks that
   *                 saw a count above the query's bound (inconsistent input),
   *                 6 blocks that started without a seed and selected from
   *                 the Bitmap Counter without running the Gate. */
  uint32_t* d_chunk_at;
  unsigned long long* d_stats;
  /* Output: number of object ranges per query used (host pointer, may be NULL). */
  uint32_t* h_blocks_per_query;
  /* Optional cudaEvent_t pair (as void*, NULL = none) recorded on `stream`
   * immediately before and after the scan kernel of the first pass, so a
   * caller can time that kernel alone with cudaEventElapsedTime. */
  void* scan_event_begin;
  void* scan_event_end;
  /* GENIE_SEARCH_* flags (0 = defaults). */
  uint32_t flags;
} genie_search_opts;

/* Each object range of a query starts its AuditThreshold at 1 (or at the
 * seed) instead of at the largest k-th count of the query's ranges already
 * finished.  Results are the same either way; this exposes the per-range
 * AuditThreshold of Theorem 3.1 in d_chunk_at. */
#define GENIE_SEARCH_PER_RANGE_AT 1u

/* Ablation: count every posting into the Bitmap Counter and select each
 * range's top-k from the counters alone, with the Gate and hash table idle
 * (the dense-count-then-select design the paper compares c-PQ with, GEN-SPQ
 * of Sec. 6.1.2, with the counters on chip).  Same results. */
#define GENIE_SEARCH_NO_GATE 2u

/* Dense keywords (genie_build_index_ex) are added as object bitmaps, and
 * their lists skipped, when they carry at least half the batch's postings;
 * NO_DENSE scans every list, DENSE adds the bitmaps whatever their share.
 * Same results either way. */
#define GENIE_SEARCH_NO_DENSE 4u
#define GENIE_SEARCH_DENSE 8u

/*
 * Top-k of every query.  By default the ranges of a query share what they
 * learn: a range starts its AuditThreshold at the largest k-th count of the
 * query's ranges finished so far, which is never above the query's k-th
 * count, so no top-k object is skipped (see GENIE_SEARCH_PER_RANGE_AT).
 *   k          1 .. GENIE_MAX_K: result slots per query (row stride).
 *   d_k        NULL, or [n_queries] uint32 device per-query k_q in 1..k.
 *   opts       NULL for defaults.
 *   d_ids, d_counts [n_queries * k] uint32, d_n_valid [n_queries] uint32:
 *              device outputs, written completely.
 * Enqueued on `stream`; without seeds the call does not synchronise.  Scratch
 * memory is allocated stream-ordered (cudaMallocAsync) and released before
 * return.  Searches on different streams may share one index (read-only).
 * Errors: INVALID_ARG (k, handles from another index), OUT_OF_MEMORY, CUDA.
 */
genie_status genie_search(const genie_index* index, const genie_queries* queries, uint32_t k,
                          const uint32_t* d_k, const genie_search_opts* opts, uint32_t* d_ids,
                          uint32_t* d_counts, uint32_t* d_n_valid, genie_stream stream);

/* The launch shape of the scan kernel genie_search runs for these arguments. */
typedef struct {
  uint32_t counter_bits;   /* bits per object counter: 4, 8 or 16 */
  uint32_t block_shift;    /* log2 of the object ids one block counts */
  uint32_t n_groups;       /* object ranges (blocks) per query */
  uint32_t threads;        /* threads per block */
  uint32_t unroll;         /* 16-byte loads in flight per thread */
  uint32_t ht_slots;       /* hash-table slots per block */
  uint64_t smem_bytes;     /* dynamic shared memory per block */
  uint32_t dense;          /* 1: dense keywords are added as object bitmaps */
  uint32_t reserved;
} genie_search_shape_info;

/*
 * End-to-end search from host memory: the query transfer, match and select
 * stages of one batch (Table 2) plus the copy of the results back, in one
 * call.
 *   h_q_off [n_queries+1] uint32, HOST, h_q_off[0] = 0; h_q_kw [h_q_off[n]]
 *              uint32 keywords, HOST: keyword queries as for
 *              genie_make_queries.  Pinned (page-locked) memory lets the
 *              copies run at full speed; pageable memory works too.
 *   n_queries  1 .. 2^24;  k, opts as for genie_search.
 *   h_k        NULL, or [n_queries] uint32 HOST per-query k_q in 1..k.
 *   h_ids, h_counts [n_queries * k], h_n_valid [n_queries] uint32: HOST
 *              outputs, written completely, in genie_search's layout.
 * The queries are copied to the device on `stream`, compiled, searched, and
 * the results copied back; the call synchronises `stream` and returns once
 * the results are in the host buffers.  Device memory is allocated
 * stream-ordered (cudaMallocAsync) and released before return.  Errors: as
 * for genie_make_queries and genie_search; INVALID_ARG for NULL buffers or
 * h_q_off[0] != 0.
 */
genie_status genie_search_host(const genie_index* index, const uint32_t* h_q_off,
                               const uint32_t* h_q_kw, uint32_t n_queries, uint32_t k,
                               const uint32_t* h_k, const genie_search_opts* opts, uint32_t* h_ids,
                               uint32_t* h_counts, uint32_t* h_n_valid, genie_stream stream);

/*
 * Fills *out with the shape genie_search(index, queries, k, ..., opts, ...)
 * would launch (opts may be NULL).  Host only: no device work, no
 * synchronisation.  Automatic choices: counters wide enough for the largest
 * count bound; 128 KB of counters per block; 512 threads with eight loads per
 * lane when a block's mean sublist per keyword holds at least 4096 postings,
 * else 1024 threads with two (768 with 4-bit counters); a search that adds
 * object bitmaps with 8-bit counters runs two 512-thread blocks per SM with
 * two loads per lane, each over 64 KB of counters.  Errors: INVALID_ARG
 * (NULL handles, k, handles from another index, tuning values out of range).
 */
genie_status genie_search_shape(const genie_index* index, const genie_queries* queries, uint32_t k,
                                const genie_search_opts* opts, genie_search_shape_info* out);

/* ------------------------------------------------------------------------ */
/* GEN-SPQ ablation: Count Table + bucket k-selection (Sec. 6.1.2, App. A)    */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t buckets;    /* buckets per k-selection iteration, 2..32 (0 = 16) */
  uint32_t reserved;   /* 0 */
  uint64_t max_bytes;  /* device memory for Count Tables and candidate lists
                          (0 = 8 GiB); queries run in passes that fit it */
} genie_spq_opts;

typedef struct {
  uint64_t count_table_bytes_per_query;  /* 4 B per object: the dense counts */
  uint64_t list_bytes_per_query;         /* 8 B per object: explicit (count, id) keys */
  uint32_t queries_per_pass;
  uint32_t passes;
  double mean_iterations;                /* bucket-selection iterations per query */
} genie_spq_info;

/*
 * The paper's GEN-SPQ: the same index and compiled queries, counted into a
 * dense Count Table in device memory (a 32-bit count per object per query,
 * Sec. 3.3's Count Table, one block per query keyword with global atomic
 * adds, Sec. 3.2), then the top-k of each query's row by the bucket
 * k-selection of Appendix A: each iteration buckets the candidates by
 * floor((count - min) / (max - min) * buckets), keeps the buckets above the
 * one that holds the k-th largest, and repeats on that bucket; all-equal
 * candidates are taken in ascending id.  An ablation of c-PQ: results equal
 * genie_search's (count desc, id asc); it uses 12 bytes per object per query
 * of device memory instead of c-PQ's on-chip counters.
 *   k, d_k, d_ids, d_counts, d_n_valid: as for genie_search.
 *   opts: NULL for defaults.  info: NULL, or receives memory per query,
 *   queries per pass and the mean iterations (then the call synchronises).
 * Scratch is allocated stream-ordered and released before return.  Reads the
 * query offsets back (synchronises `stream` once).  Errors: INVALID_ARG,
 * CAPACITY (one query exceeds max_bytes), OUT_OF_MEMORY, CUDA.
 */
genie_status genie_search_spq(const genie_index* index, const genie_queries* queries, uint32_t k,
                              const uint32_t* d_k, const genie_spq_opts* opts, uint32_t* d_ids,
                              uint32_t* d_counts, uint32_t* d_n_valid, genie_spq_info* info,
                              genie_stream stream);

/* ------------------------------------------------------------------------ */
/* Device calibration                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  double smem_atomics_per_s;      /* integer adds of a 16-bit lane's increment to its 32-bit
                                     word, old word returned and used; per second, whole GPU */
  uint32_t sms;
  double seconds;                 /* duration of the timed launch of the first form */
  double smem_red_per_s;          /* the same adds with no value returned (red) */
  double smem_f16_atomics_per_s;  /* binary16 adds of 1.0 to a 16-bit lane, old value returned */
  double smem_f16_red_per_s;      /* binary16 adds of 1.0 with no value returned */
} genie_calibration;

/*
 * Measure the ceilings of the scan kernel's counter updates: one block per SM
 * fills a 128 KB shared counter array and every thread adds to 16-bit lanes
 * at pseudo-random positions, in the four forms above.  Synchronises the
 * device.  The paper has no counterpart.
 */
genie_status genie_calibrate(genie_calibration* out);

/* ------------------------------------------------------------------------ */
/* Batched search: one persistent, CUDA-graph-captured launch per batch      */
/* ------------------------------------------------------------------------ */
/*
 * A batch plan runs all (query, object range) c-PQ passes of a batch in one
 * persistent kernel (one block per SM pulling work items range by range,
 * queries with the most postings first inside a range; Sec. 3.2.1 treats the
 * same load-balance problem by splitting long lists) and merges each query
 * as soon as its last range is done (the Sec. 3.4 merge, on the device).  The
 * kernels are captured once into a CUDA graph; each batch refreshes a small
 * descriptor and replays it.  Results equal genie_search's.
 */
typedef struct genie_batch genie_batch;

typedef struct {
  /* shape (0 = automatic; same meaning and limits as genie_search_opts) */
  uint32_t block_shift;
  uint32_t threads;
  uint32_t unroll;
  uint32_t ht_slots;
  uint32_t blocks;      /* persistent blocks, 0 = one per SM */
  float tuned_ms;       /* genie_autotune output: best time on the sample */
  uint32_t from_cache;  /* genie_autotune output: 1 if read from the cache file */
} genie_batch_opts;

/*
 * Autotuner: runs `sample` (compiled queries representative of the workload)
 * as a persistent batch (genie_batch_create + genie_batch_run) for each
 * candidate shape -- block size x 16-byte loads in flight x object-id range
 * per block -- and writes the fastest to *out.
 * cache_path (may be NULL): a text file of "key block_shift threads unroll
 * ht_slots ms" lines; a line whose key (GPU, index sizes, count bound, k and
 * the postings-per-query scale) matches is returned without timing, and a
 * new result is appended.  Synchronises the device.
 */
genie_status genie_autotune(const genie_index* index, const genie_queries* sample, uint32_t k,
                            const char* cache_path, genie_batch_opts* out);

/*
 * New batch plan for up to max_queries queries whose count bounds are at most
 * max_bound, k results per query.  Allocates its candidate lists (max_queries
 * x ranges x k x 8 bytes) and captures its graph.
 */
genie_status genie_batch_create(const genie_index* index, uint32_t max_queries, uint32_t max_bound,
                                uint32_t k, const genie_batch_opts* opts, genie_batch** out);
genie_status genie_batch_get_info(const genie_batch* batch, genie_batch_opts* out);
void genie_batch_destroy(genie_batch* batch);

/*
 * Run one batch: results as genie_search (row stride = the plan's k; d_k as
 * in genie_search, checked with one synchronisation).  Enqueued on `stream`;
 * one plan runs one batch at a time, so issue the runs of a plan on one
 * stream.  GENIE_ERR_CAPACITY if the batch exceeds max_queries or max_bound.
 */
genie_status genie_batch_run(genie_batch* batch, const genie_queries* queries, const uint32_t* d_k,
                             uint32_t* d_ids, uint32_t* d_counts, uint32_t* d_n_valid,
                             genie_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving loop with continuous batching (not in the paper)                  */
/* ------------------------------------------------------------------------ */
/*
 * A server keeps the index resident and answers requests (host keyword
 * multisets with their own k) submitted at any time.  A worker thread keeps up
 * to `streams` batches in flight on their own CUDA streams; whenever one
 * finishes, the queued requests that fit are admitted into the next batch,
 * so requests arriving while others run overlap with them on the device.
 * Admission is by device memory: each in-flight request holds, until its
 * batch completes, the bytes it occupies in its launch slot's buffers --
 * request_bytes_base (its per-query words, its result rows, its rows of
 * per-range candidate lists and count histogram) plus 4 bytes per keyword.
 * The Bitmap Counters themselves (Sec. 3.3.1) live in shared memory of the
 * blocks that count them; their n_objects x W / 8 bytes per query are
 * reported (bc_bytes_in_flight), not charged.  Results equal genie_search's
 * for the same query.  Device memory is allocated once at creation (streams
 * x slot_bytes); the loop itself neither allocates nor synchronises per
 * batch.
 */
typedef struct genie_server genie_server;

typedef struct {
  uint64_t mem_budget_bytes;   /* device bytes all in-flight requests may hold (0 = the
                                  slots' total, streams x slot_bytes) */
  uint32_t reserved;           /* 0 */
  uint32_t max_batch;          /* queries per launch (default 256) */
  uint32_t max_query_keywords; /* keywords per request (default 4096) */
  uint32_t k_max;              /* largest k of a request (default 100) */
  uint32_t streams;            /* batches in flight, 1..8 (default 2) */
  uint32_t queue_capacity;     /* queued requests (default 65536) */
} genie_server_opts;

typedef struct {
  uint64_t tag;        /* the caller's tag */
  uint32_t k;          /* the request's k */
  uint32_t n_valid;    /* results written (ranks past it are padding) */
  double t_submit;     /* genie_server_clock() at submission */
  double t_done;       /* genie_server_clock() when the worker saw the batch finish */
} genie_result_info;

typedef struct {
  uint64_t launches;               /* batches launched */
  uint64_t queries;                /* queries launched */
  uint64_t deferred_admissions;    /* requests that waited for the memory budget */
  uint64_t max_queries_in_flight;  /* largest number of queries on the device at once */
  uint64_t pending;                /* queued now */
  uint64_t reserved_bytes;         /* device bytes held by in-flight requests now */
  uint64_t slot_bytes;             /* device memory of one launch slot */
  uint64_t request_bytes_base;     /* slot bytes of one request besides its keywords */
  uint64_t mem_budget_bytes;       /* the budget in force */
  uint64_t bc_bytes_in_flight;     /* Bitmap-Counter bytes of the in-flight queries */
} genie_server_stats;

/* Monotonic clock of the server, in seconds. */
double genie_server_clock(void);

/* Start a server on `index` (which must outlive it).  opts may be NULL. */
genie_status genie_server_create(const genie_index* index, const genie_server_opts* opts,
                                 genie_server** out);

/* Finish all admitted work, stop the worker and free the server. */
void genie_server_destroy(genie_server* server);

/* Queue one request: h_kw[n_kw] host keywords (< vocab), 1 <= k <= k_max.
 * The keywords are copied.  GENIE_ERR_CAPACITY if the queue is full or one
 * query's counters exceed the whole budget; INVALID_ARG for bad input. */
genie_status genie_server_submit(genie_server* server, const uint32_t* h_kw, uint32_t n_kw,
                                 uint32_t k, uint64_t tag);

/* Completed requests, oldest first: up to max_results, waiting at most
 * timeout_us for the first.  h_ids / h_counts hold max_results rows of
 * k_max entries (the first k of row j are request j's results). */
genie_status genie_server_poll(genie_server* server, uint32_t max_results, uint32_t timeout_us,
                               genie_result_info* h_info, uint32_t* h_ids, uint32_t* h_counts,
                               uint32_t* n_out);

genie_status genie_server_get_stats(genie_server* server, genie_server_stats* out);

/* Open-loop load replay on an otherwise idle server: request i (keywords
 * h_q_kw[h_q_off[i] .. h_q_off[i+1]-1], k = h_k[i]) is submitted h_arrival_s[i]
 * seconds after the call starts; the call returns when all n completed.
 * h_latency_s[i] = completion time - scheduled arrival; results go to row i
 * of h_ids / h_counts ([n x k_max]) and h_n_valid[i].  GENIE_ERR_TIMEOUT if
 * requests are still open after timeout_ms. */
genie_status genie_server_replay(genie_server* server, const uint32_t* h_q_off,
                                 const uint32_t* h_q_kw, const uint32_t* h_k,
                                 const double* h_arrival_s, uint32_t n, uint32_t timeout_ms,
                                 double* h_latency_s, uint32_t* h_ids, uint32_t* h_counts,
                                 uint32_t* h_n_valid);

/* ------------------------------------------------------------------------ */
/* k-th-count predictor: a learned AuditThreshold seed (not in the paper)    */
/* ------------------------------------------------------------------------ */
/*
 * A 64-128-1 ReLU network predicts each query's k-th match count from the
 * query's feature histogram (genie_queries_export).  Its prediction seeds
 * the AuditThreshold of Algorithm 1 through genie_search_opts.d_seed; the
 * seeded search stays exact (it verifies every query and reruns the ones it
 * cannot certify), so the network only changes how much Gate work a search
 * does.  Parameters theta = [W1 (128 x 64, row-major: W1[j*64 + i]) | b1
 * (128) | w2 (128) | b2 (1)], genie_mlp_num_params() floats.  The library
 * keeps float32 masters (and Adam state) and bfloat16 copies of W1 and w2;
 * forward and backward use the bfloat16 weights with float32 accumulation:
 *   y = w2 . relu(W1 x + b1) + b2,  loss = mean 0.5 (y - t)^2.
 */
typedef struct genie_mlp genie_mlp;

uint32_t genie_mlp_num_params(void);

/* New network, He-uniform weights from `seed`, zero biases and Adam state. */
genie_status genie_mlp_create(uint64_t seed, genie_stream stream, genie_mlp** out);
void genie_mlp_destroy(genie_mlp* mlp);

/* Copy float32 parameters in (d_theta, device) / out; set also resets Adam. */
genie_status genie_mlp_set_params(genie_mlp* mlp, const float* d_theta, genie_stream stream);
genie_status genie_mlp_get_params(const genie_mlp* mlp, float* d_theta, genie_stream stream);

/* d_y[n] = network(d_x[n*64 ..]) for n samples (device arrays). */
genie_status genie_mlp_forward(const genie_mlp* mlp, const float* d_x, uint32_t n, float* d_y,
                               genie_stream stream);

/* Gradient of the mean loss over the n samples (d_x, targets d_t) into the
 * network's gradient buffer; if d_grad != NULL also copies it out there
 * ([num_params] floats, then the summed squared error). */
genie_status genie_mlp_gradients(genie_mlp* mlp, const float* d_x, const float* d_t, uint32_t n,
                                 float* d_grad, genie_stream stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradients. */
genie_status genie_mlp_adam_step(genie_mlp* mlp, float lr, genie_stream stream);

/* `epochs` passes of mini-batch Adam over (d_x, d_t) in order; h_loss (may be
 * NULL) receives the final mean loss over all n samples (synchronises). */
genie_status genie_mlp_train(genie_mlp* mlp, const float* d_x, const float* d_t, uint32_t n,
                             uint32_t epochs, uint32_t batch, float lr, float* h_loss,
                             genie_stream stream);

/* AuditThreshold seeds for compiled queries:
 * d_seed[q] = clamp(floor(y_q - margin), 1, B_q + 1), y_q = network(features of q). */
genie_status genie_mlp_seeds(genie_mlp* mlp, const genie_queries* queries, float margin,
                             uint32_t* d_seed, genie_stream stream);

/*
 * genie_search without any device allocation.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory while
 * they answer queries: a process under a hard memory budget, a host program
 * whose framework owns every device allocation through its own pool, or a
 * latency-critical loop that must not pay for (or fail on) an allocation.
 *
 * Same arguments, results and errors as genie_search, with these differences:
 *   - Scratch lives in one fixed 16 MiB device array inside the library
 *     (held on every GPU that loads the library until the process exits).
 *     A call needs n_queries x (object ranges per query) x k x 8 bytes of it;
 *     larger calls return GENIE_ERR_CAPACITY with the sizes in the message
 *     (split the batch, or use genie_search).  Object ranges per query =
 *     ceil(n_objects / 2^16) for 16-bit counters (B_q > 255),
 *     ceil(n_objects / 2^17) for 8-bit, ceil(n_objects / 2^18) for 4-bit,
 *     unless opts->block_shift sets it.
 *   - opts->d_seed must be NULL (seeded searches rerun queries and need
 *     genie_search); opts is otherwise honoured.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device, with that device current).
 *     Make that first call before any stream capture on that device.  The
 *     address is kept for the life of the process: after cudaDeviceReset on
 *     a device, this entry point must not be used on that device again.
 *   - Every call uses the same array.  Calls whose work overlaps on the GPU
 *     (different streams, or different host threads) race on it; serialise
 *     them, e.g. by issuing them on one stream.
 * The function itself calls no cudaMalloc, cudaFree or other allocating
 * routine.  With d_k it synchronises `stream` once to validate the per-query k.
 */
genie_status genie_search_noalloc(const genie_index* index, const genie_queries* queries,
                                  uint32_t k, const uint32_t* d_k, const genie_search_opts* opts,
                                  uint32_t* d_ids, uint32_t* d_counts, uint32_t* d_n_valid,
                                  genie_stream stream);

/* ------------------------------------------------------------------------ */
/* Multiple loadings (Sec. 3.4; Tables 3-4): an index in parts held in host  */
/* memory                                                                    */
/* ------------------------------------------------------------------------ */

/*
 * When the index of all objects does not fit in device memory, the objects
 * are split into parts by id; each part gets its own index, the parts wait in
 * (pinned) host memory, and a query batch is run against the parts one after
 * the other, its per-part top-k lists being merged (Sec. 3.4).  A part store
 * keeps two device slots sized for its largest part; while the batch runs on
 * part p, part p + 1 is copied into the other slot on a second stream.
 */
typedef struct genie_parts genie_parts;

typedef struct {
  uint32_t n_parts;
  uint32_t vocab;
  uint32_t n_objects;       /* one past the largest global object id */
  uint32_t reserved;
  uint64_t host_bytes;      /* pinned host memory held by the parts */
  uint64_t max_part_bytes;  /* bytes of the largest part (one device slot) */
} genie_parts_info;

/* An empty part store (library-owned; free it with genie_parts_destroy). */
genie_status genie_parts_create(genie_parts** out);

/* Release a part store and its host and device memory (NULL is ignored).
   Synchronises the device. */
void genie_parts_destroy(genie_parts* parts);

/*
 * Append a part: copy `index` (built by genie_build_index over the part's
 * objects, numbered 0 .. n - 1) into new pinned host memory; its objects get
 * the global ids id_base .. id_base + n - 1.  The index is not changed and
 * may be destroyed after the call.  Parts must be added in ascending,
 * disjoint id ranges and share one vocabulary; id_base + n must stay below
 * 2^32 - 1.  When the index's object ranges hold at most 2^16 ids
 * (chunk_shift <= 16), the part keeps each id as its 16-bit place in its
 * range, and the search rebuilds the ids on the device from the sublist map
 * (half the List Array's host memory and copy bytes).  Synchronises `stream`.
 * Errors: INVALID_ARG (order, overlap, vocabulary, id range), OUT_OF_MEMORY,
 * CUDA.
 */
genie_status genie_parts_add(genie_parts* parts, const genie_index* index, uint32_t id_base,
                             genie_stream stream);

genie_status genie_parts_get_info(const genie_parts* parts, genie_parts_info* out);

/*
 * Top-k of every query over all parts.
 *   d_q_off [n_queries+1], d_q_kw: keyword queries, as for genie_make_queries
 *                (device; read once per part).
 *   k, d_k, d_ids, d_counts, d_n_valid: as for genie_search; ids are global.
 * Each part is loaded into a device slot (the next one overlapped with the
 * search of the one before), its queries are compiled and searched as by
 * genie_make_queries + genie_search, and the per-part lists are merged on
 * the device.  Part p goes to slot p mod 2, and a part still in its slot
 * from the call before is not copied again: with one or two parts, only the
 * first call copies.  With an even number of parts, a call loads part 0 into
 * its slot while it searches the last part, so the next call starts without
 * a copy; each call still copies every part once when there are more than
 * two.  Results equal those of one index
 * over all objects: ids in (count desc, id asc) order, unused slots id
 * 0xFFFFFFFF and count 0.  Synchronises `stream` once per part (the query
 * compile) and waits for the copy stream before it returns.  Calls on one
 * store must not overlap (they share its device slots).  Errors: as for
 * genie_make_queries and genie_search; INVALID_ARG if the store has no part.
 */
genie_status genie_parts_search(genie_parts* parts, const uint32_t* d_q_off, const uint32_t* d_q_kw,
                                uint32_t n_queries, uint32_t k, const uint32_t* d_k,
                                uint32_t* d_ids, uint32_t* d_counts, uint32_t* d_n_valid,
                                genie_stream stream);

/*
 * Exact merge of per-part top-k lists on the host: the result merge of the
 * multiple-loading method (Sec. 3.4, Table 4), and the exchange step of a
 * search whose objects are sharded over several GPUs (each searches its
 * shard; the lists meet on one host).  No device work.
 *   h_ids[p], h_counts[p] [n_queries * k_part] uint32, HOST: part p's
 *              results with GLOBAL object ids, as genie_search writes them
 *              (ranked by count desc, id asc; padding id 0xFFFFFFFF, count 0).
 *   k          1 .. GENIE_MAX_K result slots per query of the output.
 *   h_ids_out, h_counts_out [n_queries * k], h_n_valid [n_queries]: HOST.
 * The output is the top-k of the union of the lists under (count desc, id
 * asc): the top-k over all parts' objects when every part kept its top-k
 * (k_part >= k) and no object is in two parts.  Errors: INVALID_ARG.
 */
genie_status genie_merge_host(uint32_t n_parts, const uint32_t* const* h_ids,
                              const uint32_t* const* h_counts, uint32_t n_queries, uint32_t k_part,
                              uint32_t k, uint32_t* h_ids_out, uint32_t* h_counts_out,
                              uint32_t* h_n_valid);

/* ------------------------------------------------------------------------ */
/* Sequence search by ordered n-grams (Sec. 5.1, the shotgun-and-assembly    */
/* scheme under edit distance)                                               */
/* ------------------------------------------------------------------------ */

/*
 * Ordered n-grams of sequences as keyword sets (Sec. 5.1.1).  The window
 * S[p .. p+n-1] is read as the base-sigma number g (first character most
 * significant); its occurrence number i counts the equal windows before it
 * in S; the keyword is g * R + i (< sigma^n * R, the vocabulary to build the
 * index with).
 *   d_off [n_seqs+1], d_chars: sequences in CSR form (device), characters
 *              0 .. sigma-1 (uint8).
 *   n >= 1, sigma 2 .. 256, R >= 1, with sigma^n * R <= 2^31.
 *   d_kw_off [n_seqs+1] (device, written): keyword offsets; sequence s has
 *              max(0, len - n + 1) keywords, in window order.
 *   d_kw       (device, written): the keywords; kw_capacity entries.
 *   total      (host, written): the number of keywords.
 * Synchronises `stream`.  Errors: INVALID_ARG (parameters, a character >=
 * sigma, an n-gram occurring R or more times in one sequence), CAPACITY
 * (kw_capacity < total; d_kw_off and *total are still written), CUDA.
 */
genie_status genie_sa_grams(const uint32_t* d_off, const uint8_t* d_chars, uint32_t n_seqs,
                            uint32_t n, uint32_t sigma, uint32_t R, uint32_t* d_kw_off,
                            uint32_t* d_kw, uint64_t kw_capacity, uint64_t* total,
                            genie_stream stream);

/*
 * Verification of the K candidates of each query (Algorithm 2, Theorem 5.2).
 *   d_q_off [n_queries+1], d_q_chars: query sequences (device); every query
 *              at most max_query_len <= 512 characters.
 *   d_s_off, d_s_chars: the data sequences (device).
 *   d_cand_ids, d_cand_counts [n_queries * K], d_cand_n [n_queries]: the
 *              output of genie_search (or genie_parts_search) with k = K over
 *              the sequences' n-gram index: candidates in (count desc, id
 *              asc) order.
 *   n: the n-gram length of the index; 1 <= k <= K <= GENIE_MAX_K.
 * Per query, in candidate order, the edit distance of a candidate is used
 * until the n-gram bound of Theorem 5.1 rules out every later one (the
 * filtering bound theta = |Q| - n + 1 - n (tau_k - 1), tau_k the k-th best
 * distance so far, once k candidates were taken; Algorithm 2 is the case k =
 * 1), candidates whose length differs from |Q| by more than tau_k being
 * skipped.  Outputs:
 *   d_ids, d_ed [n_queries * k]: the k best (distance asc, then candidate
 *              order); unused slots 0xFFFFFFFF.
 *   d_n_out [n_queries]: results written (min(k, candidates)).
 *   d_certified [n_queries]: 1 when Theorem 5.2 shows these are the true top-k
 *              under edit distance: the K-th candidate's count (0 with fewer
 *              than K candidates) is below |Q| - n + 1 - tau_k * n.
 *   d_examined [n_queries]: candidates whose distance the algorithm used.
 * Enqueued on `stream`.  Errors: INVALID_ARG, CUDA.
 */
genie_status genie_sa_verify(const uint32_t* d_q_off, const uint8_t* d_q_chars, uint32_t n_queries,
                             const uint32_t* d_s_off, const uint8_t* d_s_chars,
                             const uint32_t* d_cand_ids, const uint32_t* d_cand_counts,
                             const uint32_t* d_cand_n, uint32_t K, uint32_t k, uint32_t n,
                             uint32_t max_query_len, uint32_t* d_ids, uint32_t* d_ed,
                             uint32_t* d_n_out, uint32_t* d_certified, uint32_t* d_examined,
                             genie_stream stream);

/* ------------------------------------------------------------------------ */
/* LSH keywords of points (Sec. 4.1): a point becomes an object of m keywords */
/* ------------------------------------------------------------------------ */

/*
 * Hash function i of m maps point p to keyword i * D + bucket (Sec. 4.1.2,
 * O = [r_1(h_1(p)), ..., r_m(h_m(p))]); m * D <= 2^32.  Points are float32
 * rows d_points[n_points][dim] (device); the output is d_kw[n_points][m]
 * (device), which is the object CSR of genie_build_index with offsets
 * o * m (and the query CSR of genie_make_queries).  Every floating-point step
 * is one correctly rounded binary32 operation in the order given, so the
 * keywords do not depend on the launch.  The random draws are inputs (device)
 * and stay owned by the caller.  Enqueued on `stream`.  Errors: INVALID_ARG
 * (NULL, zero sizes, m * D > 2^32, w <= 0), CUDA.
 *
 * p-stable hashing (Eqn. (plsh)): d_a[m][dim] (a_i, Gaussian for l2), d_b[m]
 * (b_i in [0, w)), bucket width w:
 *   s = fma(a_i[dim-1], p[dim-1], ... fma(a_i[1], p[1], fma(a_i[0], p[0], 0)))
 *   bucket = floor((s + b_i) / w) mod D      (non-negative residue)
 */
genie_status genie_lsh_pstable(const float* d_points, uint64_t n_points, uint32_t dim,
                               const float* d_a, const float* d_b, uint32_t m, float w, uint32_t D,
                               uint32_t* d_kw, genie_stream stream);

/*
 * Random binning for the Laplacian kernel (the case study of Sec. 4.1.3):
 * d_g[m][dim] grid cell sizes (Gamma(2, sigma) for kernel width sigma),
 * d_u[m][dim] shifts in [0, g), d_key[m] re-hash keys:
 *   c_d = floor((p[d] - u_i[d]) / g_i[d])      (saturated to int32)
 *   x = key_i; for d = 0 .. dim-1: x = mix(x ^ c_d); bucket = mix(x) mod D,
 * mix = the 32-bit finalizer lowbias32 (hash-prospector): x ^= x >> 16;
 * x *= 0x7feb352d; x ^= x >> 15; x *= 0x846ca68b; x ^= x >> 16.
 */
genie_status genie_lsh_rbh(const float* d_points, uint64_t n_points, uint32_t dim,
                           const float* d_g, const float* d_u, const uint32_t* d_key, uint32_t m,
                           uint32_t D, uint32_t* d_kw, genie_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GENIE_H */
