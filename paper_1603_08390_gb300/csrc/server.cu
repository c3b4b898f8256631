// Serving loop with continuous batching.
//
// Requests (host keyword sets with their k) enter a FIFO queue.  A worker
// thread keeps up to `streams` launches in flight: whenever a launch slot is
// free it admits queued requests into a new batch while the device memory of
// all in-flight requests stays within the budget, copies the batch to the
// device and enqueues the scan + c-PQ + merge kernels on the slot's stream,
// followed by the copy of the results back.  A request is charged the slot
// memory it occupies: its keywords, its per-query words, its result rows,
// its rows of per-range candidate lists and of the count histogram.  (The
// Bitmap Counters, the memory Sec. 3.3 charges a query, live in shared
// memory of the blocks that count them and are only reported.)  Requests that arrive while other batches run
// join the next slot that frees, so batches overlap on the device.  Nothing is
// allocated and nothing blocks per batch: completion is observed with
// cudaEventQuery.  The paper has no serving component.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace genie {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  std::vector<uint32_t> kw;
  uint64_t entries = 0;  // postings its keywords' lists hold
  uint64_t dense_entries = 0;  // of them, postings of keywords with an object bitmap
  uint32_t k = 0;
  uint32_t bound = 0;
  uint64_t tag = 0;
  uint64_t dev_bytes = 0;  // device memory it holds while in flight
  uint64_t bc_bytes = 0;   // Bitmap-Counter bytes (reported only)
  double t_submit = 0.0;
  bool deferred = false;
};

struct Done {
  uint64_t tag;
  uint32_t k, n_valid;
  double t_submit, t_done;
  std::vector<uint32_t> ids, counts;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t *q_off = nullptr, *q_kw = nullptr, *bound = nullptr, *karr = nullptr;
  uint32_t *ids = nullptr, *counts = nullptr, *n_valid = nullptr;
  unsigned long long* cand = nullptr;
  size_t cand_bytes = 0;
  uint32_t* hint = nullptr;
  uint32_t* hint_hist = nullptr;  // per-query count histograms of the finished ranges
  size_t hint_hist_words = 0;
  uint32_t *h_q_off = nullptr, *h_q_kw = nullptr, *h_bound = nullptr, *h_karr = nullptr;
  uint32_t *h_ids = nullptr, *h_counts = nullptr, *h_n_valid = nullptr;
  std::vector<Request> reqs;
  uint64_t reserved = 0;     // device bytes held by the requests of the batch
  uint64_t bc_reserved = 0;  // their Bitmap-Counter bytes
  bool busy = false;
};

}  // namespace
}  // namespace genie

struct genie_server {
  const genie_index* index = nullptr;
  genie_server_opts opts{};
  int device = 0;
  std::vector<uint64_t> kw_off;  // host copy of the list offsets (postings per request), or empty
  std::vector<genie::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<genie::Request> pending;
  std::deque<genie::Done> finished;
  uint64_t reserved = 0;        // device bytes held by in-flight requests
  uint64_t bc_reserved = 0;     // their Bitmap-Counter bytes
  uint64_t slot_bytes = 0;      // device memory of one launch slot
  uint64_t per_query_bytes = 0; // slot memory of one request besides its keywords
  std::atomic<bool> stop{false};
  std::atomic<int> error{0};
  std::thread worker;
  // statistics
  uint64_t n_launches = 0, n_queries = 0, n_deferred = 0, max_in_flight = 0;
};

using namespace genie;

namespace {

void free_slot(Slot& s) {
  if (s.stream) cudaStreamDestroy(s.stream);
  if (s.done) cudaEventDestroy(s.done);
  cudaFree(s.q_off);
  cudaFree(s.q_kw);
  cudaFree(s.bound);
  cudaFree(s.karr);
  cudaFree(s.ids);
  cudaFree(s.counts);
  cudaFree(s.n_valid);
  cudaFree(s.cand);
  cudaFree(s.hint);
  cudaFree(s.hint_hist);
  cudaFreeHost(s.h_q_off);
  cudaFreeHost(s.h_q_kw);
  cudaFreeHost(s.h_bound);
  cudaFreeHost(s.h_karr);
  cudaFreeHost(s.h_ids);
  cudaFreeHost(s.h_counts);
  cudaFreeHost(s.h_n_valid);
}

// Launch the requests in `s.reqs` on the slot's stream (worker thread).
void launch_slot(genie_server* sv, Slot& s) {
  const uint32_t n = (uint32_t)s.reqs.size(), kmax = sv->opts.k_max;
  uint32_t pos = 0, max_bound = 1;
  uint64_t entries = 0, dense_entries = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const Request& r = s.reqs[i];
    entries += r.entries;
    dense_entries += r.dense_entries;
    s.h_q_off[i] = pos;
    std::memcpy(s.h_q_kw + pos, r.kw.data(), r.kw.size() * 4);
    pos += (uint32_t)r.kw.size();
    s.h_bound[i] = r.bound;
    s.h_karr[i] = r.k;
    max_bound = std::max(max_bound, r.bound);
  }
  s.h_q_off[n] = pos;
  cudaStream_t st = s.stream;
  cudaMemcpyAsync(s.q_off, s.h_q_off, (n + 1) * 4, cudaMemcpyHostToDevice, st);
  if (pos) cudaMemcpyAsync(s.q_kw, s.h_q_kw, (size_t)pos * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.bound, s.h_bound, n * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(s.karr, s.h_karr, n * 4, cudaMemcpyHostToDevice, st);
  genie_status gs = search_raw(sv->index, s.q_off, s.q_kw, s.bound, n, max_bound, kmax, s.karr,
                               s.cand, s.cand_bytes, s.hint, s.hint_hist, s.hint_hist_words, s.ids,
                               s.counts, s.n_valid, st, entries, pos, dense_entries);
  if (gs != GENIE_OK) sv->error = gs;
  cudaMemcpyAsync(s.h_ids, s.ids, (size_t)n * kmax * 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s.h_counts, s.counts, (size_t)n * kmax * 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(s.h_n_valid, s.n_valid, n * 4, cudaMemcpyDeviceToHost, st);
  cudaEventRecord(s.done, st);
  s.busy = true;
}

void worker_loop(genie_server* sv) {
  cudaSetDevice(sv->device);
  const uint32_t kmax = sv->opts.k_max;
  const uint64_t kw_cap = (uint64_t)sv->opts.max_batch * sv->opts.max_query_keywords;
  for (;;) {
    bool progressed = false;
    // completions
    for (Slot& s : sv->slots) {
      if (!s.busy || cudaEventQuery(s.done) != cudaSuccess) continue;
      const double t = now_s();
      std::lock_guard<std::mutex> lock(sv->mu);
      for (uint32_t i = 0; i < s.reqs.size(); ++i) {
        const Request& r = s.reqs[i];
        Done d;
        d.tag = r.tag;
        d.k = r.k;
        d.n_valid = s.h_n_valid[i];
        d.t_submit = r.t_submit;
        d.t_done = t;
        d.ids.assign(s.h_ids + (size_t)i * kmax, s.h_ids + (size_t)i * kmax + r.k);
        d.counts.assign(s.h_counts + (size_t)i * kmax, s.h_counts + (size_t)i * kmax + r.k);
        sv->finished.push_back(std::move(d));
      }
      sv->reserved -= s.reserved;
      sv->bc_reserved -= s.bc_reserved;
      s.reserved = 0;
      s.bc_reserved = 0;
      s.reqs.clear();
      s.busy = false;
      progressed = true;
      sv->cv_done.notify_all();
    }
    // admissions: every free slot takes the next requests that fit the budget
    for (Slot& s : sv->slots) {
      if (s.busy) continue;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        uint64_t kw = 0;
        while (!sv->pending.empty() && s.reqs.size() < sv->opts.max_batch) {
          Request& r = sv->pending.front();
          if (sv->reserved + r.dev_bytes > sv->opts.mem_budget_bytes) {
            if (!r.deferred) ++sv->n_deferred;  // waits for in-flight queries to finish
            r.deferred = true;
            break;
          }
          if (kw + r.kw.size() > kw_cap) break;
          kw += r.kw.size();
          sv->reserved += r.dev_bytes;
          s.reserved += r.dev_bytes;
          sv->bc_reserved += r.bc_bytes;
          s.bc_reserved += r.bc_bytes;
          s.reqs.push_back(std::move(r));
          sv->pending.pop_front();
        }
        if (!s.reqs.empty()) {
          ++sv->n_launches;
          sv->n_queries += s.reqs.size();
          uint64_t in_flight = s.reqs.size();
          for (Slot& o : sv->slots) in_flight += o.busy ? o.reqs.size() : 0;
          sv->max_in_flight = std::max<uint64_t>(sv->max_in_flight, in_flight);
        }
      }
      if (!s.reqs.empty()) {
        launch_slot(sv, s);
        progressed = true;
      }
    }
    bool any_busy = false;
    for (Slot& s : sv->slots) any_busy |= s.busy;
    if (sv->stop && !any_busy) {
      std::lock_guard<std::mutex> lock(sv->mu);
      if (sv->pending.empty()) break;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lock(sv->mu);
      if (any_busy)  // device work in flight: look again shortly
        sv->cv_work.wait_for(lock, std::chrono::microseconds(20));
      else if (sv->pending.empty() && !sv->stop)
        sv->cv_work.wait_for(lock, std::chrono::milliseconds(5));
    }
  }
}

uint32_t max_multiplicity(std::vector<uint32_t> kw) {
  if (kw.empty()) return 0;
  std::sort(kw.begin(), kw.end());
  uint32_t best = 1, run = 1;
  for (size_t i = 1; i < kw.size(); ++i) {
    run = kw[i] == kw[i - 1] ? run + 1 : 1;
    best = std::max(best, run);
  }
  return best;
}

}  // namespace

extern "C" double genie_server_clock(void) { return now_s(); }

extern "C" genie_status genie_server_create(const genie_index* index, const genie_server_opts* opts,
                                            genie_server** out) {
  if (!index || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_server_create: NULL argument");
  genie_server_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.max_batch == 0) o.max_batch = 256;
  if (o.max_query_keywords == 0) o.max_query_keywords = 4096;
  if (o.k_max == 0) o.k_max = 100;
  if (o.streams == 0) o.streams = 2;
  if (o.queue_capacity == 0) o.queue_capacity = 1u << 16;
  if (o.k_max > GENIE_MAX_K || o.streams > 8 || o.max_batch > 65536 || o.max_query_keywords > 65535)
    return fail(GENIE_ERR_INVALID_ARG, "genie_server_create: options out of range");
  genie_server* sv = new (std::nothrow) genie_server();
  if (!sv) return fail(GENIE_ERR_OUT_OF_MEMORY, "genie_server_create: host allocation");
  sv->index = index;
  sv->opts = o;
  cudaGetDevice(&sv->device);
  const size_t cand = search_scratch_bytes(index, 4095, o.max_batch, o.k_max);  // widest counters
  const size_t kw_cap = (size_t)o.max_batch * o.max_query_keywords;
  sv->slots.resize(o.streams);
  cudaError_t e = cudaSuccess;
  // The host copy of the list offsets only steers the launch shape (postings
  // per request); without the host memory for it the server runs the default.
  try {
    sv->kw_off.resize((size_t)index->vocab + 1);
  } catch (...) {
    std::vector<uint64_t>().swap(sv->kw_off);
  }
  if (!sv->kw_off.empty())
    e = cudaMemcpy(sv->kw_off.data(), index->kw_off, sv->kw_off.size() * 8, cudaMemcpyDeviceToHost);
  for (Slot& s : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&s.q_off, (o.max_batch + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.q_kw, kw_cap * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.bound, o.max_batch * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.karr, o.max_batch * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.ids, (size_t)o.max_batch * o.k_max * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.counts, (size_t)o.max_batch * o.k_max * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.n_valid, o.max_batch * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.cand, cand);
    if (e == cudaSuccess) e = cudaMalloc(&s.hint, o.max_batch * 4);
    const size_t hist_words =
        (size_t)o.max_batch * (std::min<uint32_t>(o.max_query_keywords, GENIE_MAX_BOUND) + 2);
    if (e == cudaSuccess && hist_words * 4 <= kHintHistMaxBytes) {
      e = cudaMalloc(&s.hint_hist, hist_words * 4);
      s.hint_hist_words = hist_words;
    }
    s.cand_bytes = cand;
    sv->slot_bytes = (uint64_t)(o.max_batch + 1) * 4 + (uint64_t)kw_cap * 4 + 3ull * o.max_batch * 4 +
                     2ull * o.max_batch * o.k_max * 4 + o.max_batch * 4ull + cand +
                     s.hint_hist_words * 4;
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_q_off, (o.max_batch + 1) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_q_kw, kw_cap * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_bound, o.max_batch * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_karr, o.max_batch * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_ids, (size_t)o.max_batch * o.k_max * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_counts, (size_t)o.max_batch * o.k_max * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_n_valid, o.max_batch * 4);
  }
  if (e != cudaSuccess || cand == 0) {
    for (Slot& s : sv->slots) free_slot(s);
    delete sv;
    return e != cudaSuccess ? fail_cuda(e, "genie_server_create")
                            : fail(GENIE_ERR_INVALID_ARG, "genie_server_create: cannot plan the search");
  }
  // a request's share of a slot: its keywords, then one row of everything
  // else the slot holds per query
  const uint64_t hist_row = sv->slots.empty() ? 0 : sv->slots[0].hint_hist_words / o.max_batch;
  sv->per_query_bytes = 20 + 8ull * o.k_max + cand / o.max_batch + hist_row * 4;
  if (sv->opts.mem_budget_bytes == 0) sv->opts.mem_budget_bytes = sv->slot_bytes * o.streams;
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return GENIE_OK;
}

extern "C" void genie_server_destroy(genie_server* sv) {
  if (!sv) return;
  sv->stop = true;
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (Slot& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    free_slot(s);
  }
  delete sv;
}

extern "C" genie_status genie_server_submit(genie_server* sv, const uint32_t* h_kw, uint32_t n_kw,
                                            uint32_t k, uint64_t tag) {
  if (!sv || (n_kw && !h_kw)) return fail(GENIE_ERR_INVALID_ARG, "genie_server_submit: NULL argument");
  if (k == 0 || k > sv->opts.k_max) return fail(GENIE_ERR_INVALID_ARG, "genie_server_submit: k must be in 1..k_max");
  if (n_kw > sv->opts.max_query_keywords)
    return fail(GENIE_ERR_INVALID_ARG, "genie_server_submit: query longer than max_query_keywords");
  Request r;
  r.kw.assign(h_kw, h_kw + n_kw);
  for (uint32_t v : r.kw) {
    if (v >= sv->index->vocab) return fail(GENIE_ERR_INVALID_ARG, "genie_server_submit: keyword >= vocab");
    if (!sv->kw_off.empty()) {
      const uint64_t df = sv->kw_off[v + 1] - sv->kw_off[v];
      r.entries += df;
      if (sv->index->n_dense && df >= sv->index->dense_min_df) r.dense_entries += df;
    }
  }
  // count bound as in genie_make_queries
  const uint64_t cap = (uint64_t)sv->index->max_object_len * max_multiplicity(r.kw);
  r.bound = (uint32_t)std::min<uint64_t>(n_kw, cap);
  if (r.bound > GENIE_MAX_BOUND)
    return fail(GENIE_ERR_INVALID_ARG, "genie_server_submit: count bound exceeds GENIE_MAX_BOUND");
  // the counter width the search picks for this bound (reported, Sec. 3.3.1)
  const uint32_t width = r.bound <= 15 ? 4 : (r.bound <= 255 ? 8 : 16);
  r.bc_bytes = ((uint64_t)sv->index->n_objects * width + 7) / 8;
  r.dev_bytes = sv->per_query_bytes + 4ull * n_kw;
  if (r.dev_bytes > sv->opts.mem_budget_bytes)
    return fail(GENIE_ERR_CAPACITY, "genie_server_submit: one request needs more device memory than the budget");
  r.k = k;
  r.tag = tag;
  r.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->pending.size() >= sv->opts.queue_capacity)
      return fail(GENIE_ERR_CAPACITY, "genie_server_submit: request queue is full");
    sv->pending.push_back(std::move(r));
  }
  sv->cv_work.notify_one();
  return GENIE_OK;
}

extern "C" genie_status genie_server_poll(genie_server* sv, uint32_t max_results, uint32_t timeout_us,
                                          genie_result_info* h_info, uint32_t* h_ids,
                                          uint32_t* h_counts, uint32_t* n_out) {
  if (!sv || !n_out || (max_results && (!h_info || !h_ids || !h_counts)))
    return fail(GENIE_ERR_INVALID_ARG, "genie_server_poll: NULL argument");
  *n_out = 0;
  if (sv->error) return fail(sv->error.load(), "genie_server_poll: a launch failed");
  std::unique_lock<std::mutex> lock(sv->mu);
  if (sv->finished.empty() && timeout_us)
    sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us),
                         [&] { return !sv->finished.empty(); });
  uint32_t n = 0;
  const uint32_t kmax = sv->opts.k_max;
  while (n < max_results && !sv->finished.empty()) {
    Done& d = sv->finished.front();
    h_info[n].tag = d.tag;
    h_info[n].k = d.k;
    h_info[n].n_valid = d.n_valid;
    h_info[n].t_submit = d.t_submit;
    h_info[n].t_done = d.t_done;
    std::memcpy(h_ids + (size_t)n * kmax, d.ids.data(), d.k * 4);
    std::memcpy(h_counts + (size_t)n * kmax, d.counts.data(), d.k * 4);
    sv->finished.pop_front();
    ++n;
  }
  *n_out = n;
  return GENIE_OK;
}

extern "C" genie_status genie_server_get_stats(genie_server* sv, genie_server_stats* out) {
  if (!sv || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  out->launches = sv->n_launches;
  out->queries = sv->n_queries;
  out->deferred_admissions = sv->n_deferred;
  out->max_queries_in_flight = sv->max_in_flight;
  out->pending = sv->pending.size();
  out->reserved_bytes = sv->reserved;
  out->slot_bytes = sv->slot_bytes;
  out->request_bytes_base = sv->per_query_bytes;
  out->mem_budget_bytes = sv->opts.mem_budget_bytes;
  out->bc_bytes_in_flight = sv->bc_reserved;
  return GENIE_OK;
}

extern "C" genie_status genie_server_replay(genie_server* sv, const uint32_t* h_q_off,
                                            const uint32_t* h_q_kw, const uint32_t* h_k,
                                            const double* h_arrival_s, uint32_t n,
                                            uint32_t timeout_ms, double* h_latency_s,
                                            uint32_t* h_ids, uint32_t* h_counts,
                                            uint32_t* h_n_valid) {
  if (!sv || !h_q_off || !h_k || !h_arrival_s || !h_latency_s || !h_ids || !h_counts || !h_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_server_replay: NULL argument");
  const uint32_t kmax = sv->opts.k_max;
  std::vector<double> due(n);
  std::atomic<int> submit_err{0};
  const double t0 = now_s();
  // open loop: request i is submitted at t0 + arrival_s[i] whatever the server does
  std::thread feeder([&] {
    for (uint32_t i = 0; i < n; ++i) {
      const double t = t0 + h_arrival_s[i];
      for (;;) {
        const double dt = t - now_s();
        if (dt <= 0) break;
        if (dt > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(dt - 1e-4));
      }
      due[i] = t;
      genie_status st;
      do {  // a full queue only delays the submission (the latency keeps counting)
        st = genie_server_submit(sv, h_q_kw + h_q_off[i], h_q_off[i + 1] - h_q_off[i], h_k[i], i);
        if (st == GENIE_ERR_CAPACITY) std::this_thread::sleep_for(std::chrono::microseconds(50));
      } while (st == GENIE_ERR_CAPACITY && now_s() - t0 < timeout_ms * 1e-3);
      if (st != GENIE_OK) {
        submit_err = st;
        return;
      }
    }
  });
  std::vector<genie_result_info> info(256);
  std::vector<uint32_t> ids((size_t)256 * kmax), cnt((size_t)256 * kmax);
  uint32_t got = 0;
  genie_status st = GENIE_OK;
  while (got < n && st == GENIE_OK) {
    if (submit_err) {
      st = (genie_status)submit_err.load();
      break;
    }
    if (now_s() - t0 > timeout_ms * 1e-3) {
      st = fail(GENIE_ERR_TIMEOUT, "genie_server_replay: requests still open at the time limit");
      break;
    }
    uint32_t m = 0;
    st = genie_server_poll(sv, 256, 2000, info.data(), ids.data(), cnt.data(), &m);
    for (uint32_t j = 0; j < m && st == GENIE_OK; ++j) {
      const uint64_t i = info[j].tag;
      h_latency_s[i] = info[j].t_done - due[i];
      h_n_valid[i] = info[j].n_valid;
      std::memcpy(h_ids + i * kmax, ids.data() + (size_t)j * kmax, info[j].k * 4);
      std::memcpy(h_counts + i * kmax, cnt.data() + (size_t)j * kmax, info[j].k * 4);
      for (uint32_t c = info[j].k; c < kmax; ++c) {
        h_ids[i * kmax + c] = 0xFFFFFFFFu;
        h_counts[i * kmax + c] = 0;
      }
      ++got;
    }
  }
  feeder.join();
  return st;
}
