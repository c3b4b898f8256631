// Batched search in one persistent, CUDA-graph-captured launch, and the
// autotuner that picks its tile shapes and work split.
//
// A batch of Q queries against an index split into G object ranges is Q x G
// work items, each the c-PQ pass of one (query, range) (cpq_item).  One block
// per SM pulls items from a device counter range by range, so that the
// blocks resident at one time share one range of the List Array in L2.  The
// per-range top-k lists are merged by a second kernel (Sec. 3.4, on the
// device).  Both launches are captured once into a CUDA graph; each batch
// sets the kernels' arguments on the graph's nodes and replays it.  The
// scan arguments are kernel parameters, as in the one-block-per-item search,
// so an item runs the same code as in scan_cpq_kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "cpq_device.cuh"
#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

// Per-batch arguments of the two captured kernels (set on their graph nodes).
struct BatchDesc {
  ScanArgs scan;
  MergeArgs merge;
};

// Persistent blocks: each pulls the next (query, range) item from *work until
// the batch is done.
template <int LOG2W, int U, int THREADS, bool DENSE>
__global__ void __launch_bounds__(THREADS, 1)
    batch_cpq_kernel(const __grid_constant__ ScanArgs SA, uint32_t* __restrict__ work) {
  extern __shared__ uint4 smem_raw[];
  __shared__ BlockShared S;
  const uint32_t Q = SA.n_sel;
  const uint32_t total = Q * SA.n_groups;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t item = S.item;
    if (item >= total) break;
    const uint32_t g = item / Q;
    cpq_item<LOG2W, U, DENSE>(SA, item - g * Q, g, smem_raw, S);
    __syncthreads();
  }
}

// launch = false only raises the kernel's shared-memory limit (done before a
// stream capture begins)
template <int LOG2W, int U, int THREADS>
cudaError_t launch_batch(uint32_t* work, const BatchDesc& args, uint32_t blocks, size_t smem,
                         cudaStream_t s, bool launch, bool dense) {
  auto kern = (LOG2W >= 3 && dense) ? batch_cpq_kernel<LOG2W, U, THREADS, LOG2W >= 3>
                                    : batch_cpq_kernel<LOG2W, U, THREADS, false>;
  if (!launch) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<blocks, THREADS, smem, s>>>(args.scan, work);
  return cudaGetLastError();
}

template <int LOG2W>
cudaError_t batch_width(uint32_t* d, const BatchDesc& args, uint32_t blocks, size_t smem,
                        uint32_t threads, uint32_t unroll, cudaStream_t s, bool launch, bool dense) {
  if (threads == 512) return unroll == 8 ? launch_batch<LOG2W, 8, 512>(d, args, blocks, smem, s, launch, dense)
                                         : launch_batch<LOG2W, 4, 512>(d, args, blocks, smem, s, launch, dense);
  if (threads == 768) return unroll == 4 ? launch_batch<LOG2W, 4, 768>(d, args, blocks, smem, s, launch, dense)
                                         : launch_batch<LOG2W, 2, 768>(d, args, blocks, smem, s, launch, dense);
  if (threads == 896) return launch_batch<LOG2W, 2, 896>(d, args, blocks, smem, s, launch, dense);
  return unroll == 4 ? launch_batch<LOG2W, 4, 1024>(d, args, blocks, smem, s, launch, dense)
                     : launch_batch<LOG2W, 2, 1024>(d, args, blocks, smem, s, launch, dense);
}

cudaError_t batch_dispatch(const genie_batch* b, bool launch);

std::string tune_key(const genie_index* idx, const genie_queries* qs, uint32_t k) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  // postings per query, bucketed by powers of two, describes the workload
  const double epq = qs->n_queries ? (double)qs->n_entries / qs->n_queries : 0.0;
  std::ostringstream os;
  os << prop.name << "|sm" << prop.multiProcessorCount << "|N" << idx->n_objects << "|V"
     << idx->vocab << "|nnz" << idx->nnz << "|cs" << idx->chunk_shift << "|B" << qs->max_bound
     << "|k" << k << "|epq2^" << (int)std::floor(std::log2(std::max(1.0, epq)));
  std::string key = os.str();
  std::replace(key.begin(), key.end(), ' ', '_');
  return key;
}

}  // namespace
}  // namespace genie

struct genie_batch {
  const genie_index* index = nullptr;
  int device = 0;
  uint32_t max_queries = 0, max_bound = 0, k = 0;
  uint32_t log2w = 0, block_shift = 0, n_groups = 0, threads = 0, unroll = 0, ht_slots = 0;
  uint32_t blocks = 0;
  bool dense = false;      // the instantiation being captured adds dense keywords' bitmaps
  bool can_dense = false;  // the index has object bitmaps: a second graph adds them
  size_t smem = 0;
  genie::BatchDesc host_desc{};  // the arguments' fixed part, as captured
  unsigned long long* cand = nullptr;
  uint32_t* counters = nullptr;  // [0] work, [1 ..] per-query seeds, then histograms
  uint64_t counter_words = 0;
  cudaStream_t capture_stream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};      // [1]: dense keywords as bitmaps
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t node[2] = {nullptr, nullptr};   // the persistent kernel's node of each graph
  cudaKernelNodeParams node_params[2];            // its launch, as captured
  cudaGraphNode_t mnode[2] = {nullptr, nullptr};  // the merge kernel's node
  cudaKernelNodeParams mnode_params[2];
};

using namespace genie;

namespace genie {
namespace {
cudaError_t batch_dispatch(const genie_batch* b, bool launch) {
  cudaStream_t s = b->capture_stream;
  return b->log2w == 2 ? batch_width<2>(b->counters, b->host_desc, b->blocks, b->smem, b->threads, b->unroll, s, launch, b->dense)
       : b->log2w == 3 ? batch_width<3>(b->counters, b->host_desc, b->blocks, b->smem, b->threads, b->unroll, s, launch, b->dense)
                       : batch_width<4>(b->counters, b->host_desc, b->blocks, b->smem, b->threads, b->unroll, s, launch, b->dense);
}
}  // namespace
}  // namespace genie

namespace {
void free_batch(genie_batch* b) {
  if (!b) return;
  for (int i = 0; i < 2; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
  }
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  cudaFree(b->cand);

  cudaFree(b->counters);
  delete b;
}
}  // namespace

extern "C" genie_status genie_batch_create(const genie_index* index, uint32_t max_queries,
                                           uint32_t max_bound, uint32_t k,
                                           const genie_batch_opts* opts, genie_batch** out) {
  if (!index || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_batch_create: NULL argument");
  if (max_queries == 0 || max_queries > (1u << 24))
    return fail(GENIE_ERR_INVALID_ARG, "genie_batch_create: max_queries must be in 1..2^24");
  if (max_bound == 0 || max_bound > GENIE_MAX_BOUND)
    return fail(GENIE_ERR_INVALID_ARG, "genie_batch_create: max_bound must be in 1..GENIE_MAX_BOUND");
  if (k == 0 || k > GENIE_MAX_K) return fail(GENIE_ERR_INVALID_ARG, "genie_batch_create: k must be in 1..GENIE_MAX_K");
  genie_queries probe;  // only the fields make_plan reads
  probe.index = index;
  probe.max_bound = max_bound;
  genie_search_opts so;
  std::memset(&so, 0, sizeof(so));
  if (opts) {
    so.block_shift = opts->block_shift;
    so.threads = opts->threads;
    so.unroll = opts->unroll;
    so.ht_slots = opts->ht_slots;
  }
  Plan p;
  genie_status st = make_plan(index, &probe, k, &so, &p);
  if (st != GENIE_OK) return st;
  if (p.threads == 512 && p.unroll == 2)
    return fail(GENIE_ERR_INVALID_ARG, "genie_batch_create: 512 threads run 4 or 8 loads per lane in a batch");
  genie_batch* b = new (std::nothrow) genie_batch();
  if (!b) return fail(GENIE_ERR_OUT_OF_MEMORY, "genie_batch_create: host allocation");
  cudaGetDevice(&b->device);
  b->index = index;
  b->max_queries = max_queries;
  b->max_bound = max_bound;
  b->k = k;
  b->log2w = p.log2w;
  b->block_shift = p.block_shift;
  b->n_groups = p.n_groups;
  b->threads = p.threads;
  b->unroll = p.unroll;
  b->ht_slots = p.ht_slots;
  b->smem = p.smem;
  // a batch's queries are known only when it runs: with object bitmaps in the
  // index, a second graph adds them, and each run picks one (as genie_search
  // does, by the share of the batch's postings the dense keywords carry)
  b->can_dense = index->n_dense && p.log2w >= 3;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->blocks = (opts && opts->blocks) ? opts->blocks : (uint32_t)sms;
  const size_t merge_smem = (size_t)dev::next_pow2(k) * 8 + (size_t)p.za_len * 4;
  b->smem = std::max(b->smem, merge_smem);
  cudaError_t e = cudaMalloc(&b->cand, (uint64_t)max_queries * p.n_groups * k * 8);
  // work counter, per-query seeds, then per-query count histograms of the
  // finished ranges (when they stay small)
  const uint64_t hist_words = (uint64_t)max_queries * p.za_len;
  const bool use_hist = hist_words * 4 <= kHintHistMaxBytes;
  b->counter_words = (uint64_t)max_queries + 1 + (use_hist ? hist_words : 0);
  if (e == cudaSuccess) e = cudaMalloc(&b->counters, b->counter_words * 4);

  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return fail_cuda(e, "genie_batch_create");
  }
  // fixed part of the descriptor; per-batch fields are filled by genie_batch_run
  BatchDesc& d = b->host_desc;
  std::memset(&d, 0, sizeof(d));
  d.scan.kw_off = index->kw_off;
  d.scan.post_ids = index->post_ids;
  d.scan.chunk_pos = index->chunk_pos;
  d.scan.n_chunks = index->n_chunks;
  d.scan.chunk_shift = index->chunk_shift;
  d.scan.n_objects = index->n_objects;
  d.scan.k = k;
  d.scan.block_shift = p.block_shift;
  d.scan.chunks_per_block = 1u << (p.block_shift - index->chunk_shift);
  d.scan.dense_slot = b->can_dense ? index->dense_slot : nullptr;
  d.scan.dense_bits = b->can_dense ? index->dense_bits : nullptr;
  d.scan.map_words = index->map_words;
  d.scan.n_groups = p.n_groups;
  d.scan.ht_slots = p.ht_slots;
  d.scan.za_len = p.za_len;
  d.scan.cand = b->cand;
  d.scan.at_hint = b->counters + 1;
  d.scan.hint_hist = use_hist ? b->counters + 1 + (uint64_t)max_queries : nullptr;
  d.scan.hint_stride = p.za_len;
  d.merge.cand = b->cand;
  d.merge.n_groups = p.n_groups;
  d.merge.k = k;
  d.merge.za_len = p.za_len;
  // capture: clear the counters, run the persistent kernel, merge
  cudaStream_t cs = b->capture_stream;
  const size_t msmem = (size_t)dev::next_pow2(k) * 8 + (size_t)p.za_len * 4;
  e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
  for (int gi = 0; gi < (b->can_dense ? 2 : 1) && e == cudaSuccess; ++gi) {
    b->dense = gi == 1;
    e = batch_dispatch(b, false);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(b->counters, 0, b->counter_words * 4, cs);
      cudaError_t le = batch_dispatch(b, true);
      merge_kernel<<<std::min<uint32_t>(max_queries, 152u * 16u), kMergeThreads, msmem, cs>>>(b->host_desc.merge);
      e = cudaStreamEndCapture(cs, &b->graph[gi]);
      if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[gi], b->graph[gi], 0);
    // the two kernel nodes: their arguments are set by each run
    size_t n_nodes = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(b->graph[gi], nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(b->graph[gi], nodes.data(), &n_nodes);
    for (size_t i = 0; i < n_nodes && e == cudaSuccess; ++i) {
      cudaGraphNodeType type;
      e = cudaGraphNodeGetType(nodes[i], &type);
      if (e != cudaSuccess || type != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
      if (e != cudaSuccess) break;
      if (kp.func == reinterpret_cast<void*>(merge_kernel)) {
        b->mnode[gi] = nodes[i];
        b->mnode_params[gi] = kp;
      } else {
        b->node[gi] = nodes[i];
        b->node_params[gi] = kp;
      }
    }
    if (e == cudaSuccess && (!b->node[gi] || !b->mnode[gi])) e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return fail_cuda(e, "genie_batch_create: graph capture");
  }
  *out = b;
  return GENIE_OK;
}

extern "C" void genie_batch_destroy(genie_batch* batch) {
  if (!batch) return;
  cudaDeviceSynchronize();
  free_batch(batch);
}

extern "C" genie_status genie_batch_get_info(const genie_batch* b, genie_batch_opts* out) {
  if (!b || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_batch_get_info: NULL argument");
  out->block_shift = b->block_shift;
  out->threads = b->threads;
  out->unroll = b->unroll;
  out->ht_slots = b->ht_slots;
  out->blocks = b->blocks;
  return GENIE_OK;
}

extern "C" genie_status genie_batch_run(genie_batch* b, const genie_queries* queries,
                                        const uint32_t* d_k, uint32_t* d_ids, uint32_t* d_counts,
                                        uint32_t* d_n_valid, genie_stream stream) {
  if (!b || !queries || !d_ids || !d_counts || !d_n_valid)
    return fail(GENIE_ERR_INVALID_ARG, "genie_batch_run: NULL argument");
  if (queries->index != b->index)
    return fail(GENIE_ERR_INVALID_ARG, "genie_batch_run: queries were compiled for another index");
  if (queries->n_queries > b->max_queries)
    return fail(GENIE_ERR_CAPACITY, "genie_batch_run: more queries than the batch was created for");
  if (queries->max_bound > b->max_bound)
    return fail(GENIE_ERR_CAPACITY, "genie_batch_run: a query's count bound exceeds the batch's max_bound");
  cudaStream_t s = as_stream(stream);
  if (d_k) {  // per-query k must lie in 1..k (one synchronisation)
    uint32_t bad = 0;
    GENIE_CUDA_TRY(cudaMemsetAsync(b->counters, 0, 4, s));
    check_k_kernel<<<std::min<uint32_t>((queries->n_queries + 255) / 256, 1024u), 256, 0, s>>>(
        queries->n_queries, b->k, d_k, b->counters);
    GENIE_CUDA_TRY(cudaMemcpyAsync(&bad, b->counters, 4, cudaMemcpyDeviceToHost, s));
    GENIE_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) return fail(GENIE_ERR_INVALID_ARG, "genie_batch_run: a per-query k is 0 or larger than k");
  }
  BatchDesc d = b->host_desc;
  d.scan.q_off = queries->q_off;
  d.scan.q_kw = queries->q_kw;
  d.scan.bound = queries->bound;
  d.scan.q_sel = nullptr;
  d.scan.n_sel = queries->n_queries;
  d.scan.k_arr = d_k;
  d.scan.seed = nullptr;
  d.scan.chunk_at = nullptr;
  d.scan.stats = nullptr;
  d.merge.n_sel = queries->n_queries;
  d.merge.q_sel = nullptr;
  d.merge.k_arr = d_k;
  d.merge.bound = queries->bound;
  d.merge.ids = d_ids;
  d.merge.counts = d_counts;
  d.merge.n_valid = d_n_valid;
  const bool dense = b->can_dense && queries->n_dense_entries > 0 &&
                     2 * queries->n_dense_entries >= queries->n_entries;
  const int gi = dense ? 1 : 0;
  // this batch's arguments on the two kernel nodes (copied by the calls; the
  // graph's next launch uses them)
  cudaKernelNodeParams kp = b->node_params[gi];
  uint32_t* work = b->counters;
  void* args[] = {&d.scan, &work};
  kp.kernelParams = args;
  kp.extra = nullptr;
  GENIE_CUDA_TRY(cudaGraphExecKernelNodeSetParams(b->exec[gi], b->node[gi], &kp));
  cudaKernelNodeParams mp = b->mnode_params[gi];
  void* margs[] = {&d.merge};
  mp.kernelParams = margs;
  mp.extra = nullptr;
  mp.gridDim = dim3(std::min<uint32_t>(queries->n_queries, 152u * 16u));
  GENIE_CUDA_TRY(cudaGraphExecKernelNodeSetParams(b->exec[gi], b->mnode[gi], &mp));
  GENIE_CUDA_TRY(cudaGraphLaunch(b->exec[gi], s));
  return GENIE_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------

extern "C" genie_status genie_autotune(const genie_index* index, const genie_queries* sample,
                                       uint32_t k, const char* cache_path, genie_batch_opts* out) {
  if (!index || !sample || !out) return fail(GENIE_ERR_INVALID_ARG, "genie_autotune: NULL argument");
  if (k == 0 || k > GENIE_MAX_K) return fail(GENIE_ERR_INVALID_ARG, "genie_autotune: k must be in 1..GENIE_MAX_K");
  const std::string key = tune_key(index, sample, k);
  if (cache_path && *cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string kk;
      genie_batch_opts o;
      std::memset(&o, 0, sizeof(o));
      if ((ls >> kk >> o.block_shift >> o.threads >> o.unroll >> o.ht_slots >> o.tuned_ms) && kk == key) {
        *out = o;
        out->from_cache = 1;
        return GENIE_OK;
      }
    }
  }
  // candidate shapes: block size x loads in flight x object range per block
  genie_queries probe;
  probe.index = index;
  probe.max_bound = sample->max_bound;
  Plan base;
  genie_status st = make_plan(index, &probe, k, nullptr, &base);
  if (st != GENIE_OK) return st;
  std::vector<genie_batch_opts> cands;
  const uint32_t shapes[][2] = {{768, 2}, {768, 4}, {896, 2}, {1024, 2}, {1024, 4}, {512, 4},
                                {512, 8}};
  for (uint32_t ds = 0; ds < 2; ++ds) {
    uint32_t bs = base.block_shift - ds;
    if (ds && bs < index->chunk_shift) continue;
    for (auto& sh : shapes) {
      genie_batch_opts o;
      std::memset(&o, 0, sizeof(o));
      o.block_shift = bs;
      o.threads = sh[0];
      o.unroll = sh[1];
      o.ht_slots = base.ht_slots;
      cands.push_back(o);
    }
  }
  const uint32_t Q = sample->n_queries;
  uint32_t *ids = nullptr, *cnt = nullptr, *nv = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&ids, (uint64_t)Q * k * 4);
  if (e == cudaSuccess) e = cudaMalloc(&cnt, (uint64_t)Q * k * 4);
  if (e == cudaSuccess) e = cudaMalloc(&nv, (uint64_t)Q * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  genie_batch_opts best_o = cands.empty() ? genie_batch_opts{} : cands[0];
  // each candidate runs as the persistent batch it would become (its kernel
  // differs from the one-block-per-item search in registers and scheduling)
  for (size_t c = 0; c < cands.size() && e == cudaSuccess; ++c) {
    genie_batch* cb = nullptr;
    st = genie_batch_create(index, Q, sample->max_bound, k, &cands[c], &cb);
    float t = 1e30f;
    for (int rep = 0; rep < 3 && st == GENIE_OK; ++rep) {  // first run warms up
      cudaEventRecord(e0, s);
      st = genie_batch_run(cb, sample, nullptr, ids, cnt, nv, (genie_stream)s);
      cudaEventRecord(e1, s);
      if (st != GENIE_OK) break;
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t = std::min(t, ms);
    }
    if (cb) genie_batch_destroy(cb);
    if (st != GENIE_OK) { st = GENIE_OK; continue; }  // a shape this GPU cannot run
    cands[c].tuned_ms = t;
    if (t < best) {
      best = t;
      best_o = cands[c];
    }
  }
  cudaFree(ids);
  cudaFree(cnt);
  cudaFree(nv);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail_cuda(e, "genie_autotune");
  *out = best_o;
  out->from_cache = 0;
  if (cache_path && *cache_path) {
    std::ofstream o(cache_path, std::ios::app);
    o << key << " " << best_o.block_shift << " " << best_o.threads << " " << best_o.unroll << " "
      << best_o.ht_slots << " " << best_o.tuned_ms << "\n";
  }
  return GENIE_OK;
}
