// Device ceilings for the counter updates of the search.
//
// The scan kernel's dominant cost is one shared-memory atomic add per
// posting into a counter array at (effectively) random addresses.  This
// kernel measures how many such updates per second the GPU sustains when it
// does nothing else: every resident block fills the same 128 KB counter array
// the search uses and every thread adds to a 16-bit lane at pseudo-random
// positions.  Four forms are timed:
//   * an integer add of the lane's increment to its 32-bit word, with the old
//     word returned and consumed (what the Gate needs),
//   * the same add with no value returned (red),
//   * a binary16 add of 1.0 to the lane itself, old value returned (integers
//     up to 2048 are exact in binary16, so this counts exactly),
//   * the binary16 add with no value returned.
// The results are the rooflines the scan kernel is compared with beside HBM
// bandwidth.
#include <cuda_fp16.h>

#include <cstdint>

#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kCalThreads = 768;
constexpr uint32_t kCalWords = 32768;  // 128 KB of counters per block

enum CalMode : int { kAtomU32 = 0, kRedU32 = 1, kAtomF16 = 2, kRedF16 = 3 };

template <int MODE>
__global__ void __launch_bounds__(kCalThreads, 1) smem_atomic_kernel(uint32_t iters,
                                                                     unsigned long long* sink) {
  extern __shared__ uint32_t cnt[];
  for (uint32_t i = threadIdx.x; i < kCalWords; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(cnt);
  uint32_t x = 0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  uint32_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      x ^= x << 13;
      x ^= x >> 17;
      x ^= x << 5;  // xorshift32 (Marsaglia 2003)
      const uint32_t lane16 = x & (2 * kCalWords - 1);  // a 16-bit lane of the array
      if (MODE == kAtomU32 || MODE == kRedU32) {
        const uint32_t sh = (lane16 & 1u) << 4;
        const uint32_t addr = base + ((lane16 >> 1) << 2);
        if (MODE == kAtomU32) {
          uint32_t old;
          asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(1u << sh) : "memory");
          acc += old >> sh;
        } else {
          asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(1u << sh) : "memory");
        }
      } else {
        const uint32_t addr = base + (lane16 << 1);
        const unsigned short one = 0x3C00u;  // binary16 1.0
        if (MODE == kAtomF16) {
          unsigned short old;
          asm volatile("atom.shared.add.noftz.f16 %0, [%1], %2;" : "=h"(old) : "r"(addr), "h"(one) : "memory");
          acc += old;
        } else {
          asm volatile("red.shared.add.noftz.f16 [%0], %1;" ::"r"(addr), "h"(one) : "memory");
        }
      }
    }
  }
  if (MODE == kRedU32 || MODE == kRedF16) {
    __syncthreads();
    acc = cnt[threadIdx.x];
  }
  if (acc == 0xFFFFFFFFu) atomicAdd(sink, 1ull);  // keeps the returned values live
}

template <int MODE>
cudaError_t time_mode(int sms, unsigned long long* sink, cudaStream_t s, cudaEvent_t e0,
                      cudaEvent_t e1, uint32_t iters, float* best_ms) {
  const size_t smem = kCalWords * 4;
  cudaError_t e = cudaFuncSetAttribute(smem_atomic_kernel<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    smem_atomic_kernel<MODE><<<sms, kCalThreads, smem, s>>>(iters, sink);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = ms < best ? ms : best;  // first launch warms up
  }
  *best_ms = best;
  return e;
}

}  // namespace
}  // namespace genie

using namespace genie;

extern "C" genie_status genie_calibrate(genie_calibration* out) {
  if (!out) return fail(GENIE_ERR_INVALID_ARG, "genie_calibrate: out is NULL");
  int dev = 0, sms = 0;
  GENIE_CUDA_TRY(cudaGetDevice(&dev));
  GENIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  unsigned long long* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint32_t iters = 4096;
  float ms[4] = {0.f, 0.f, 0.f, 0.f};
  if (e == cudaSuccess) e = time_mode<kAtomU32>(sms, sink, s, e0, e1, iters, &ms[0]);
  if (e == cudaSuccess) e = time_mode<kRedU32>(sms, sink, s, e0, e1, iters, &ms[1]);
  if (e == cudaSuccess) e = time_mode<kAtomF16>(sms, sink, s, e0, e1, iters, &ms[2]);
  if (e == cudaSuccess) e = time_mode<kRedF16>(sms, sink, s, e0, e1, iters, &ms[3]);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail_cuda(e, "genie_calibrate");
  const double ops = (double)sms * kCalThreads * iters * 8;
  out->smem_atomics_per_s = ops / (ms[0] * 1e-3);
  out->sms = (uint32_t)sms;
  out->seconds = ms[0] * 1e-3;
  out->smem_red_per_s = ops / (ms[1] * 1e-3);
  out->smem_f16_atomics_per_s = ops / (ms[2] * 1e-3);
  out->smem_f16_red_per_s = ops / (ms[3] * 1e-3);
  return GENIE_OK;
}
