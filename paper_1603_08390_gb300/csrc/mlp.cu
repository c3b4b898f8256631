// The k-th-count predictor: a 64-128-1 ReLU network whose output seeds the
// c-PQ AuditThreshold (Sec. 3.3.1) of each query.  The paper has no learned
// component; the network only changes where the Gate starts, never a count,
// and the seeded search verifies every query (see genie_search).
//
// Weights are held as float32 master copies (Adam state beside them) and as
// bfloat16 working copies used by the forward and backward passes; every
// product is accumulated in float32.  Biases stay float32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace genie {
namespace {

constexpr uint32_t kIn = 64, kHid = 128;
constexpr uint32_t kW1 = kHid * kIn;                 // W1[j][i], row j = hidden unit
constexpr uint32_t kNParams = kW1 + kHid + kHid + 1;  // W1 | b1 | w2 | b2
constexpr uint32_t kTileSamples = 32;

struct Params {
  const __nv_bfloat16* W1;  // [kHid][kIn]
  const float* b1;          // [kHid]
  const __nv_bfloat16* w2;  // [kHid]
  const float* b2;          // [1]
};

// y[n] = w2 . relu(W1 x[n] + b1) + b2; one block of 128 threads (one per
// hidden unit) per tile of samples.
__global__ void __launch_bounds__(kHid) mlp_forward_kernel(const float* __restrict__ x, uint32_t n,
                                                           const Params P, float* __restrict__ y) {
  __shared__ float xs[kTileSamples][kIn];
  __shared__ float red[kTileSamples][kHid / 32];
  const uint32_t j = threadIdx.x, lane = j & 31, warp = j >> 5;
  float w[kIn];
#pragma unroll
  for (uint32_t i = 0; i < kIn; ++i) w[i] = __bfloat162float(P.W1[j * kIn + i]);
  const float bj = P.b1[j], vj = __bfloat162float(P.w2[j]), b2 = P.b2[0];
  for (uint32_t base = blockIdx.x * kTileSamples; base < n; base += gridDim.x * kTileSamples) {
    const uint32_t ns = min(kTileSamples, n - base);
    for (uint32_t t = j; t < kTileSamples * kIn; t += kHid) {
      uint32_t s = t / kIn, i = t % kIn;
      xs[s][i] = s < ns ? x[(uint64_t)(base + s) * kIn + i] : 0.f;
    }
    __syncthreads();
    for (uint32_t s = 0; s < ns; ++s) {
      float pre = bj;
#pragma unroll
      for (uint32_t i = 0; i < kIn; ++i) pre = fmaf(w[i], xs[s][i], pre);
      float part = vj * fmaxf(pre, 0.f);
      part = dev::warp_sum(part);
      if (lane == 0) red[s][warp] = part;
    }
    __syncthreads();
    if (j < ns) {
      float acc = b2;
#pragma unroll
      for (uint32_t w4 = 0; w4 < kHid / 32; ++w4) acc += red[j][w4];
      y[base + j] = acc;
    }
    __syncthreads();
  }
}

// Gradients of L = (1/n_total) sum 0.5 (y - t)^2 over the samples given,
// accumulated (atomicAdd) into grad = [dW1 | db1 | dw2 | db2]; also adds the
// summed squared error to *sse.
__global__ void __launch_bounds__(kHid) mlp_backward_kernel(const float* __restrict__ x,
                                                            const float* __restrict__ t, uint32_t n,
                                                            float inv_total, const Params P,
                                                            float* __restrict__ grad, float* sse) {
  __shared__ float xs[kTileSamples][kIn];
  __shared__ float red[kTileSamples][kHid / 32];
  __shared__ float dys[kTileSamples];
  __shared__ float pres[kTileSamples][kHid];
  const uint32_t j = threadIdx.x, lane = j & 31, warp = j >> 5;
  float w[kIn], gw[kIn];
#pragma unroll
  for (uint32_t i = 0; i < kIn; ++i) {
    w[i] = __bfloat162float(P.W1[j * kIn + i]);
    gw[i] = 0.f;
  }
  const float bj = P.b1[j], vj = __bfloat162float(P.w2[j]), b2 = P.b2[0];
  float gb1 = 0.f, gw2 = 0.f, gb2 = 0.f, err2 = 0.f;
  for (uint32_t base = blockIdx.x * kTileSamples; base < n; base += gridDim.x * kTileSamples) {
    const uint32_t ns = min(kTileSamples, n - base);
    for (uint32_t q = j; q < kTileSamples * kIn; q += kHid) {
      uint32_t s = q / kIn, i = q % kIn;
      xs[s][i] = s < ns ? x[(uint64_t)(base + s) * kIn + i] : 0.f;
    }
    __syncthreads();
    for (uint32_t s = 0; s < ns; ++s) {
      float pre = bj;
#pragma unroll
      for (uint32_t i = 0; i < kIn; ++i) pre = fmaf(w[i], xs[s][i], pre);
      pres[s][j] = pre;
      float part = vj * fmaxf(pre, 0.f);
      part = dev::warp_sum(part);
      if (lane == 0) red[s][warp] = part;
    }
    __syncthreads();
    if (j < ns) {
      float yv = b2;
#pragma unroll
      for (uint32_t w4 = 0; w4 < kHid / 32; ++w4) yv += red[j][w4];
      const float e = yv - t[base + j];
      dys[j] = e * inv_total;
      err2 += e * e;
    }
    __syncthreads();
    for (uint32_t s = 0; s < ns; ++s) {
      const float dy = dys[s];
      const float pre = pres[s][j];
      const float h = fmaxf(pre, 0.f);
      gw2 = fmaf(dy, h, gw2);
      if (j == 0) gb2 += dy;
      const float dpre = pre > 0.f ? dy * vj : 0.f;
      gb1 += dpre;
#pragma unroll
      for (uint32_t i = 0; i < kIn; ++i) gw[i] = fmaf(dpre, xs[s][i], gw[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (uint32_t i = 0; i < kIn; ++i) atomicAdd(&grad[j * kIn + i], gw[i]);
  atomicAdd(&grad[kW1 + j], gb1);
  atomicAdd(&grad[kW1 + kHid + j], gw2);
  if (j == 0) atomicAdd(&grad[kW1 + 2 * kHid], gb2);
  err2 = dev::warp_sum(err2);
  if (lane == 0) atomicAdd(sse, err2);
}

// Adam (Kingma & Ba 2015) on the float32 masters, then refresh the bf16
// working copies of the weights.
__global__ void mlp_adam_kernel(float* __restrict__ theta, const float* __restrict__ grad,
                                float* __restrict__ m, float* __restrict__ v, float lr, float beta1,
                                float beta2, float eps, float bc1, float bc2,
                                __nv_bfloat16* __restrict__ W1h, __nv_bfloat16* __restrict__ w2h) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    theta[i] = th;
    if (i < kW1) W1h[i] = __float2bfloat16_rn(th);
    else if (i >= kW1 + kHid && i < kW1 + 2 * kHid) w2h[i - kW1 - kHid] = __float2bfloat16_rn(th);
  }
}

__global__ void mlp_round_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ W1h,
                                 __nv_bfloat16* __restrict__ w2h) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < kW1 + kHid; i += gridDim.x * blockDim.x) {
    if (i < kW1) W1h[i] = __float2bfloat16_rn(theta[i]);
    else w2h[i - kW1] = __float2bfloat16_rn(theta[kW1 + kHid + (i - kW1)]);
  }
}

// seed_q = clamp(floor(y_q - margin), 1, B_q + 1); a non-finite prediction
// gives the paper's start value 1
__global__ void mlp_seed_kernel(const float* __restrict__ y, const uint32_t* __restrict__ bound,
                                uint32_t n, float margin, uint32_t* __restrict__ seed) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float p = y[q] - margin;
    uint32_t s = 1;
    if (isfinite(p) && p >= 1.f) s = (uint32_t)fminf(floorf(p), (float)(bound[q] + 1));
    seed[q] = max(1u, s);
  }
}

__global__ void mlp_init_kernel(float* __restrict__ theta, uint64_t seed) {
  // He-uniform init from a counter-based hash (SplitMix64 output function)
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.0f / 16777216.0f) * 2.f - 1.f;  // U(-1, 1)
    float val = 0.f;
    if (i < kW1) val = u * sqrtf(6.f / kIn);
    else if (i >= kW1 + kHid && i < kW1 + 2 * kHid) val = u * sqrtf(6.f / kHid);
    theta[i] = val;
  }
}

int grid_samples(uint32_t n) {
  return (int)std::max<uint32_t>(1, std::min<uint32_t>((n + kTileSamples - 1) / kTileSamples, 152u * 8u));
}

}  // namespace
}  // namespace genie

struct genie_mlp {
  float* theta = nullptr;  // float32 masters [kNParams]
  float* grad = nullptr;   // [kNParams] + 1 (summed squared error)
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* W1h = nullptr;
  __nv_bfloat16* w2h = nullptr;
  float* y = nullptr;      // prediction scratch for seeds
  uint32_t y_cap = 0;
  uint64_t step = 0;
};

using namespace genie;

namespace {
Params params_of(const genie_mlp* m) {
  return Params{m->W1h, m->theta + kW1, m->w2h, m->theta + kW1 + 2 * kHid};
}
void free_mlp(genie_mlp* m) {
  if (!m) return;
  cudaFree(m->theta);
  cudaFree(m->grad);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->W1h);
  cudaFree(m->w2h);
  cudaFree(m->y);
  delete m;
}
}  // namespace

extern "C" uint32_t genie_mlp_num_params(void) { return kNParams; }

extern "C" genie_status genie_mlp_create(uint64_t seed, genie_stream stream, genie_mlp** out) {
  if (!out) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_create: out is NULL");
  genie_mlp* m = new (std::nothrow) genie_mlp();
  if (!m) return fail(GENIE_ERR_OUT_OF_MEMORY, "genie_mlp_create: host allocation");
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMalloc(&m->theta, kNParams * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, (kNParams + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, kNParams * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, kNParams * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->W1h, kW1 * 2);
  if (e == cudaSuccess) e = cudaMalloc(&m->w2h, kHid * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, kNParams * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, kNParams * 4, s);
  if (e == cudaSuccess) {
    mlp_init_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(m->theta, seed);
    mlp_round_kernel<<<(kW1 + kHid + 255) / 256, 256, 0, s>>>(m->theta, m->W1h, m->w2h);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    free_mlp(m);
    return fail_cuda(e, "genie_mlp_create");
  }
  *out = m;
  return GENIE_OK;
}

extern "C" void genie_mlp_destroy(genie_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  free_mlp(m);
}

extern "C" genie_status genie_mlp_set_params(genie_mlp* m, const float* d_theta, genie_stream stream) {
  if (!m || !d_theta) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_set_params: NULL argument");
  cudaStream_t s = as_stream(stream);
  GENIE_CUDA_TRY(cudaMemcpyAsync(m->theta, d_theta, kNParams * 4, cudaMemcpyDeviceToDevice, s));
  GENIE_CUDA_TRY(cudaMemsetAsync(m->m, 0, kNParams * 4, s));
  GENIE_CUDA_TRY(cudaMemsetAsync(m->v, 0, kNParams * 4, s));
  m->step = 0;
  mlp_round_kernel<<<(kW1 + kHid + 255) / 256, 256, 0, s>>>(m->theta, m->W1h, m->w2h);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_get_params(const genie_mlp* m, float* d_theta, genie_stream stream) {
  if (!m || !d_theta) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_get_params: NULL argument");
  GENIE_CUDA_TRY(cudaMemcpyAsync(d_theta, m->theta, kNParams * 4, cudaMemcpyDeviceToDevice,
                                 as_stream(stream)));
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_forward(const genie_mlp* m, const float* d_x, uint32_t n,
                                          float* d_y, genie_stream stream) {
  if (!m || (n && (!d_x || !d_y))) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_forward: NULL argument");
  if (n == 0) return GENIE_OK;
  mlp_forward_kernel<<<grid_samples(n), kHid, 0, as_stream(stream)>>>(d_x, n, params_of(m), d_y);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_gradients(genie_mlp* m, const float* d_x, const float* d_t,
                                            uint32_t n, float* d_grad, genie_stream stream) {
  if (!m || !d_x || !d_t || n == 0) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_gradients: bad argument");
  cudaStream_t s = as_stream(stream);
  GENIE_CUDA_TRY(cudaMemsetAsync(m->grad, 0, (kNParams + 1) * 4, s));
  mlp_backward_kernel<<<grid_samples(n), kHid, 0, s>>>(d_x, d_t, n, 1.f / (float)n, params_of(m),
                                                       m->grad, m->grad + kNParams);
  GENIE_CUDA_TRY(cudaGetLastError());
  if (d_grad)
    GENIE_CUDA_TRY(cudaMemcpyAsync(d_grad, m->grad, (kNParams + 1) * 4, cudaMemcpyDeviceToDevice, s));
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_adam_step(genie_mlp* m, float lr, genie_stream stream) {
  if (!m || !(lr > 0.f)) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_adam_step: bad argument");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m->step += 1;
  const float bc1 = 1.f - powf(b1, (float)m->step), bc2 = 1.f - powf(b2, (float)m->step);
  mlp_adam_kernel<<<(kNParams + 255) / 256, 256, 0, as_stream(stream)>>>(
      m->theta, m->grad, m->m, m->v, lr, b1, b2, eps, bc1, bc2, m->W1h, m->w2h);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_train(genie_mlp* m, const float* d_x, const float* d_t, uint32_t n,
                                        uint32_t epochs, uint32_t batch, float lr, float* h_loss,
                                        genie_stream stream) {
  if (!m || !d_x || !d_t || n == 0 || batch == 0 || !(lr > 0.f))
    return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_train: bad argument");
  cudaStream_t s = as_stream(stream);
  float sse_sum = 0.f;
  for (uint32_t ep = 0; ep < epochs; ++ep) {
    for (uint32_t b0 = 0; b0 < n; b0 += batch) {
      const uint32_t nb = std::min(batch, n - b0);
      genie_status st = genie_mlp_gradients(m, d_x + (uint64_t)b0 * kIn, d_t + b0, nb, nullptr, stream);
      if (st != GENIE_OK) return st;
      st = genie_mlp_adam_step(m, lr, stream);
      if (st != GENIE_OK) return st;
    }
  }
  if (h_loss) {  // mean 0.5 (y - t)^2 over the whole set after training
    GENIE_CUDA_TRY(cudaMemsetAsync(m->grad, 0, (kNParams + 1) * 4, s));
    mlp_backward_kernel<<<grid_samples(n), kHid, 0, s>>>(d_x, d_t, n, 1.f / (float)n, params_of(m),
                                                         m->grad, m->grad + kNParams);
    GENIE_CUDA_TRY(cudaGetLastError());
    GENIE_CUDA_TRY(cudaMemcpyAsync(&sse_sum, m->grad + kNParams, 4, cudaMemcpyDeviceToHost, s));
    GENIE_CUDA_TRY(cudaStreamSynchronize(s));
    *h_loss = 0.5f * sse_sum / (float)n;
  }
  return GENIE_OK;
}

extern "C" genie_status genie_mlp_seeds(genie_mlp* m, const genie_queries* queries, float margin,
                                        uint32_t* d_seed, genie_stream stream) {
  if (!m || !queries || !d_seed) return fail(GENIE_ERR_INVALID_ARG, "genie_mlp_seeds: NULL argument");
  cudaStream_t s = as_stream(stream);
  const uint32_t n = queries->n_queries;
  if (m->y_cap < n) {
    cudaFree(m->y);
    m->y = nullptr;
    m->y_cap = 0;
    GENIE_CUDA_TRY(cudaMalloc(&m->y, (uint64_t)n * 4));
    m->y_cap = n;
  }
  mlp_forward_kernel<<<grid_samples(n), kHid, 0, s>>>(queries->features, n, params_of(m), m->y);
  mlp_seed_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>((n + 255) / 256, 1024)), 256, 0, s>>>(
      m->y, queries->bound, n, margin, d_seed);
  GENIE_CUDA_TRY(cudaGetLastError());
  return GENIE_OK;
}
