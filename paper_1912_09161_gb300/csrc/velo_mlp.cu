// Training of the ghost-track classifier on the GPU: 10 -> 32 -> 32 -> 1,
// ReLU, sigmoid output, binary cross-entropy on the logit, Adam on FP32
// master weights, BF16 copies of the weights and BF16 activations in the
// forward pass with FP32 accumulation (the paper has no classifier of its
// own; its HLT1 selections use MVA lines, section 2.3.6).
//
// One step = two kernels:
//   grad  -- one block per 128 samples: forward and backward per thread
//            (activations and deltas in shared memory), then the block's
//            weight gradients as sums over its samples in a fixed order,
//            written as one partial per block;
//   adam  -- per parameter: the sum of the block partials in block order,
//            then the Adam update and the BF16 copy.
// No atomics are involved, so a step is deterministic and a run resumes bit
// for bit from a checkpoint of (weights, moments, step).
//
// The network is tiny (1441 parameters, K = 10 and 32): the whole training
// of 200,000 tracks takes milliseconds per epoch, so plain FMA pipes serve;
// the tensor cores would not change the wall time measurably.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "velo_mlp.cuh"

namespace velo {
void set_last_error(const char* msg);
}

using namespace velo;

namespace {

constexpr int kGradThreads = 128;
constexpr int kPartial = kMlpParams + 1;  // parameters, then the loss

int report(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  velo::set_last_error(buf);
  return code;
}

#define MLP_TRY(expr)                                                                                   \
  do {                                                                                                  \
    cudaError_t _e = (expr);                                                                            \
    if (_e != cudaSuccess) return report(VELO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));       \
  } while (0)

// Per-sample shared arrays of the gradient kernel.
struct GradSmem {
  float x[kGradThreads][kMlpIn];
  float h1[kGradThreads][kMlpH];
  float h2[kGradThreads][kMlpH];
  float d1[kGradThreads][kMlpH];
  float d2[kGradThreads][kMlpH];
  float dout[kGradThreads];
  float loss[kGradThreads];
};

__global__ void __launch_bounds__(kGradThreads)
    mlp_grad_kernel(const float* __restrict__ feats, const float* __restrict__ labels, uint32_t n, float inv_n,
                    const uint16_t* __restrict__ w, const float* __restrict__ norm, float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
  const int t = threadIdx.x;
  const uint32_t i = blockIdx.x * kGradThreads + t;
  float x[kMlpIn], a1[kMlpH], h1[kMlpH];
  if (i < n) {
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k)
      x[k] = bf16_round(fmul(fsub(feats[(size_t)i * kMlpIn + k], norm[k]), norm[kMlpIn + k]));
  } else {
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = 0.0f;
  }
  // forward
#pragma unroll 4
  for (int j = 0; j < kMlpH; ++j) {
    float acc = bf16_value(w[kOffB1 + j]);
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) acc = fadd(acc, fmul(bf16_value(w[kOffW1 + j * kMlpIn + k]), x[k]));
    a1[j] = acc;
    h1[j] = bf16_round(fmaxf(acc, 0.0f));
  }
  float out = bf16_value(w[kOffB3]);
  for (int j = 0; j < kMlpH; ++j) {
    float acc = bf16_value(w[kOffB2 + j]);
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) acc = fadd(acc, fmul(bf16_value(w[kOffW2 + j * kMlpH + k]), h1[k]));
    const float h2 = bf16_round(fmaxf(acc, 0.0f));
    S.h2[t][j] = h2;
    S.d2[t][j] = acc;  // pre-activation, until the delta replaces it
    out = fadd(out, fmul(bf16_value(w[kOffW3 + j]), h2));
  }
  // loss and output delta (mean over the batch)
  float dout = 0.0f, loss = 0.0f;
  if (i < n) {
    const float y = labels[i];
    const float p = 1.0f / (1.0f + expf(-out));
    dout = (p - y) * inv_n;
    loss = (fmaxf(out, 0.0f) - out * y + log1pf(expf(-fabsf(out)))) * inv_n;
  }
  // hidden deltas
  for (int j = 0; j < kMlpH; ++j) {
    const float a2 = S.d2[t][j];
    S.d2[t][j] = a2 > 0.0f ? dout * bf16_value(w[kOffW3 + j]) : 0.0f;
  }
  for (int k = 0; k < kMlpH; ++k) {
    float acc = 0.0f;
    for (int j = 0; j < kMlpH; ++j) acc += S.d2[t][j] * bf16_value(w[kOffW2 + j * kMlpH + k]);
    S.d1[t][k] = a1[k] > 0.0f ? acc : 0.0f;
    S.h1[t][k] = h1[k];
  }
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) S.x[t][k] = x[k];
  S.dout[t] = dout;
  S.loss[t] = loss;
  __syncthreads();
  // weight gradients: sums over the block's samples in sample order
  float* P = partial + (size_t)blockIdx.x * kPartial;
  for (int p = t; p < kPartial; p += kGradThreads) {
    float g = 0.0f;
    if (p < kOffB1) {
      const int j = p / kMlpIn, k = p % kMlpIn;
      for (int s = 0; s < kGradThreads; ++s) g += S.d1[s][j] * S.x[s][k];
    } else if (p < kOffW2) {
      const int j = p - kOffB1;
      for (int s = 0; s < kGradThreads; ++s) g += S.d1[s][j];
    } else if (p < kOffB2) {
      const int j = (p - kOffW2) / kMlpH, k = (p - kOffW2) % kMlpH;
      for (int s = 0; s < kGradThreads; ++s) g += S.d2[s][j] * S.h1[s][k];
    } else if (p < kOffW3) {
      const int j = p - kOffB2;
      for (int s = 0; s < kGradThreads; ++s) g += S.d2[s][j];
    } else if (p < kOffB3) {
      const int j = p - kOffW3;
      for (int s = 0; s < kGradThreads; ++s) g += S.dout[s] * S.h2[s][j];
    } else if (p == kOffB3) {
      for (int s = 0; s < kGradThreads; ++s) g += S.dout[s];
    } else {
      for (int s = 0; s < kGradThreads; ++s) g += S.loss[s];
    }
    P[p] = g;
  }
}

// Sum of the block partials in block order; with adam != 0 also the update.
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, uint32_t nblk, float* __restrict__ grad,
                                  int adam, float* __restrict__ master, float* __restrict__ m1,
                                  float* __restrict__ m2, uint16_t* __restrict__ wbf, float lr, float b1, float b2,
                                  float omb1, float omb2, float c1, float c2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kPartial) return;
  float g = 0.0f;
  for (uint32_t b = 0; b < nblk; ++b) g += partial[(size_t)b * kPartial + p];
  grad[p] = g;
  if (!adam || p >= kMlpParams) return;
  // omb1 = 1 - beta1 and omb2 = 1 - beta2, rounded once from double (1.0f -
  // 0.999f would be 1.3e-5 off 0.001)
  const float m = b1 * m1[p] + omb1 * g;
  const float v = b2 * m2[p] + omb2 * g * g;
  m1[p] = m;
  m2[p] = v;
  const float w = master[p] - lr * (m * c1) / (sqrtf(v * c2) + eps);
  master[p] = w;
  wbf[p] = bf16_bits(w);
}

__global__ void mlp_to_bf16_kernel(const float* __restrict__ master, uint16_t* __restrict__ wbf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) wbf[p] = bf16_bits(master[p]);
}

__global__ void mlp_logits_kernel(const float* __restrict__ feats, uint32_t n, const uint16_t* __restrict__ w,
                                  const float* __restrict__ norm, float* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float f[kMlpIn];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) f[k] = feats[(size_t)i * kMlpIn + k];
  out[i] = mlp_logit(f, w, norm, norm + kMlpIn);
}

}  // namespace

struct velo_mlp_trainer {
  uint32_t max_batch = 0, step = 0;
  float* master = nullptr;   // [kMlpParams]
  float* m1 = nullptr;
  float* m2 = nullptr;
  uint16_t* wbf = nullptr;   // [kMlpParams]
  float* norm = nullptr;     // [2 * kMlpIn]
  float* partial = nullptr;  // [blocks][kPartial]
  float* grad = nullptr;     // [kPartial]
};

extern "C" {

void velo_mlp_destroy(velo_mlp_trainer* t) {
  if (!t) return;
  for (void* p : {(void*)t->master, (void*)t->m1, (void*)t->m2, (void*)t->wbf, (void*)t->norm, (void*)t->partial,
                  (void*)t->grad})
    if (p) cudaFree(p);
  delete t;
}

int velo_mlp_create(const float* params, const float* mean, const float* istd, uint32_t max_batch,
                    velo_mlp_trainer** out) {
  if (!out || !params || !mean || !istd || max_batch == 0) return report(VELO_ERR_INPUT, "velo_mlp_create: bad argument");
  *out = nullptr;
  velo_mlp_trainer* t = new (std::nothrow) velo_mlp_trainer();
  if (!t) return report(VELO_ERR_NOMEM, "velo_mlp_create: host allocation failed");
  t->max_batch = max_batch;
  const uint32_t nblk = (max_batch + kGradThreads - 1) / kGradThreads;
  float norm[2 * kMlpIn];
  memcpy(norm, mean, sizeof(float) * kMlpIn);
  memcpy(norm + kMlpIn, istd, sizeof(float) * kMlpIn);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&t->master, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->m1, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->m2, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->wbf, sizeof(uint16_t) * kMlpParams);
  if (e == cudaSuccess) e = cudaMalloc(&t->norm, sizeof(norm));
  if (e == cudaSuccess) e = cudaMalloc(&t->partial, sizeof(float) * kPartial * nblk);
  if (e == cudaSuccess) e = cudaMalloc(&t->grad, sizeof(float) * kPartial);
  if (e == cudaSuccess) e = cudaMemcpy(t->master, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->m1, 0, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMemset(t->m2, 0, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMemcpy(t->norm, norm, sizeof(norm), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem));
  if (e == cudaSuccess) {
    mlp_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256>>>(t->master, t->wbf);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    velo_mlp_destroy(t);
    return report(VELO_ERR_CUDA, "velo_mlp_create: %s", cudaGetErrorString(e));
  }
  *out = t;
  return VELO_OK;
}

static int run_grad(velo_mlp_trainer* t, const float* feats, const float* labels, uint32_t n, cudaStream_t st) {
  if (n == 0 || n > t->max_batch) return report(VELO_ERR_INPUT, "batch of %u samples outside [1, %u]", n, t->max_batch);
  const uint32_t nblk = (n + kGradThreads - 1) / kGradThreads;
  mlp_grad_kernel<<<nblk, kGradThreads, sizeof(GradSmem), st>>>(feats, labels, n, 1.0f / (float)n, t->wbf, t->norm,
                                                                 t->partial);
  MLP_TRY(cudaGetLastError());
  return VELO_OK;
}

int velo_mlp_step(velo_mlp_trainer* t, const float* features, const float* labels, uint32_t n, float lr, void* stream) {
  if (!t || !features || !labels) return report(VELO_ERR_INPUT, "velo_mlp_step: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = run_grad(t, features, labels, n, st);
  if (rc != VELO_OK) return rc;
  t->step++;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)t->step)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)t->step)));
  const uint32_t nblk = (n + kGradThreads - 1) / kGradThreads;
  mlp_reduce_kernel<<<(kPartial + 255) / 256, 256, 0, st>>>(t->partial, nblk, t->grad, 1, t->master, t->m1, t->m2,
                                                             t->wbf, lr, (float)b1, (float)b2, (float)(1.0 - b1),
                                                             (float)(1.0 - b2), c1, c2, 1e-8f);
  MLP_TRY(cudaGetLastError());
  return VELO_OK;
}

int velo_mlp_gradient(velo_mlp_trainer* t, const float* features, const float* labels, uint32_t n, float* grad_host,
                      float* loss_host, void* stream) {
  if (!t || !features || !labels || !grad_host) return report(VELO_ERR_INPUT, "velo_mlp_gradient: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = run_grad(t, features, labels, n, st);
  if (rc != VELO_OK) return rc;
  const uint32_t nblk = (n + kGradThreads - 1) / kGradThreads;
  mlp_reduce_kernel<<<(kPartial + 255) / 256, 256, 0, st>>>(t->partial, nblk, t->grad, 0, nullptr, nullptr, nullptr,
                                                             nullptr, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f);
  MLP_TRY(cudaGetLastError());
  float buf[kPartial];
  MLP_TRY(cudaMemcpyAsync(buf, t->grad, sizeof(buf), cudaMemcpyDeviceToHost, st));
  MLP_TRY(cudaStreamSynchronize(st));
  memcpy(grad_host, buf, sizeof(float) * kMlpParams);
  if (loss_host) *loss_host = buf[kMlpParams];
  return VELO_OK;
}

int velo_mlp_logits(velo_mlp_trainer* t, const float* features, uint32_t n, float* logits, void* stream) {
  if (!t || (n && (!features || !logits))) return report(VELO_ERR_INPUT, "velo_mlp_logits: null argument");
  if (n == 0) return VELO_OK;
  mlp_logits_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(features, n, t->wbf, t->norm, logits);
  MLP_TRY(cudaGetLastError());
  return VELO_OK;
}

int velo_mlp_get_state(velo_mlp_trainer* t, float* params, uint16_t* params_bf16, float* m1, float* m2,
                       uint32_t* step) {
  if (!t) return report(VELO_ERR_INPUT, "velo_mlp_get_state: null trainer");
  MLP_TRY(cudaDeviceSynchronize());
  if (params) MLP_TRY(cudaMemcpy(params, t->master, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  if (params_bf16) MLP_TRY(cudaMemcpy(params_bf16, t->wbf, sizeof(uint16_t) * kMlpParams, cudaMemcpyDeviceToHost));
  if (m1) MLP_TRY(cudaMemcpy(m1, t->m1, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  if (m2) MLP_TRY(cudaMemcpy(m2, t->m2, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  if (step) *step = t->step;
  return VELO_OK;
}

int velo_mlp_set_state(velo_mlp_trainer* t, const float* params, const float* m1, const float* m2, uint32_t step) {
  if (!t || !params || !m1 || !m2) return report(VELO_ERR_INPUT, "velo_mlp_set_state: null argument");
  MLP_TRY(cudaMemcpy(t->master, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  MLP_TRY(cudaMemcpy(t->m1, m1, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  MLP_TRY(cudaMemcpy(t->m2, m2, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  mlp_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256>>>(t->master, t->wbf);
  MLP_TRY(cudaDeviceSynchronize());
  t->step = step;
  return VELO_OK;
}

}  // extern "C"
