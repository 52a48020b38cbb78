// Learned control variate v_theta (Eq. 11, 37-39): training kernels (FP32
// forward, backward and Adam, one thread per sample point), the staging of the
// network for in-path use (BF16 64x64 layer), and a standalone evaluation of
// v and grad v with the same tensor-core warp routine the path kernel uses.
//
// The paper builds F = sigma^T grad u0 from a warm-up solution u0 (Sec. 4.2);
// here u0 is represented by a small MLP fitted to the warm-up nodal values and
// boundary samples, and grad v_theta is evaluated where each path is.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "pdds.h"
#include "pdds_internal.h"
#include "pdds_mlp.cuh"

namespace pdds {
namespace {

constexpr int kTrainThreads = 64;
constexpr int kOffW1 = 0, kOffB1 = 128, kOffW2 = 192, kOffB2 = 4288, kOffW3 = 4352, kOffB3 = 4416;
// shared layout of the training kernel (floats)
constexpr int kSmW = 4480;                           // theta copy (padded)
constexpr int kSmStride = kTrainThreads + 1;        // row stride: rows fall in distinct banks
constexpr int kSmArr = kMlpHidden * kSmStride;       // one [64][64] activation array (padded)
constexpr size_t kTrainSmemBytes = (kSmW + 4 * kSmArr + 4 * kTrainThreads) * sizeof(float);

__device__ __forceinline__ float logistic(float a) { return 1.0f / (1.0f + __expf(-a)); }

// Mean-squared-error loss (1/N) sum (v(x_p) - target_p)^2 and its gradient
// with respect to theta; one thread per point, block partial sums are added
// to grad with atomics.  Every dot product runs as four independent FMA chains
// (four outputs, or four parameters, at a time): with 64-point blocks there
// are few warps per SM, so latency, not issue, is the limit.
__global__ void __launch_bounds__(kTrainThreads) mlp_grad_kernel(
    const float* __restrict__ theta, const float* __restrict__ xy, const float* __restrict__ tgt,
    int64_t npts, float scale, float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ float sm[];
  float* T = sm;                       // theta
  float* H1 = sm + kSmW;               // [64][P] SiLU(a1)
  float* D1 = H1 + kSmArr;             // [64][P] SiLU'(a1), later dL/da1
  float* H2 = D1 + kSmArr;             // [64][P] SiLU(a2)
  float* G2 = H2 + kSmArr;             // [64][P] dL/da2
  float* PX = G2 + kSmArr;             // [P] x, y, dL/dv
  float* PY = PX + kTrainThreads;
  float* DV = PY + kTrainThreads;
  float* RL = DV + kTrainThreads;      // squared residuals
  constexpr int P = kTrainThreads;
  constexpr int S = kSmStride;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpParams; i += P) T[i] = theta[i];
  const int64_t p = (int64_t)blockIdx.x * P + tid;
  const bool valid = p < npts;
  const float x = valid ? xy[2 * p] : 0.f, y = valid ? xy[2 * p + 1] : 0.f;
  PX[tid] = x;
  PY[tid] = y;
  __syncthreads();
  for (int u = 0; u < kMlpHidden; ++u) {
    const float a = fmaf(T[kOffW1 + 2 * u], x, fmaf(T[kOffW1 + 2 * u + 1], y, T[kOffB1 + u]));
    const float s = logistic(a);
    H1[u * S + tid] = valid ? a * s : 0.f;
    D1[u * S + tid] = s * (1.f + a * (1.f - s));
  }
  float v = T[kOffB3];
  for (int o = 0; o < kMlpHidden; o += 4) {
    float a[4] = {T[kOffB2 + o], T[kOffB2 + o + 1], T[kOffB2 + o + 2], T[kOffB2 + o + 3]};
    for (int u = 0; u < kMlpHidden; ++u) {
      const float h1 = H1[u * S + tid];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = fmaf(T[kOffW2 + (o + q) * kMlpHidden + u], h1, a[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float s = logistic(a[q]);
      const float h = a[q] * s;
      H2[(o + q) * S + tid] = h;
      G2[(o + q) * S + tid] = T[kOffW3 + o + q] * s * (1.f + a[q] * (1.f - s));
      v = fmaf(T[kOffW3 + o + q], h, v);
    }
  }
  const float r = valid ? v - tgt[p] : 0.f;
  const float dv = scale * r;  // scale = 2 / N
  DV[tid] = dv;
  RL[tid] = r * r;
  for (int o = 0; o < kMlpHidden; ++o) G2[o * S + tid] *= dv;
  // dL/da1 = SiLU'(a1) * sum_o W2[o][u] dL/da2[o]
  for (int u = 0; u < kMlpHidden; u += 4) {
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    for (int o = 0; o < kMlpHidden; ++o) {
      const float g = G2[o * S + tid];
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] = fmaf(T[kOffW2 + o * kMlpHidden + u + q], g, t[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) D1[(u + q) * S + tid] *= t[q];
  }
  __syncthreads();
  // block reductions over the P points: thread tid owns row o = tid of the
  // 64x64 weight gradient, four columns at a time
  {
    const int o = tid;  // P == kMlpHidden
    for (int u = 0; u < kMlpHidden; u += 4) {
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      for (int q = 0; q < P; ++q) {
        const float g = G2[o * S + q];
#pragma unroll
        for (int c = 0; c < 4; ++c) t[c] = fmaf(g, H1[(u + c) * S + q], t[c]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) atomicAdd(grad + kOffW2 + o * kMlpHidden + u + c, t[c]);
    }
    float gb2 = 0.f, gw3 = 0.f, gw10 = 0.f, gw11 = 0.f, gb1 = 0.f;
    for (int q = 0; q < P; ++q) {
      gb2 += G2[o * S + q];
      gw3 = fmaf(DV[q], H2[o * S + q], gw3);
      const float d = D1[o * S + q];
      gw10 = fmaf(d, PX[q], gw10);
      gw11 = fmaf(d, PY[q], gw11);
      gb1 += d;
    }
    atomicAdd(grad + kOffB2 + o, gb2);
    atomicAdd(grad + kOffW3 + o, gw3);
    atomicAdd(grad + kOffW1 + 2 * o, gw10);
    atomicAdd(grad + kOffW1 + 2 * o + 1, gw11);
    atomicAdd(grad + kOffB1 + o, gb1);
  }
  if (tid == 0) {
    float gb3 = 0.f;
    double l = 0.0;
    for (int q = 0; q < P; ++q) { gb3 += DV[q]; l += (double)RL[q]; }
    atomicAdd(grad + kOffB3, gb3);
    atomicAdd(loss, l / (double)npts);
  }
}
static_assert(kTrainThreads == kMlpHidden, "one weight-gradient row per thread");

// Adam (Kingma & Ba 2015) with bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// theta (FP32) -> the shared-memory image used in-path (BF16 64x64 layer).
__global__ void mlp_stage_kernel(const float* __restrict__ theta, MlpSmem* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpHidden * kMlpHidden) {
    const int o = i / kMlpHidden, u = i % kMlpHidden;
    const __nv_bfloat16 w = __float2bfloat16_rn(theta[kOffW2 + i]);
    out->W2[o][u] = w;
    out->W2t[u][o] = w;
  }
  if (i < kMlpHidden * (kW2Pitch - kMlpHidden)) {  // zero the padding
    const int r = i / (kW2Pitch - kMlpHidden), c = kMlpHidden + i % (kW2Pitch - kMlpHidden);
    out->W2[r][c] = __float2bfloat16_rn(0.f);
    out->W2t[r][c] = __float2bfloat16_rn(0.f);
  }
  if (i < kMlpHidden) {
    out->W1[i][0] = theta[kOffW1 + 2 * i];
    out->W1[i][1] = theta[kOffW1 + 2 * i + 1];
    out->b1[i] = theta[kOffB1 + i];
    out->b2[i] = theta[kOffB2 + i];
    out->w3[i] = theta[kOffW3 + i];
  }
  if (i == 0) {
    out->b3 = theta[kOffB3];
    out->pad_[0] = out->pad_[1] = out->pad_[2] = 0.f;
  }
}

__device__ void copy_mlp_to_smem(MlpSmem& dst, const MlpSmem* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) d[i] = s[i];
}

// v and grad v at npts points, one warp per 32 points, with the in-path
// tensor-core routine (all lanes converged; the tail lanes evaluate copies).
__global__ void mlp_eval_kernel(const MlpSmem* __restrict__ img, const float* __restrict__ xy,
                                int64_t npts, float* __restrict__ v, float* __restrict__ gxy) {
  __shared__ __align__(16) MlpSmem M;
  copy_mlp_to_smem(M, img);
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q = p < npts ? p : npts - 1;
  float gx, gy, val;
  mlp_grad_warp<true>(M, xy[2 * q], xy[2 * q + 1], gx, gy, val);
  if (p < npts) {
    if (v) v[p] = val;
    gxy[2 * p] = gx;
    gxy[2 * p + 1] = gy;
  }
}

}  // namespace

size_t mlp_image_bytes() { return sizeof(MlpSmem); }

cudaError_t mlp_stage(const float* theta, void* image, cudaStream_t s) {
  mlp_stage_kernel<<<(kMlpHidden * kMlpHidden + 255) / 256, 256, 0, s>>>(
      theta, reinterpret_cast<MlpSmem*>(image));
  return cudaGetLastError();
}

}  // namespace pdds

using namespace pdds;

namespace {
pdds_status mlp_fail(pdds_status s, const std::string& m) {
  set_global_error(m);
  return s;
}
pdds_status mlp_cuda(cudaError_t e, const char* what) {
  return mlp_fail(PDDS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define MCK(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return mlp_cuda(e_, #call); \
  } while (0)

cudaError_t grad_pass(const float* theta, const float* xy, const float* tgt, int64_t npts,
                      float* grad, double* loss, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrainSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t blocks = (npts + kTrainThreads - 1) / kTrainThreads;
  mlp_grad_kernel<<<(unsigned)blocks, kTrainThreads, kTrainSmemBytes, s>>>(
      theta, xy, tgt, npts, 2.0f / (float)npts, grad, loss);
  return cudaGetLastError();
}
}  // namespace

extern "C" pdds_status pdds_mlp_loss_grad(const float* theta, const float* xy, const float* target,
                                          int64_t npts, float* grad, double* loss,
                                          void* cuda_stream) {
  if (!theta || !xy || !target || !grad || !loss || npts < 1)
    return mlp_fail(PDDS_EINVAL, "mlp_loss_grad: NULL pointer or npts < 1");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  MCK(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s));
  MCK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  MCK(grad_pass(theta, xy, target, npts, grad, loss, s));
  return PDDS_OK;
}

extern "C" pdds_status pdds_mlp_train(float* theta, const float* xy, const float* target,
                                      int64_t npts, int32_t steps, double lr,
                                      double* loss_history_host, void* cuda_stream) {
  if (!theta || !xy || !target || npts < 1 || steps < 1 || !(lr > 0))
    return mlp_fail(PDDS_EINVAL, "mlp_train: NULL pointer, npts < 1, steps < 1 or lr <= 0");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* buf = nullptr;  // grad, m, v
  double* hist = nullptr;
  MCK(cudaMalloc(reinterpret_cast<void**>(&buf), 3 * kMlpParams * sizeof(float)));
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&hist), steps * sizeof(double));
  if (e != cudaSuccess) { cudaFree(buf); return mlp_cuda(e, "mlp_train history alloc"); }
  float *grad = buf, *m = buf + kMlpParams, *v = buf + 2 * kMlpParams;
  auto run = [&]() -> cudaError_t {
    cudaError_t r;
    if ((r = cudaMemsetAsync(buf + kMlpParams, 0, 2 * kMlpParams * sizeof(float), s))) return r;
    if ((r = cudaMemsetAsync(hist, 0, steps * sizeof(double), s))) return r;
    const double b1 = 0.9, b2 = 0.999;
    for (int t = 1; t <= steps; ++t) {
      if ((r = cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s))) return r;
      if ((r = grad_pass(theta, xy, target, npts, grad, hist + (t - 1), s))) return r;
      adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(
          theta, grad, m, v, kMlpParams, (float)lr, (float)b1, (float)b2,
          (float)(1.0 - std::pow(b1, t)), (float)(1.0 - std::pow(b2, t)), 1e-8f);
      if ((r = cudaGetLastError())) return r;
    }
    if (loss_history_host) {
      if ((r = cudaMemcpyAsync(loss_history_host, hist, steps * sizeof(double),
                               cudaMemcpyDeviceToHost, s)))
        return r;
    }
    return cudaStreamSynchronize(s);
  };
  e = run();
  cudaFree(buf);
  cudaFree(hist);
  if (e != cudaSuccess) return mlp_cuda(e, "mlp_train");
  return PDDS_OK;
}

extern "C" pdds_status pdds_mlp_eval(const float* theta, const float* xy, int64_t npts, float* v,
                                     float* grad_xy, void* cuda_stream) {
  if (!theta || !xy || !grad_xy || npts < 1)
    return mlp_fail(PDDS_EINVAL, "mlp_eval: NULL pointer or npts < 1");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* img = nullptr;
  MCK(cudaMalloc(&img, sizeof(MlpSmem)));
  cudaError_t e = mlp_stage(theta, img, s);
  if (e == cudaSuccess) {
    const int64_t blocks = (npts + 255) / 256;
    mlp_eval_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const MlpSmem*>(img), xy,
                                                      npts, v, grad_xy);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(img);
  if (e != cudaSuccess) return mlp_cuda(e, "mlp_eval");
  return PDDS_OK;
}
