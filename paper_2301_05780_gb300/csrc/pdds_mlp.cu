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

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <string>
#include <vector>

#include "pdds.h"
#include "pdds_internal.h"
#include "mlp_train.h"
#include "pdds_mlp.cuh"

namespace pdds {
namespace {

// ------------------------------------------------------------- training
// One launch = one full-batch gradient of the loss (1/N) sum_p (v(x_p) -
// target_p)^2 and, in the training variant, the Adam step that follows it.
//
// A CTA takes tiles of 64 points; 256 threads form a 16 x 16 grid, thread
// (ty, tx) owning a 4 x 4 micro-tile (rows 4ty.., columns 4tx..) of each
// 64 x 64 product of the tile:
//   forward   a2[p][o] = b2[o] + sum_u h1[p][u] W2[o][u]
//   backward  dW2[o][u] += sum_p g2[p][o] h1[p][u]      (kept in registers
//                                                       across the CTA's tiles)
//             dh1[p][u] = sum_o g2[p][o] W2[o][u]
// with h1 and g2 = dL/da2 staged in shared memory (rows padded to 68 floats:
// the two row groups a warp reads fall in different banks).  The CTA's
// partial gradient is added to grad with FP32 reductions.
//
// Training: launch t first applies the Adam update t (Kingma & Ba 2015) to
// the previous launch's parameters with the previous launch's gradient --
// every CTA computes it into its own shared-memory image of theta, CTA 0
// writes theta, m and v back -- then takes the gradient at the new theta.
// Gradients rotate through three buffers (accumulated in launch t, read in
// t + 1, cleared by CTA 0 in t + 2 for t + 3), theta, m and v through two,
// so no launch reads what it writes and nothing waits on other CTAs.  The
// CTA that arrives last (a counter) advances the step index and the powers
// beta^t; launch `steps` applies the last update only.  The step index lives
// on the device, so identical launches can be queued.
constexpr int kTileP = 64;
constexpr int kMR = 4;                              // rows of a thread's micro-tile
constexpr int kTrainThreads = 16 * (kTileP / kMR);  // 16 column groups x kTileP / kMR row groups
constexpr int kLd = 68;
struct TrainSmem {
  float W2r[kMlpHidden][kLd];  // W2[o][u]
  float W2c[kMlpHidden][kLd];  // W2[o][u] at [u][o]
  float H1[kTileP][kLd];       // SiLU(a1)   [p][u]
  float G2[kTileP][kLd];       // dL/da2     [p][o]
  float w1x[kMlpHidden], w1y[kMlpHidden], b1[kMlpHidden], b2[kMlpHidden], w3[kMlpHidden];
  float b3;
  float red_b3[kTileP / kMR];
  double red_loss[kTileP / kMR];
};
constexpr size_t kTrainSmemBytes = sizeof(TrainSmem);
// the end-of-CTA column sums [5][16][64] are staged over h1 and g2 (adjacent)
static_assert(offsetof(TrainSmem, G2) == offsetof(TrainSmem, H1) + sizeof(float) * kTileP * kLd,
              "g2 follows h1");
static_assert(5 * (kTrainThreads / 32) * 64 <= 2 * kTileP * kLd,
              "column-sum staging fits in h1 and g2");

// Parameter i of theta (layout W1[64][2], b1, W2[64][64], b2, w3, b3) into
// the shared-memory image.
__device__ __forceinline__ void stage_param(TrainSmem& S, int i, float w) {
  if (i < kOffB1) {
    if (i & 1) S.w1y[i >> 1] = w;
    else S.w1x[i >> 1] = w;
  } else if (i < kOffW2) {
    S.b1[i - kOffB1] = w;
  } else if (i < kOffB2) {
    const int j = i - kOffW2;
    S.W2r[j >> 6][j & 63] = w;
    S.W2c[j & 63][j >> 6] = w;
  } else if (i < kOffW3) {
    S.b2[i - kOffB2] = w;
  } else if (i < kOffB3) {
    S.w3[i - kOffW3] = w;
  } else {
    S.b3 = w;
  }
}

__device__ __forceinline__ float logistic(float a) { return 1.0f / (1.0f + __expf(-a)); }

template <bool ADAM>
__global__ void __launch_bounds__(kTrainThreads, 2) mlp_train_kernel(const TrainArgs A) {
  extern __shared__ __align__(16) unsigned char train_smem[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(train_smem);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  constexpr int kPer = (kMlpParams + kTrainThreads - 1) / kTrainThreads;
  int t = 0;
  if constexpr (ADAM) {
    t = __ldcg(&A.st->t);
    if (t > A.steps) return;  // a launch queued past the last one
  }
  const bool grad_pass = !ADAM || t < A.steps;
  if (!ADAM || t == 0) {
    // theta as given; launch 0 of a training run also keeps a copy
    float w[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kTrainThreads;
      w[q] = i < kMlpParams ? A.theta[i] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kTrainThreads;
      if (i < kMlpParams) {
        stage_param(S, i, w[q]);
        if (ADAM && blockIdx.x == 0) A.th2[i] = w[q];
      }
    }
  } else if (grad_pass || blockIdx.x == 0) {
    // Adam update t from the parameters, moments and gradient of launch t - 1
    const int rd = ((t - 1) & 1) * kMlpParams, wr = (t & 1) * kMlpParams;
    const float* gp = A.grad + ((t - 1) % 3) * kMlpParams;
    const float c1 = (float)(1.0 - __ldcg(&A.st->p1)), c2 = (float)(1.0 - __ldcg(&A.st->p2));
    float g[kPer], mo[kPer], vo[kPer], to[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kTrainThreads;
      if (i < kMlpParams) {
        g[q] = __ldcg(gp + i);
        mo[q] = __ldcg(A.m2 + rd + i);
        vo[q] = __ldcg(A.v2 + rd + i);
        to[q] = __ldcg(A.th2 + rd + i);
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kTrainThreads;
      if (i < kMlpParams) {
        const float mi = A.beta1 * mo[q] + (1.f - A.beta1) * g[q];
        const float vi = A.beta2 * vo[q] + (1.f - A.beta2) * g[q] * g[q];
        const float th = to[q] - A.lr * (mi / c1) / (sqrtf(vi / c2) + A.eps);
        stage_param(S, i, th);
        if (blockIdx.x == 0) {
          A.th2[wr + i] = th;
          A.m2[wr + i] = mi;
          A.v2[wr + i] = vi;
          if (!grad_pass) A.theta[i] = th;  // the last update: the result
        }
      }
    }
  }
  if (ADAM && blockIdx.x == 0) {
    // clear the gradient buffer launch t + 1 accumulates into (last read by t - 1)
    float* gz = A.grad + ((t + 1) % 3) * kMlpParams;
    for (int i = tid; i < kMlpParams; i += kTrainThreads) gz[i] = 0.f;
  }
  __syncthreads();
  if (grad_pass) {
  float* gacc = A.grad + (ADAM ? (t % 3) * kMlpParams : 0);
  const int c0 = 4 * tx, r0 = kMR * ty;
  float dW2[kMR][4] = {};                          // o = r0 + i, u = c0 + j
  float gw1x[4] = {}, gw1y[4] = {}, gb1[4] = {};  // u = c0 + j
  float gb2[4] = {}, gw3[4] = {};                 // o = c0 + j
  float gb3 = 0.f;
  double lsum = 0.0;
  const int64_t ntiles = (A.npts + kTileP - 1) / kTileP;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p0 = tile * kTileP + r0;
    float px[kMR], py[kMR], pt[kMR];
    bool pv[kMR];
#pragma unroll
    for (int i = 0; i < kMR; ++i) {
      pv[i] = p0 + i < A.npts;
      px[i] = pv[i] ? A.xy[2 * (p0 + i)] : 0.f;
      py[i] = pv[i] ? A.xy[2 * (p0 + i) + 1] : 0.f;
      pt[i] = pv[i] ? A.tgt[p0 + i] : 0.f;
    }
    // h1 = SiLU(W1 x + b1) and SiLU'(a1) of this thread's (p, u) block
    float d1[kMR][4];
    {
      const float4 wx = *reinterpret_cast<const float4*>(&S.w1x[c0]);
      const float4 wy = *reinterpret_cast<const float4*>(&S.w1y[c0]);
      const float4 bb = *reinterpret_cast<const float4*>(&S.b1[c0]);
      const float cwx[4] = {wx.x, wx.y, wx.z, wx.w}, cwy[4] = {wy.x, wy.y, wy.z, wy.w};
      const float cb[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
      for (int i = 0; i < kMR; ++i) {
        float h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float a = fmaf(cwx[j], px[i], fmaf(cwy[j], py[i], cb[j]));
          const float sg = logistic(a);
          h[j] = pv[i] ? a * sg : 0.f;
          d1[i][j] = sg * (1.f + a * (1.f - sg));
        }
        *reinterpret_cast<float4*>(&S.H1[r0 + i][c0]) = make_float4(h[0], h[1], h[2], h[3]);
      }
    }
    __syncthreads();
    // forward: a2 = h1 W2^T + b2 (p = r0 + i, o = c0 + j)
    float acc[kMR][4];
    {
      const float4 bb = *reinterpret_cast<const float4*>(&S.b2[c0]);
#pragma unroll
      for (int i = 0; i < kMR; ++i) {
        acc[i][0] = bb.x; acc[i][1] = bb.y; acc[i][2] = bb.z; acc[i][3] = bb.w;
      }
    }
#pragma unroll 8
    for (int u = 0; u < kMlpHidden; ++u) {
      const float4 w = *reinterpret_cast<const float4*>(&S.W2c[u][c0]);
      const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int i = 0; i < kMR; ++i) {
        const float h = S.H1[r0 + i][u];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(h, wv[j], acc[i][j]);
      }
    }
    // h2, v, the residual, and g2 = dL/da2 = (2/N) r w3 SiLU'(a2)
    {
      const float4 w = *reinterpret_cast<const float4*>(&S.w3[c0]);
      const float cw3[4] = {w.x, w.y, w.z, w.w};
      const float b3 = S.b3;
#pragma unroll
      for (int i = 0; i < kMR; ++i) {
        float h2[4], sp[4], vp = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float a = acc[i][j];
          const float sg = logistic(a);
          h2[j] = a * sg;
          sp[j] = sg * (1.f + a * (1.f - sg));
          vp = fmaf(cw3[j], h2[j], vp);
        }
        // v: sum over the 16 column groups (lanes with equal ty, one half-warp)
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) vp += __shfl_xor_sync(0xffffffffu, vp, off);
        const float r = pv[i] ? (vp + b3) - pt[i] : 0.f;
        const float dv = A.scale * r;
        float g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          g[j] = dv * cw3[j] * sp[j];
          gb2[j] += g[j];
          gw3[j] = fmaf(dv, h2[j], gw3[j]);
        }
        *reinterpret_cast<float4*>(&S.G2[r0 + i][c0]) = make_float4(g[0], g[1], g[2], g[3]);
        if (tx == 0) {
          gb3 += dv;
          lsum += (double)(r * r);
        }
      }
    }
    __syncthreads();
    // dW2[o][u] += sum_p g2[p][o] h1[p][u] (o = r0 + i, u = c0 + j)
#pragma unroll 8
    for (int p = 0; p < kTileP; ++p) {
      float gv[kMR];
      if constexpr (kMR == 4) {
        const float4 g = *reinterpret_cast<const float4*>(&S.G2[p][r0]);
        gv[0] = g.x; gv[1] = g.y; gv[2] = g.z; gv[3] = g.w;
      } else {
        const float2 g = *reinterpret_cast<const float2*>(&S.G2[p][r0]);
        gv[0] = g.x; gv[1] = g.y;
      }
      const float4 h = *reinterpret_cast<const float4*>(&S.H1[p][c0]);
      const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
      for (int i = 0; i < kMR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dW2[i][j] = fmaf(gv[i], hv[j], dW2[i][j]);
    }
    // dh1[p][u] = sum_o g2[p][o] W2[o][u] (p = r0 + i, u = c0 + j), then
    // da1 = dh1 SiLU'(a1) into the first layer's gradient
    {
      float dh[kMR][4] = {};
#pragma unroll 8
      for (int o = 0; o < kMlpHidden; ++o) {
        const float4 w = *reinterpret_cast<const float4*>(&S.W2r[o][c0]);
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < kMR; ++i) {
          const float g = S.G2[r0 + i][o];
#pragma unroll
          for (int j = 0; j < 4; ++j) dh[i][j] = fmaf(g, wv[j], dh[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < kMR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float da = dh[i][j] * d1[i][j];
          gw1x[j] = fmaf(da, px[i], gw1x[j]);
          gw1y[j] = fmaf(da, py[i], gw1y[j]);
          gb1[j] += da;
        }
    }
    __syncthreads();  // h1 and g2 are overwritten by the next tile
  }
  // ---- the CTA's partial gradient into grad
#pragma unroll
  for (int i = 0; i < kMR; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(gacc + kOffW2 + (r0 + i) * kMlpHidden + c0 + j, dW2[i][j]);
  // column sums: the two row groups of a warp (lanes 0-15, 16-31) by a
  // shuffle, then over the warps (staged over h1 and g2)
  constexpr int kWarps = kTrainThreads / 32;
  float* red = &S.H1[0][0];  // [5][kWarps][64]
  const int wp = tid >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float v[5] = {gw1x[j], gw1y[j], gb1[j], gb2[j], gw3[j]};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float sum2 = v[q] + __shfl_xor_sync(0xffffffffu, v[q], 16);
      if (!(tid & 16)) red[(q * kWarps + wp) * 64 + c0 + j] = sum2;
    }
  }
  if (tx == 0) {
    S.red_b3[ty] = gb3;
    S.red_loss[ty] = lsum;
  }
  __syncthreads();
  for (int e = tid; e < 5 * 64; e += kTrainThreads) {
    const int q = e >> 6, c = e & 63;
    float sum = 0.f;
#pragma unroll
    for (int r = 0; r < kWarps; ++r) sum += red[(q * kWarps + r) * 64 + c];
    const int off = q == 0 ? kOffW1 + 2 * c : q == 1 ? kOffW1 + 2 * c + 1
                  : q == 2 ? kOffB1 + c : q == 3 ? kOffB2 + c : kOffW3 + c;
    atomicAdd(gacc + off, sum);
  }
  if (tid == 0) {
    float b = 0.f;
    double l = 0.0;
    for (int r = 0; r < kTileP / kMR; ++r) { b += S.red_b3[r]; l += S.red_loss[r]; }
    atomicAdd(gacc + kOffB3, b);
    atomicAdd(A.loss + t, l * A.inv_n);
  }
  }
  if constexpr (ADAM) {
    // the last CTA to arrive advances the step: every CTA read t and the
    // powers before its arrival, and nothing else in this launch depends on
    // what the last one writes
    if (tid == 0 && atomicAdd(&A.st->count, 1u) == gridDim.x - 1) {
      A.st->count = 0;
      A.st->p1 = (t == 0 ? 1.0 : A.st->p1) * (double)A.beta1;
      A.st->p2 = (t == 0 ? 1.0 : A.st->p2) * (double)A.beta2;
      A.st->t = t + 1;
    }
  }
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

// CTAs of a gradient launch: one per 64-point tile, at most two per SM (the
// occupancy the shared-memory footprint allows).
cudaError_t train_grid(int64_t npts, unsigned* grid) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static bool attr[256] = {};  // per device: the shared-memory opt-in
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(mlp_train_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTrainSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_train_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTrainSmemBytes);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (npts + kTileP - 1) / kTileP;
  *grid = (unsigned)std::min<int64_t>(tiles, 2 * (int64_t)sms);
  return cudaSuccess;
}

// Kernel and launch shape of a training engine: 0 the FP32 SIMT kernel, 1 the
// tensor-core kernel.
cudaError_t train_config(int engine, bool adam, int64_t npts, const void** fn, unsigned* grid,
                         unsigned* threads, size_t* smem) {
  if (engine == 1) return train_tc_launch_config(adam, npts, fn, grid, threads, smem);
  cudaError_t e = train_grid(npts, grid);
  if (e != cudaSuccess) return e;
  *fn = adam ? reinterpret_cast<const void*>(&mlp_train_kernel<true>)
             : reinterpret_cast<const void*>(&mlp_train_kernel<false>);
  *threads = kTrainThreads;
  *smem = kTrainSmemBytes;
  return cudaSuccess;
}

cudaError_t launch_train(const void* fn, unsigned grid, unsigned threads, size_t smem,
                         const TrainArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<TrainArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

pdds_status loss_grad_impl(int engine, const char* name, const float* theta, const float* xy,
                           const float* target, int64_t npts, float* grad, double* loss,
                           void* cuda_stream) {
  if (!theta || !xy || !target || !grad || !loss || npts < 1)
    return mlp_fail(PDDS_EINVAL, std::string(name) + ": NULL pointer or npts < 1");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const void* fn = nullptr;
  unsigned grid = 0, threads = 0;
  size_t smem = 0;
  MCK(train_config(engine, false, npts, &fn, &grid, &threads, &smem));
  MCK(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s));
  MCK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  TrainArgs a{};
  a.theta = const_cast<float*>(theta);  // the gradient variant does not write theta
  a.xy = xy;
  a.tgt = target;
  a.npts = npts;
  a.scale = 2.0f / (float)npts;
  a.inv_n = 1.0 / (double)npts;
  a.grad = grad;
  a.loss = loss;
  MCK(launch_train(fn, grid, threads, smem, a, s));
  return PDDS_OK;
}
}  // namespace

extern "C" pdds_status pdds_mlp_loss_grad(const float* theta, const float* xy, const float* target,
                                          int64_t npts, float* grad, double* loss,
                                          void* cuda_stream) {
  return loss_grad_impl(0, "mlp_loss_grad", theta, xy, target, npts, grad, loss, cuda_stream);
}

extern "C" pdds_status pdds_mlp_loss_grad_tc(const float* theta, const float* xy,
                                             const float* target, int64_t npts, float* grad,
                                             double* loss, void* cuda_stream) {
  return loss_grad_impl(1, "mlp_loss_grad_tc", theta, xy, target, npts, grad, loss, cuda_stream);
}

namespace {
pdds_status train_impl(int engine, const char* name, float* theta, const float* xy,
                       const float* target, int64_t npts, int32_t steps, double lr,
                       double* loss_history_host, void* cuda_stream) {
  if (!theta || !xy || !target || npts < 1 || steps < 1 || !(lr > 0))
    return mlp_fail(PDDS_EINVAL,
                    std::string(name) + ": NULL pointer, npts < 1, steps < 1 or lr <= 0");
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const void* fn = nullptr;
  unsigned grid = 0, threads = 0;
  size_t smem = 0;
  MCK(train_config(engine, true, npts, &fn, &grid, &threads, &smem));
  // scratch: three gradients and two each of theta, m, v (FP32), the step
  // state, the loss history
  const size_t fbytes = 9 * kMlpParams * sizeof(float);
  const size_t sbytes = (fbytes + 15) / 16 * 16;
  const size_t bytes = sbytes + sizeof(TrainState) + (size_t)steps * sizeof(double);
  char* buf = nullptr;
  MCK(cudaMalloc(reinterpret_cast<void**>(&buf), bytes));
  float* f = reinterpret_cast<float*>(buf);
  TrainArgs a{};
  a.theta = theta;
  a.xy = xy;
  a.tgt = target;
  a.npts = npts;
  a.scale = 2.0f / (float)npts;
  a.inv_n = 1.0 / (double)npts;
  a.grad = f;
  a.th2 = f + 3 * kMlpParams;
  a.m2 = f + 5 * kMlpParams;
  a.v2 = f + 7 * kMlpParams;
  a.st = reinterpret_cast<TrainState*>(buf + sbytes);
  a.loss = reinterpret_cast<double*>(buf + sbytes + sizeof(TrainState));
  a.steps = steps;
  a.lr = (float)lr;
  a.beta1 = 0.9f;
  a.beta2 = 0.999f;
  a.eps = 1e-8f;
  auto run = [&]() -> cudaError_t {
    cudaError_t r = cudaMemsetAsync(buf, 0, bytes, s);
    if (r != cudaSuccess) return r;
    // steps + 1 launches (gradients 0..steps-1, updates 1..steps) run as a
    // CUDA graph of 64 identical launches replayed on a private stream (the
    // launch index is read on the device; launches past the last return at
    // once): one graph launch per 64 kernel launches.
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto body = [&]() -> cudaError_t {
      cudaError_t q;
      if ((q = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) return q;
      if ((q = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return q;
      if ((q = cudaEventRecord(ev, s))) return q;
      if ((q = cudaStreamWaitEvent(cs, ev, 0))) return q;
      const int launches = steps + 1;
      const int chunk = std::min(launches, 64);
      if ((q = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))) return q;
      cudaError_t lq = cudaSuccess;
      for (int k = 0; k < chunk && lq == cudaSuccess; ++k)
        lq = launch_train(fn, grid, threads, smem, a, cs);
      q = cudaStreamEndCapture(cs, &graph);
      if (lq) return lq;
      if (q) return q;
      if ((q = cudaGraphInstantiate(&exec, graph, 0))) return q;
      for (int done = 0; done < launches; done += chunk)
        if ((q = cudaGraphLaunch(exec, cs))) return q;
      if ((q = cudaEventRecord(ev, cs))) return q;
      return cudaStreamWaitEvent(s, ev, 0);
    };
    r = body();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (r == cudaSuccess && cs) r = cudaStreamSynchronize(cs);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    if (r != cudaSuccess) return r;
    if (loss_history_host) {
      r = cudaMemcpyAsync(loss_history_host, a.loss, steps * sizeof(double),
                          cudaMemcpyDeviceToHost, s);
      if (r != cudaSuccess) return r;
    }
    return cudaStreamSynchronize(s);
  };
  cudaError_t e = run();
  cudaFree(buf);
  if (e != cudaSuccess) return mlp_cuda(e, name);
  return PDDS_OK;
}
}  // namespace

extern "C" pdds_status pdds_mlp_train(float* theta, const float* xy, const float* target,
                                      int64_t npts, int32_t steps, double lr,
                                      double* loss_history_host, void* cuda_stream) {
  return train_impl(0, "mlp_train", theta, xy, target, npts, steps, lr, loss_history_host,
                    cuda_stream);
}

extern "C" pdds_status pdds_mlp_train_tc(float* theta, const float* xy, const float* target,
                                         int64_t npts, int32_t steps, double lr,
                                         double* loss_history_host, void* cuda_stream) {
  return train_impl(1, "mlp_train_tc", theta, xy, target, npts, steps, lr, loss_history_host,
                    cuda_stream);
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
