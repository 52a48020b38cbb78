// The network v_theta (2 -> 64 -> 64 -> 1, SiLU; Eq. 11, 37-39) on the
// fifth-generation tensor cores: v and grad v at many points, tile by tile.
//
// A CTA of two warpgroups (256 threads); each warpgroup takes its own tiles of
// 128 points, thread t of the group owning point t of the tile (TMEM lane t),
// with its own operand buffers, mbarrier and TMEM columns, and synchronises on
// its own named barrier, so the two groups' MMAs and SIMT work overlap.
// Per tile:
//   layer 1 (FP32 SIMT)    a1 = W1 x + b1, h1 = SiLU(a1), SiLU'(a1) kept
//   forward (tcgen05)      D1 = h1 W2^T            [128 x 64], TMEM cols 0-63
//   output  (FP32 SIMT)    a2 = D1 + b2, v = w3 . SiLU(a2) + b3,
//                          g2 = w3 * SiLU'(a2) = dv / da2
//   backward (tcgen05)     D2 = g2 W2               [128 x 64], TMEM cols 64-127
//   input gradient (SIMT)  grad v = W1^T (D2 * SiLU'(a1))
// h1 and g2 are the M x K operand (K-major, 128-byte swizzle), W2 and W2^T
// the N x K operands, staged once per CTA.  Every product is the 3xTF32 split
// (tc_sm103.cuh), so v and grad v carry FP32 rounding only.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "pdds.h"
#include "pdds_internal.h"
#include "tc_sm103.cuh"

namespace pdds {
namespace {

constexpr int kH = 64;    // hidden width
constexpr int kTP = 128;  // points per tile = MMA M
constexpr int kOffW2 = 192, kOffB1 = 128, kOffB2 = 4288, kOffW3 = 4352, kOffB3 = 4416;

constexpr int kGroups = 2;  // warpgroups per CTA

struct alignas(1024) EvalTcSmem {
  float B1[2][kH * kH];           // W2 as N = out x K = in, hi and lo parts
  float B2[2][kH * kH];           // W2^T as N = in x K = out
  float A[kGroups][2][kTP * kH];  // per group: h1, then g2 (M = point x K = unit)
  float w1x[kH], w1y[kH], b1[kH], b2[kH], w3[kH];
  float b3;
  unsigned long long mbar[kGroups];
  unsigned tmem;
};
constexpr size_t kEvalTcSmemBytes = sizeof(EvalTcSmem) + 1024;  // + alignment slack

// 1 / (1 + e^-a) with the fast reciprocal-based division (a few ulp; 0 when
// e^-a overflows)
__device__ __forceinline__ float logistic(float a) { return __fdividef(1.0f, 1.0f + __expf(-a)); }
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kTP) : "memory");
}

__device__ __forceinline__ void put_split(float* hi_base, float* lo_base, int off_bytes, float4 v) {
  float4 h = make_float4(tc::tf32_hi(v.x), tc::tf32_hi(v.y), tc::tf32_hi(v.z), tc::tf32_hi(v.w));
  float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
  *reinterpret_cast<float4*>(reinterpret_cast<char*>(hi_base) + off_bytes) = h;
  *reinterpret_cast<float4*>(reinterpret_cast<char*>(lo_base) + off_bytes) = l;
}

// D (TMEM, 64 columns at d) = A B^T with the 3xTF32 split: 3 x 8 K-steps.
__device__ __forceinline__ void mma_3xtf32(unsigned d, const float* const (&A)[2],
                                           const float* const (&B)[2]) {
  constexpr uint32_t idesc = tc::idesc_tf32(kTP, kH);
  bool acc = false;
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    const int ia = pr == 2 ? 1 : 0, ib = pr == 1 ? 1 : 0;  // hi hi, hi lo, lo hi
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const unsigned ka = (kk >> 2) * kTP * 128 + (kk & 3) * 32;
      const unsigned kb = (kk >> 2) * kH * 128 + (kk & 3) * 32;
      tc::mma_tf32(d, tc::sdesc_k128(tc::smem_addr(A[ia]) + ka),
                   tc::sdesc_k128(tc::smem_addr(B[ib]) + kb), idesc, acc);
      acc = true;
    }
  }
}

__global__ void __launch_bounds__(kGroups * kTP, 1)
    mlp_eval_tc_kernel(const float* __restrict__ theta, const float* __restrict__ xy, int64_t npts,
                       float* __restrict__ v, float* __restrict__ gxy, int* __restrict__ err) {
  extern __shared__ unsigned char eval_raw[];
  EvalTcSmem& S = *reinterpret_cast<EvalTcSmem*>(
      (reinterpret_cast<uintptr_t>(eval_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid / kTP, t = tid % kTP;  // warpgroup, point of the tile
  // the network, staged once: W2 and W2^T split into their TF32 hi / lo parts
  for (int i = tid; i < kH * kH; i += kGroups * kTP) {
    const float w = theta[kOffW2 + i], wh = tc::tf32_hi(w);
    const int o = i / kH, u = i % kH;
    const int ob = tc::swz_offset(o, u, kH), ot = tc::swz_offset(u, o, kH);
    *reinterpret_cast<float*>(reinterpret_cast<char*>(S.B1[0]) + ob) = wh;
    *reinterpret_cast<float*>(reinterpret_cast<char*>(S.B1[1]) + ob) = w - wh;
    *reinterpret_cast<float*>(reinterpret_cast<char*>(S.B2[0]) + ot) = wh;
    *reinterpret_cast<float*>(reinterpret_cast<char*>(S.B2[1]) + ot) = w - wh;
  }
  if (tid < kH) {
    S.w1x[tid] = theta[2 * tid];
    S.w1y[tid] = theta[2 * tid + 1];
    S.b1[tid] = theta[kOffB1 + tid];
    S.b2[tid] = theta[kOffB2 + tid];
    S.w3[tid] = theta[kOffW3 + tid];
  }
  if (tid == 0) {
    S.b3 = theta[kOffB3];
    for (int q = 0; q < kGroups; ++q) tc::mbar_init(&S.mbar[q]);
  }
  if (warp == 0) tc::tmem_alloc(&S.tmem, 128 * kGroups);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // group g: TMEM columns [128 g, 128 g + 128); its warps read lanes 32 (warp % 4) ..
  const unsigned tm = S.tmem + 128u * g;
  const unsigned lane = (unsigned)((warp & 3) * 32) << 16;
  float* const A0 = S.A[g][0];
  float* const A1 = S.A[g][1];
  const float* const Aop[2] = {A0, A1};
  const float* const B1op[2] = {S.B1[0], S.B1[1]};
  const float* const B2op[2] = {S.B2[0], S.B2[1]};
  unsigned long long* const mbar = &S.mbar[g];
  unsigned phase = 0;
  bool ok = true;
  for (int64_t tile = (int64_t)kGroups * blockIdx.x + g; tile * kTP < npts;
       tile += (int64_t)kGroups * gridDim.x) {
    const int64_t p = tile * kTP + t;
    const bool valid = p < npts;
    const float x = valid ? xy[2 * p] : 0.f, y = valid ? xy[2 * p + 1] : 0.f;
    // layer 1: h1 into the A tile, SiLU'(a1) kept
    float s1[kH];
#pragma unroll
    for (int c = 0; c < kH / 4; ++c) {
      float h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = 4 * c + j;
        const float a = fmaf(S.w1x[u], x, fmaf(S.w1y[u], y, S.b1[u]));
        const float sg = logistic(a);
        h[j] = a * sg;
        s1[u] = sg * (1.0f + a * (1.0f - sg));
      }
      put_split(A0, A1, tc::swz_chunk(t, c, kTP), make_float4(h[0], h[1], h[2], h[3]));
    }
    tc::fence_async_smem();
    tc::fence_before();
    group_sync(g);
    if (t == 0) {
      tc::fence_after();
      mma_3xtf32(tm, Aop, B1op);
      tc::commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, 2000000000ull) && ok;
    phase ^= 1u;
    tc::fence_after();
    // a2 -> v and g2 = w3 SiLU'(a2) (into the A tile: the forward MMA is done)
    float vs = S.b3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float d[32];
      tc::tmem_ld32(tm + lane + 32 * half, d);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int o = 32 * half + 4 * c + j;
          const float a = d[4 * c + j] + S.b2[o];
          const float sg = logistic(a);
          vs = fmaf(S.w3[o], a * sg, vs);
          g[j] = S.w3[o] * (sg * (1.0f + a * (1.0f - sg)));
        }
        put_split(A0, A1, tc::swz_chunk(t, 8 * half + c, kTP),
                  make_float4(g[0], g[1], g[2], g[3]));
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    group_sync(g);
    if (t == 0) {
      tc::fence_after();
      mma_3xtf32(tm + 64, Aop, B2op);
      tc::commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, 2000000000ull) && ok;
    phase ^= 1u;
    tc::fence_after();
    // grad v = W1^T (dh1 * SiLU'(a1))
    float gx = 0.f, gy = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float d[32];
      tc::tmem_ld32(tm + lane + 64 + 32 * half, d);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int u = 32 * half + j;
        const float da = d[j] * s1[u];
        gx = fmaf(da, S.w1x[u], gx);
        gy = fmaf(da, S.w1y[u], gy);
      }
    }
    if (valid) {
      if (v) v[p] = vs;
      gxy[2 * p] = gx;
      gxy[2 * p + 1] = gy;
    }
    // TMEM reads of this tile done before the group's next MMAs
    tc::fence_before();
    group_sync(g);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(S.tmem, 128 * kGroups);
  }
  if (!ok && t == 0) atomicExch(err, (int)PDDS_ETIMEOUT);
}

}  // namespace
}  // namespace pdds

using namespace pdds;

extern "C" pdds_status pdds_mlp_eval_tc(const float* theta, const float* xy, int64_t npts, float* v,
                                        float* grad_xy, void* cuda_stream) {
  if (!theta || !xy || !grad_xy || npts < 1) {
    set_global_error("mlp_eval_tc: NULL pointer or npts < 1");
    return PDDS_EINVAL;
  }
  (void)cudaGetLastError();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int* d_err = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_eval_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kEvalTcSmemBytes);
  if (e == cudaSuccess) {
    const int64_t tiles = (npts + kTP - 1) / kTP;
    const int grid = (int)std::min<int64_t>((tiles + kGroups - 1) / kGroups, sms);
    mlp_eval_tc_kernel<<<grid, kGroups * kTP, kEvalTcSmemBytes, s>>>(theta, xy, npts, v, grad_xy,
                                                                      d_err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) {
    set_global_error(std::string("mlp_eval_tc: ") + cudaGetErrorString(e));
    return PDDS_ECUDA;
  }
  if (herr != 0) {
    set_global_error("mlp_eval_tc: a tensor-core wait ran out (results incomplete)");
    return PDDS_ETIMEOUT;
  }
  return PDDS_OK;
}
