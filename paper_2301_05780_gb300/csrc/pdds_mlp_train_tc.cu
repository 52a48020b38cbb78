// Training of v_theta (Eq. 11, 37-39; the fit of Phase I, Sec. 4.3) with the
// three 64 x 64 products of a step on the fifth-generation tensor cores
// (tcgen05.mma kind::f16: BF16 operands, FP32 accumulators in TMEM).
//
// A CTA of two warpgroups takes tiles of 128 points: thread p of a group owns
// point p of the tile (and TMEM lane p), and group g computes hidden units
// [32 g, 32 g + 32) of every point (the two halves of v meet in shared
// memory).  Per tile:
//   layer 1 (FP32)        a1 = W1 x + b1, h1 = SiLU(a1); SiLU'(a1) into TMEM
//   forward  (tcgen05)    D = h1 W2^T                 (M = 128 points, N = 64, K = 64)
//   output   (FP32)       h2 = SiLU(D + b2), v = w3 . h2 + b3, r = v - target,
//                         g2 = (2/N) r w3 * SiLU'(a2) = dL/da2
//   backward (tcgen05)    D = g2 W2                   (M = 128 points, N = 64, K = 64)
//                         g1 = D * SiLU'(a1) = dL/da1
//   gradient (tcgen05)    [g2 | g1]^T [h1 | x | y | 1]  (M = 128 units, N = 80,
//                         K = 128 points) and h2^T dv (N = 16), accumulated in
//                         TMEM over the CTA's tiles: dW2, db2, dW1, db1 and dw3
// The point-major tiles (h1, g2) are the K-major A operands of the forward and
// backward products; the gradient products contract over the points, so each
// thread also writes its column of the unit-major tiles (g2^T, g1^T, h2^T,
// h1^T, x, y, 1, dv).  All tiles are K-major BF16 with the 128-byte swizzle.
//
// The Adam step, the rotation of the gradient, parameter and moment buffers
// across launches and the step counter are those of the FP32 kernel
// (pdds_mlp.cu); only the gradient differs, by the BF16 rounding of the
// products' operands.  Waits on the tensor core are bounded (2 s); a wait
// that runs out turns the step's loss into NaN.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "mlp_train.h"
#include "pdds.h"
#include "pdds_mlp.cuh"
#include "tc_sm103.cuh"

namespace pdds {
namespace {

constexpr int kTT = 128;         // points per tile = MMA M
constexpr int kThreads = 2 * kTT;  // two warpgroups, each half of the hidden units
constexpr int kHU = kMlpHidden;  // 64
constexpr int kGR = 192;         // rows of the gradient A tile: g2^T, g1^T, h2^T
constexpr int kBR = 80;          // rows of the gradient B tile: h1^T, x, y, 1, zeros
constexpr int kVR = 16;          // rows of the dv tile: dv, zeros
// TMEM columns: the forward / backward product, SiLU'(a1), the gradient
// accumulators [g2 | g1]^T [h1 | x | y | 1] and h2^T dv
constexpr unsigned kColD = 0, kColS1 = 64, kColG = 128, kColW3 = 208, kTmemCols = 256;
constexpr uint64_t kWaitNs = 2000000000ull;

struct alignas(1024) TrainTcSmem {
  uint16_t W2o[kHU * kHU];  // forward B: W2 as N = out x K = in
  uint16_t W2t[kHU * kHU];  // backward B: W2^T as N = in x K = out
  uint16_t P[kTT * kHU];    // forward / backward A: h1, then g2 (M = point x K = unit)
  uint16_t GA[kGR * kTT];   // gradient A: unit rows x K = point (two 64-point atom columns)
  uint16_t GB[kBR * kTT];   // gradient B: h1^T, x, y, 1, zeros
  uint16_t DV[kVR * kTT];   // dv, zeros
  // W1[:, 0], W1[:, 1], b1, b2 and w3 halved (the SiLU algebra works with
  // a/2), w3 as it is (v)
  float w1xh[kHU], w1yh[kHU], b1h[kHU], b2h[kHU], w3h[kHU], w3[kHU];
  float b3;
  float red_v[2][kTT];  // the two groups' parts of v
  float red_b3[kThreads / 32];
  double red_loss[kThreads / 32];
  unsigned long long mbar;
  unsigned tmem;
};
constexpr size_t kTrainTcSmemBytes = sizeof(TrainTcSmem) + 1024;  // + alignment slack

// Byte offset of element (r, k) of a K-major, 128-byte-swizzled BF16 tile
// with R rows per 64-element atom column: the 16-byte chunk c of row r of an
// atom column sits at chunk position c ^ (r % 8), 8-row groups 1024 bytes
// apart, atom columns R * 128 bytes apart.
__device__ __forceinline__ int bo(int r, int k, int R) {
  return (k >> 6) * R * 128 + (r >> 3) * 1024 + (r & 7) * 128 +
         ((((k & 63) >> 3) ^ (r & 7)) << 4) + ((k & 7) << 1);
}
__device__ __forceinline__ void put_bf16(uint16_t* tile, int off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(tile) + off) = __float2bfloat16_rn(v);
}

// Parameter i of theta into the shared-memory image: W2 as the two BF16 B
// operands (the forward one halved, so that the product gives a2/2; halving
// is exact), the vectors of the SiLU algebra halved.
__device__ __forceinline__ void stage_tc(TrainTcSmem& S, int i, float w) {
  if (i < kOffB1) {
    if (i & 1) S.w1yh[i >> 1] = 0.5f * w;
    else S.w1xh[i >> 1] = 0.5f * w;
  } else if (i < kOffW2) {
    S.b1h[i - kOffB1] = 0.5f * w;
  } else if (i < kOffB2) {
    const int j = i - kOffW2, o = j >> 6, u = j & 63;
    put_bf16(S.W2o, bo(o, u, kHU), 0.5f * __bfloat162float(__float2bfloat16_rn(w)));
    put_bf16(S.W2t, bo(u, o, kHU), w);
  } else if (i < kOffW3) {
    S.b2h[i - kOffB2] = 0.5f * w;
  } else if (i < kOffB3) {
    S.w3[i - kOffW3] = w;
    S.w3h[i - kOffW3] = 0.5f * w;
  } else {
    S.b3 = w;
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 tanh2(float2 a) { return f2(tanh_approx(a.x), tanh_approx(a.y)); }
// With a' = a/2 and t = tanh(a'): SiLU(a) = a' (1 + t), and
// SiLU'(a) = (1 + u) / 2 with u = t + a' (1 - t^2).
__device__ __forceinline__ float2 silu_u(float2 a, float2 t) {
  return __ffma2_rn(a, __ffma2_rn(t, f2(-t.x, -t.y), f2(1.0f, 1.0f)), t);
}

// D [+]= A B^T over nk K-steps of 16 points or units; A and B K-major with Ra
// and Rb rows per atom column (four K-steps per atom column).
__device__ __forceinline__ void mma_ksteps(unsigned d, unsigned a, int Ra, unsigned b, int Rb,
                                           int nk, uint32_t idesc, bool accumulate) {
  for (int kk = 0; kk < nk; ++kk) {
    const unsigned ka = (unsigned)((kk >> 2) * Ra * 128 + (kk & 3) * 32);
    const unsigned kb = (unsigned)((kk >> 2) * Rb * 128 + (kk & 3) * 32);
    tc::mma_bf16(d, tc::sdesc_k128(a + ka), tc::sdesc_k128(b + kb), idesc, accumulate || kk > 0);
  }
}

template <bool ADAM>
__global__ void __launch_bounds__(kThreads, 2) mlp_train_tc_kernel(const TrainArgs A) {
  extern __shared__ __align__(128) unsigned char tsm_raw[];
  char* const sbase =
      reinterpret_cast<char*>(tsm_raw) + ((1024u - (tc::smem_addr(tsm_raw) & 1023u)) & 1023u);
  TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(sbase);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kPer = (kMlpParams + kThreads - 1) / kThreads;
  int t = 0;
  if constexpr (ADAM) {
    t = __ldcg(&A.st->t);
    if (t > A.steps) return;  // a launch queued past the last one
  }
  const bool grad_pass = !ADAM || t < A.steps;
  if (!ADAM || t == 0) {
    // theta as given; launch 0 of a training run also keeps a copy
    float w_[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kThreads;
      w_[q] = i < kMlpParams ? A.theta[i] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kThreads;
      if (i < kMlpParams) {
        const float w = w_[q];
        stage_tc(S, i, w);
        if (ADAM && blockIdx.x == 0) A.th2[i] = w;
      }
    }
  } else if (grad_pass || blockIdx.x == 0) {
    // Adam update t from the parameters, moments and gradient of launch t - 1
    const int rd = ((t - 1) & 1) * kMlpParams, wr = (t & 1) * kMlpParams;
    const float* gp = A.grad + ((t - 1) % 3) * kMlpParams;
    const float c1 = (float)(1.0 - __ldcg(&A.st->p1)), c2 = (float)(1.0 - __ldcg(&A.st->p2));
    // all of a thread's loads in flight at once, then the updates
    float g_[kPer], m_[kPer], v_[kPer], t_[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kThreads;
      if (i < kMlpParams) {
        g_[q] = __ldcg(gp + i);
        m_[q] = __ldcg(A.m2 + rd + i);
        v_[q] = __ldcg(A.v2 + rd + i);
        t_[q] = __ldcg(A.th2 + rd + i);
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = tid + q * kThreads;
      if (i < kMlpParams) {
        const float g = g_[q];
        const float mi = A.beta1 * m_[q] + (1.f - A.beta1) * g;
        const float vi = A.beta2 * v_[q] + (1.f - A.beta2) * g * g;
        const float th = t_[q] - A.lr * (mi / c1) / (sqrtf(vi / c2) + A.eps);
        stage_tc(S, i, th);
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
    for (int i = tid; i < kMlpParams; i += kThreads) gz[i] = 0.f;
  }
  // rows 64-79 of the gradient B tile (x, y and 1 are rewritten per tile, the
  // rest stay zero) and the whole dv tile
  for (int i = tid; i < 2 * 16 * 128 / 16; i += kThreads) {
    const int a = i / 128, w = i % 128;  // atom column, 16-byte word within rows 64-79
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.GB) + a * kBR * 128 + 8 * 1024 + 16 * w) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = tid; i < kVR * kTT * 2 / 16; i += kThreads)
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.DV) + 16 * i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) tc::mbar_init(&S.mbar);
  if (warp == 0) tc::tmem_alloc(&S.tmem, kTmemCols);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // warpgroup g takes hidden units [32 g, 32 g + 32) of every point; thread
  // pl of the group owns point pl of the tile and TMEM lane pl
  const int g = tid / kTT, pl = tid % kTT;
  const unsigned tm = S.tmem, tl = (unsigned)((warp & 3) * 32) << 16;
  const unsigned sP = tc::smem_addr(S.P), sGA = tc::smem_addr(S.GA), sGB = tc::smem_addr(S.GB);
  const unsigned sDV = tc::smem_addr(S.DV);
  unsigned phase = 0;
  bool ok = true;
  float gb3 = 0.f;
  double lsum = 0.0;
  int done = 0;  // tiles this CTA has taken
  const int64_t ntiles = grad_pass ? (A.npts + kTT - 1) / kTT : 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * kTT + pl;
    const bool valid = p < A.npts;
    const float x = valid ? A.xy[2 * p] : 0.f, y = valid ? A.xy[2 * p + 1] : 0.f;
    const float tg = valid ? A.tgt[p] : 0.f;
    // ---- layer 1: h1 into P (row pl) and h1^T (column pl), SiLU'(a1) into TMEM
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      const int q = 2 * g + qq;  // 16-unit chunk
      float s1[16];
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        uint32_t hp[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int u = 16 * q + 8 * c2 + 2 * j;
          const float2 a = __ffma2_rn(ld2(&S.w1xh[u]), f2(x, x),
                                      __ffma2_rn(ld2(&S.w1yh[u]), f2(y, y), ld2(&S.b1h[u])));
          const float2 t = tanh2(a);
          const float2 h = __ffma2_rn(a, t, a);                                    // SiLU(a1)
          const float2 d = __ffma2_rn(f2(0.5f, 0.5f), silu_u(a, t), f2(0.5f, 0.5f));  // SiLU'
          const float h0 = valid ? h.x : 0.f, h1 = valid ? h.y : 0.f;
          hp[j] = pack_bf16x2(h0, h1);
          s1[8 * c2 + 2 * j] = d.x;
          s1[8 * c2 + 2 * j + 1] = d.y;
          put_bf16(S.GB, bo(u, pl, kBR), h0);
          put_bf16(S.GB, bo(u + 1, pl, kBR), h1);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.P) + bo(pl, 16 * q + 8 * c2, kTT)) =
            make_uint4(hp[0], hp[1], hp[2], hp[3]);
      }
      tc::tmem_st16(tm + tl + kColS1 + 16 * q, s1);
    }
    if (g == 0) {
      put_bf16(S.GB, bo(64, pl, kBR), x);
      put_bf16(S.GB, bo(65, pl, kBR), y);
      put_bf16(S.GB, bo(66, pl, kBR), valid ? 1.f : 0.f);
    }
    tc::st_wait();
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_ksteps(tm + kColD, sP, kTT, tc::smem_addr(S.W2o), kHU, 4, tc::idesc_bf16(kTT, kHU),
                 false);
      tc::commit(&S.mbar);
    }
    ok = tc::mbar_wait(&S.mbar, phase, kWaitNs) && ok;
    phase ^= 1u;
    tc::fence_after();
    // ---- output: h2^T (column pl) and the group's part of v; then v, the
    // residual, dv, and g2 into P and g2^T
    float2 us[16];  // u of each unit pair: SiLU'(a2) = (1 + u) / 2
    float2 vp = f2(0.f, 0.f);
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      const int q = 2 * g + qq;
      float a2[16];
      tc::tmem_ld16(tm + tl + kColD + 16 * q, a2);  // a2 / 2 - b2 / 2
#pragma unroll
      for (int j = 0; j < 16; j += 2) {
        const int o = 16 * q + j;
        const float2 a = __fadd2_rn(f2(a2[j], a2[j + 1]), ld2(&S.b2h[o]));
        const float2 t = tanh2(a);
        const float2 h = __ffma2_rn(a, t, a);  // SiLU(a2)
        us[8 * qq + j / 2] = silu_u(a, t);
        vp = __ffma2_rn(ld2(&S.w3[o]), h, vp);
        put_bf16(S.GA, bo(128 + o, pl, kGR), h.x);
        put_bf16(S.GA, bo(128 + o + 1, pl, kGR), h.y);
      }
    }
    S.red_v[g][pl] = vp.x + vp.y;
    __syncthreads();
    const float vs = S.b3 + S.red_v[0][pl] + S.red_v[1][pl];  // the same in both groups
    const float r = valid ? vs - tg : 0.f;
    const float dv = A.scale * r;
    if (g == 0) {
      lsum += (double)r * (double)r;
      gb3 += dv;
      put_bf16(S.DV, bo(0, pl, kVR), dv);
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = 4 * g + cc;  // 8-unit chunk
      uint32_t gp[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = 8 * c + 2 * j;
        const float2 dw = __fmul2_rn(ld2(&S.w3h[o]), f2(dv, dv));
        const float2 gg = __ffma2_rn(dw, us[4 * cc + j], dw);  // dv w3 SiLU'(a2)
        const float g0 = gg.x, g1 = gg.y;
        gp[j] = pack_bf16x2(g0, g1);
        put_bf16(S.GA, bo(o, pl, kGR), g0);
        put_bf16(S.GA, bo(o + 1, pl, kGR), g1);
      }
      *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.P) + bo(pl, 8 * c, kTT)) =
          make_uint4(gp[0], gp[1], gp[2], gp[3]);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      mma_ksteps(tm + kColD, sP, kTT, tc::smem_addr(S.W2t), kHU, 4, tc::idesc_bf16(kTT, kHU),
                 false);
      tc::commit(&S.mbar);
    }
    ok = tc::mbar_wait(&S.mbar, phase, kWaitNs) && ok;
    phase ^= 1u;
    tc::fence_after();
    // ---- g1 = dh1 * SiLU'(a1) into g1^T (column pl)
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      const int q = 2 * g + qq;
      float dh[16], s1[16];
      tc::tmem_ld16(tm + tl + kColD + 16 * q, dh);
      tc::tmem_ld16(tm + tl + kColS1 + 16 * q, s1);
#pragma unroll
      for (int j = 0; j < 16; ++j) put_bf16(S.GA, bo(64 + 16 * q + j, pl, kGR), dh[j] * s1[j]);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      // [g2 | g1]^T [h1 | x | y | 1]: rows 0-127 of GA against GB
      mma_ksteps(tm + kColG, sGA, kGR, sGB, kBR, 8, tc::idesc_bf16(kTT, kBR), done > 0);
      // h2^T dv: rows 64-191 of GA (the last 64 are h2^T) against the dv tile
      mma_ksteps(tm + kColW3, sGA + 8 * 1024, kGR, sDV, kVR, 8, tc::idesc_bf16(kTT, kVR),
                 done > 0);
      tc::commit(&S.mbar);
    }
    // the next tile rewrites the operand tiles: wait here
    ok = tc::mbar_wait(&S.mbar, phase, kWaitNs) && ok;
    phase ^= 1u;
    tc::fence_after();
    ++done;
  }
  if (done > 0) {
    // ---- the CTA's partial gradient: TMEM lane pl holds accumulator row pl;
    // the two groups split the columns
    float* gacc = A.grad + (ADAM ? (t % 3) * kMlpParams : 0);
    float gv[16];
    if ((warp & 3) < 2) {  // rows 0-63: output unit o = pl
      const int o = pl;
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * g + qq;
        tc::tmem_ld16(tm + tl + kColG + 16 * q, gv);
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(gacc + kOffW2 + o * kHU + 16 * q + j, gv[j]);
      }
      if (g == 0) {
        tc::tmem_ld16(tm + tl + kColG + 64, gv);
        atomicAdd(gacc + kOffB2 + o, gv[2]);
      }
    } else if (g == 0) {  // rows 64-127: hidden unit u = pl - 64
      const int u = pl - 64;
      tc::tmem_ld16(tm + tl + kColG + 64, gv);
      atomicAdd(gacc + kOffW1 + 2 * u, gv[0]);
      atomicAdd(gacc + kOffW1 + 2 * u + 1, gv[1]);
      atomicAdd(gacc + kOffB1 + u, gv[2]);
    } else {
      const int u = pl - 64;
      tc::tmem_ld16(tm + tl + kColW3, gv);
      atomicAdd(gacc + kOffW3 + u, gv[0]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
      lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if (lane == 0) {
      S.red_b3[warp] = gb3;
      S.red_loss[warp] = lsum;
    }
    __syncthreads();
    if (tid == 0) {
      float b = 0.f;
      double l = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { b += S.red_b3[w]; l += S.red_loss[w]; }
      atomicAdd(gacc + kOffB3, b);
      atomicAdd(A.loss + t, l * A.inv_n);
    }
  }
  if (!ok && tid == 0) atomicAdd(A.loss + t, __longlong_as_double(0x7ff8000000000000ll));
  if constexpr (ADAM) {
    // the last CTA to arrive advances the step (as in the FP32 kernel)
    if (tid == 0 && atomicAdd(&A.st->count, 1u) == gridDim.x - 1) {
      A.st->count = 0;
      A.st->p1 = (t == 0 ? 1.0 : A.st->p1) * (double)A.beta1;
      A.st->p2 = (t == 0 ? 1.0 : A.st->p2) * (double)A.beta2;
      A.st->t = t + 1;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tm, kTmemCols);
  }
}

}  // namespace

cudaError_t train_tc_launch_config(bool adam, int64_t npts, const void** fn, unsigned* grid,
                                   unsigned* threads, size_t* smem) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static bool attr[256] = {};  // per device: the shared-memory opt-in
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(mlp_train_tc_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainTcSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(mlp_train_tc_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainTcSmemBytes);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (npts + kTT - 1) / kTT;
  // two CTAs per SM: shared memory (~107 KB each) and TMEM (256 columns each)
  *grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * (int64_t)sms));
  *fn = adam ? reinterpret_cast<const void*>(&mlp_train_tc_kernel<true>)
             : reinterpret_cast<const void*>(&mlp_train_tc_kernel<false>);
  *threads = kThreads;
  *smem = kTrainTcSmemBytes;
  return cudaSuccess;
}

}  // namespace pdds
