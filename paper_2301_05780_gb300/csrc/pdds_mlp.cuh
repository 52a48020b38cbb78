// v_theta : R^2 -> R (2 -> 64 -> 64 -> 1, SiLU) for the pathwise control
// variate xi = -int Y sigma^T grad v . dW of Eq. 37 (variance reduction of
// Eq. 11, 38-39).  This header holds the warp-batched evaluation of grad v used
// inside the path kernel: the 32 lanes of a warp each hold one path position,
// the 64x64 layer runs on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation), everything else is FP32.
//
// Parameter vector theta (FP32, 4417 values): W1[64][2], b1[64], W2[64][64]
// (row = output unit), b2[64], w3[64], b3.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace pdds {

constexpr int kMlpHidden = 64;
constexpr int kMlpParams = 64 * 2 + 64 + 64 * 64 + 64 + 64 + 1;
constexpr int kW2Pitch = 72;  // bf16 per padded row: 36 words, conflict-free fragment loads

// The network as staged in shared memory (17.9 KB), built once per control
// variate by the host from theta.
struct MlpSmem {
  __nv_bfloat16 W2[kMlpHidden][kW2Pitch];   // [out][in]   B operand of h1 W2^T
  __nv_bfloat16 W2t[kMlpHidden][kW2Pitch];  // [in][out]   B operand of g2 W2
  float W1[kMlpHidden][2];
  float b1[kMlpHidden];
  float b2[kMlpHidden];
  float w3[kMlpHidden];
  float b3;
  float pad_[3];
};

// Bytes the staged network takes at the start of a CV path kernel's dynamic
// shared memory (128-byte aligned so the unit ring keeps its alignment).
constexpr int kMlpSmemBytes = (int)((sizeof(MlpSmem) + 127) / 128 * 128);

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// logistic(a) = 1/2 + tanh(a/2)/2; SiLU(a) = a logistic(a);
// SiLU'(a) = s (1 + a (1 - s)).
__device__ __forceinline__ void silu_and_slope(float a, float& h, float& d) {
  const float s = fmaf(0.5f, tanh_approx(0.5f * a), 0.5f);
  h = a * s;
  d = fmaf(h, 1.0f - s, s);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Whole warp (all 32 lanes converged): lane L holds the point (x, y) and gets
// back grad v at its own point (and v if want_value).  Rows of the MMA tiles
// are points: m-tile mt covers lanes 16 mt .. 16 mt + 15; the thread with
// group g = lane / 4 and t = lane % 4 owns rows g and g + 8 of a tile and units
// 16 kt + 2t + {0, 1, 8, 9} of each 16-unit k-tile kt.  The layer-2
// accumulator is reused in place as the A operand of the backward product
// (the C and A fragments hold the same (row, unit) pairs), so no shared memory
// round trip is needed between the two products.
template <bool WANT_VALUE>
__device__ __forceinline__ void mlp_grad_warp(const MlpSmem& M, float x, float y, float& gx,
                                              float& gy, float& v) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  gx = 0.f;
  gy = 0.f;
  v = 0.f;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    const int p0 = 16 * mt + g, p1 = p0 + 8;
    const float x0 = __shfl_sync(0xffffffffu, x, p0), y0 = __shfl_sync(0xffffffffu, y, p0);
    const float x1 = __shfl_sync(0xffffffffu, x, p1), y1 = __shfl_sync(0xffffffffu, y, p1);
    // ---- layer 1 in A-fragment layout: h1 (bf16) and SiLU'(a1) (fp32)
    uint32_t A[4][4];
    uint32_t D1[4][4];  // SiLU'(a1) for rows (g, g + 8) of each unit, packed BF16 pairs
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {                 // unit u = 16kt + 2t + {0,1} + 8*(j>>1)
        const int u = 16 * kt + 2 * t + (j & 1) + 8 * (j >> 1);
        const float w0 = M.W1[u][0], w1 = M.W1[u][1], bb = M.b1[u];
        float h0, d0, h1, d1;
        silu_and_slope(fmaf(w0, x0, fmaf(w1, y0, bb)), h0, d0);   // row g
        silu_and_slope(fmaf(w0, x1, fmaf(w1, y1, bb)), h1, d1);   // row g + 8
        D1[kt][j] = pack_bf16x2(d0, d1);
        // stash h in D-order first; packed below
        if (j == 0) { A[kt][0] = __float_as_uint(h0); A[kt][1] = __float_as_uint(h1); }
        if (j == 1) {
          A[kt][0] = pack_bf16x2(__uint_as_float(A[kt][0]), h0);
          A[kt][1] = pack_bf16x2(__uint_as_float(A[kt][1]), h1);
        }
        if (j == 2) { A[kt][2] = __float_as_uint(h0); A[kt][3] = __float_as_uint(h1); }
        if (j == 3) {
          A[kt][2] = pack_bf16x2(__uint_as_float(A[kt][2]), h0);
          A[kt][3] = pack_bf16x2(__uint_as_float(A[kt][3]), h1);
        }
      }
    }
    // ---- layer 2: a2 = h1 W2^T + b2, two n-tiles (16 output units) at a time,
    // each turned at once into dv/da2 = w3 SiLU'(a2), the A fragment of the
    // backward product for that 16-unit k-tile (keeps few accumulators live)
    uint32_t A2[4][4];
    float vr0 = 0.f, vr1 = 0.f;
#pragma unroll
    for (int kt2 = 0; kt2 < 4; ++kt2) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int nt = 2 * kt2 + half;
        float C[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* row = reinterpret_cast<const uint32_t*>(&M.W2[8 * nt + g][0]);
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
          mma_bf16(C, A[kt][0], A[kt][1], A[kt][2], A[kt][3], row[8 * kt + t], row[8 * kt + 4 + t]);
        const int o0 = 8 * nt + 2 * t;
        float h, d, e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = o0 + (q & 1);
          silu_and_slope(C[q] + M.b2[o], h, d);
          e[q] = M.w3[o] * d;
          if (WANT_VALUE) { if (q < 2) vr0 = fmaf(M.w3[o], h, vr0); else vr1 = fmaf(M.w3[o], h, vr1); }
        }
        A2[kt2][0 + 2 * half] = pack_bf16x2(e[0], e[1]);  // row g
        A2[kt2][1 + 2 * half] = pack_bf16x2(e[2], e[3]);  // row g + 8
      }
    }
    // ---- dv/dh1 = (dv/da2) W2, then dv/da1 = dv/dh1 SiLU'(a1), then W1^T
    float gx0 = 0.f, gy0 = 0.f, gx1 = 0.f, gy1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float G[4] = {0.f, 0.f, 0.f, 0.f};
      const uint32_t* row = reinterpret_cast<const uint32_t*>(&M.W2t[8 * nt + g][0]);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
        mma_bf16(G, A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3], row[8 * kt + t], row[8 * kt + 4 + t]);
      const int kt1 = nt >> 1, jb = (nt & 1) * 2;   // same units as layer-1 element j
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int u = 8 * nt + 2 * t + q;
        const float w0 = M.W1[u][0], w1 = M.W1[u][1];
        const __nv_bfloat162 dd = *reinterpret_cast<const __nv_bfloat162*>(&D1[kt1][jb + q]);
        const float r0 = G[q] * __low2float(dd);        // row g
        const float r1 = G[2 + q] * __high2float(dd);   // row g + 8
        gx0 = fmaf(w0, r0, gx0); gy0 = fmaf(w1, r0, gy0);
        gx1 = fmaf(w0, r1, gx1); gy1 = fmaf(w1, r1, gy1);
      }
    }
    // ---- reduce over the quad (the four threads sharing rows g, g + 8)
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      gx0 += __shfl_xor_sync(0xffffffffu, gx0, o);
      gy0 += __shfl_xor_sync(0xffffffffu, gy0, o);
      gx1 += __shfl_xor_sync(0xffffffffu, gx1, o);
      gy1 += __shfl_xor_sync(0xffffffffu, gy1, o);
      if (WANT_VALUE) {
        vr0 += __shfl_xor_sync(0xffffffffu, vr0, o);
        vr1 += __shfl_xor_sync(0xffffffffu, vr1, o);
      }
    }
    // ---- hand each point's result to its owner lane
    const int r = lane - 16 * mt;              // owner's row in this tile (if 0..15)
    const int src = 4 * (r & 7);
    const float ax = __shfl_sync(0xffffffffu, gx0, src), bx = __shfl_sync(0xffffffffu, gx1, src);
    const float ay = __shfl_sync(0xffffffffu, gy0, src), by = __shfl_sync(0xffffffffu, gy1, src);
    float av = 0.f, bv = 0.f;
    if (WANT_VALUE) {
      av = __shfl_sync(0xffffffffu, vr0, src);
      bv = __shfl_sync(0xffffffffu, vr1, src);
    }
    if (r >= 0 && r < 16) {
      gx = r < 8 ? ax : bx;
      gy = r < 8 ? ay : by;
      if (WANT_VALUE) v = (r < 8 ? av : bv) + M.b3;
    }
  }
}

}  // namespace pdds
