// Persistent Feynman-Kac path kernel of the PDDSparse assembly (sm_103a).
//
// What it computes (arXiv 2301.05780): for every interfacial knot x_k and
// every path p < N_k, the Euler-Maruyama discretisation (Sec. 2.3) of
//   dX = d(X) dt + s(X) dW,  dY = c(X) Y dt,  dZ = -f(X) Y dt   (Eq. 9)
// started at x_k and stopped at the first step outside the closed patch
// Pi(x_k) (Eq. 15); the exit contributes Y g to b_k on the boundary of Omega
// or, on an interface side, Y times the linear interpolation weights of the
// two nearest stencil knots to row k of G (Eq. 21-25).  The FP64 sums become
// G and b in the finalize kernel (Eq. 24-25).
//
// How it runs on the GPU:
//  - one path per lane; a warp steps its 32 paths in lockstep and refills a
//    lane from the CTA's current work unit as soon as a few of its paths have
//    exited (exit times are wildly uneven, so lanes never wait for a whole
//    batch of paths);
//  - work units are (problem, knot, path range) taken from one global atomic
//    queue; each CTA keeps a two-stage ring of units in shared memory (knot
//    data, FP64 slot accumulators, TMA-staged coefficient tiles) so warps move
//    on to the next unit while the stragglers of the previous one finish;
//  - the warp that completes the last path of a unit flushes its accumulators
//    to the CSR values with FP64 atomics and loads the next unit in its place;
//  - positions are integrated in FP32 relative to the knot; accumulation is
//    FP64; every wait is bounded by a timer and reports PDDS_ETIMEOUT;
//  - the extended-exit variants (EXT) take each knot's own step h_k (Sec. 4.2)
//    and can move the patch sides inwards by the Gobet-Menozzi shift
//    0.5826 |s(P)| sqrt(h_k) (Sec. 2.3): a lane tests against the box moved
//    by the largest shift (4 compares, as for the naive exit) and evaluates
//    the per-side shifts only when that cheap test fires.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdds.h"
#include "pdds_internal.h"
#include "pdds_mlp.cuh"
#include "pdds_rbf.cuh"

namespace pdds {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kFixedOne = 1073741824.0f;             // 2^30: one path's full weight
constexpr double kFixedInv = 1.0 / 1073741824.0;       // 2^-30

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications whose high halves are xored with the other words
// and the round key; the key advances by two Weyl constants between rounds.
// rk: the ten round keys of each key word (the key advanced by the Weyl
// constants), precomputed on the host so that every round reads them as
// launch constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = c.x * 0xD2511F53u, hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u, hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// The counter of path p of knot k is (q, p, k, tag) with only q = n / 2
// changing along the path, so the parts of rounds 1 and 2 that depend on p, k
// and tag alone are computed once per path:
//   round 1: (x1, y1) = (hi(M1 k) ^ p ^ key, lo(M1 k)) are constant, and
//            z1 = hi(M0 q) ^ tag ^ key', w1 = lo(M0 q);
//   round 2: the product M0 x1 is constant: z2 = hi(M0 x1) ^ w1 ^ key'',
//            w2 = lo(M0 x1).
// Five of the 60 integer operations of a call, for four more registers per
// lane: the extended-exit kernels without a control variate use it (1.5 %
// faster); the plain ones, held to 56 registers, and the control-variate ones
// spill more with it and run slower.
struct PhiloxPath {
  uint32_t y1;  // lo(M1 k)
  uint32_t c1;  // tag ^ round-1 key of word 3
  uint32_t a2;  // hi(M0 x1) ^ round-2 key of word 3
  uint32_t b2;  // lo(M0 x1)
};
__device__ __forceinline__ PhiloxPath philox_path(uint32_t p, uint32_t k, uint32_t tag,
                                                  const uint32_t (&rk)[20]) {
  PhiloxPath f;
  const uint32_t x1 = __umulhi(k, 0xCD9E8D57u) ^ p ^ rk[0];
  f.y1 = k * 0xCD9E8D57u;
  f.c1 = tag ^ rk[1];
  f.a2 = __umulhi(x1, 0xD2511F53u) ^ rk[3];
  f.b2 = x1 * 0xD2511F53u;
  return f;
}
// Philox4x32-10 of the counter (q, p, k, tag) from the path's constants.
__device__ __forceinline__ uint4 philox_step(uint32_t q, const PhiloxPath& f,
                                             const uint32_t (&rk)[20]) {
  const uint32_t z1 = __umulhi(q, 0xD2511F53u) ^ f.c1, w1 = q * 0xD2511F53u;
  uint4 c = make_uint4(__umulhi(z1, 0xCD9E8D57u) ^ f.y1 ^ rk[2], z1 * 0xCD9E8D57u, f.a2 ^ w1, f.b2);
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint32_t lo0 = c.x * 0xD2511F53u, hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u, hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller (1958) on two 32-bit words: u = (w + 1/2) 2^-32,
// rho = sqrt(-2 ln u_a), theta = 2 pi u_b (reduced to [-pi, pi] before the
// hardware sine/cosine, which is exact in value).  u_a keeps all 32 bits (its
// logarithm decides the tail of rho); u_b is built from its top 23 bits,
// (w_b >> 9 + 1/2) 2^-23, which moves theta by at most 2^-23 pi.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float s32 = 2.3283064365386963e-10f;  // 2^-32
  const float ua = fmaf(__uint2float_rn(a), s32, 0.5f * s32);
  const float rho = sqrt_approx(-1.38629436111989061f * lg2_approx(ua));  // -2 ln u_a
  // u_b - 1/2 in [-1/2, 1/2) (both steps exact): cos and sin of 2 pi u_b are
  // minus those of 2 pi (u_b - 1/2), absorbed by the sign of rho
  const float r = (__uint_as_float(0x3f800000u | (b >> 9)) - 1.5f) + 5.9604644775390625e-8f;
  float sn, cs;
  __sincosf(kTwoPi * r, &sn, &cs);
  z0 = -rho * cs;
  z1 = -rho * sn;
}

// Packed FP32 pairs (Blackwell FFMA2 / FMUL2 / FADD2: one instruction for two
// independent FP32 operations, each rounded exactly as its scalar form).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Box-Muller on all four words of one Philox call, both pairs at once in
// packed arithmetic (the same operations as box_muller, so the same values):
// gA = rho_a (cos, sin) of the angle of r.y, gB likewise from r.z, r.w.  These
// are the NEGATED normals of box_muller (z = -g), i.e. dW = -sqrt(h) g.
__device__ __forceinline__ void box_muller4(uint4 r, float2& gA, float2& gB) {
  const float s32 = 2.3283064365386963e-10f;  // 2^-32
  const float2 ua = fma2(f2(__uint2float_rn(r.x), __uint2float_rn(r.z)), f2(s32, s32),
                         f2(0.5f * s32, 0.5f * s32));
  const float2 l = mul2(f2(-1.38629436111989061f, -1.38629436111989061f),
                        f2(lg2_approx(ua.x), lg2_approx(ua.y)));  // -2 ln u
  const float ra = sqrt_approx(l.x), rb = sqrt_approx(l.y);
  float2 t = f2(__uint_as_float(0x3f800000u | (r.y >> 9)), __uint_as_float(0x3f800000u | (r.w >> 9)));
  t = add2(add2(t, f2(-1.5f, -1.5f)), f2(5.9604644775390625e-8f, 5.9604644775390625e-8f));
  t = mul2(f2(kTwoPi, kTwoPi), t);
  float sa, ca, sb, cb;
  __sincosf(t.x, &sa, &ca);
  __sincosf(t.y, &sb, &cb);
  gA = mul2(f2(ra, ra), f2(ca, sa));
  gB = mul2(f2(rb, rb), f2(cb, sb));
}

// sin(2 pi t), cos(2 pi t) for any t (argument reduced to [-1/2, 1/2]).
__device__ __forceinline__ void sincos_2pi(float t, float& s, float& c) {
  const float r = t - rintf(t);
  __sincosf(kTwoPi * r, &s, &c);
}

// --------------------------------------------------------------- the stage
// One entry of a CTA's two-stage unit ring, at the start of its slice of
// dynamic shared memory; the FP64 slot accumulators and the coefficient tiles
// follow it.
struct alignas(16) Stage {
  // ctrl = state << 32 | next path to hand out.  state = 2q while unit q (the
  // q-th unit of this CTA) is published, 2q+1 while it is being loaded.  Paths
  // are claimed with one 64-bit shared atomic add, so a claim always knows
  // which unit it came from.
  unsigned long long ctrl;
  int term;       // 1: the global queue is empty, no unit here
  int prob, k;
  int p_begin, p_end, total;
  int done;       // paths finished (shared atomic)
  int tma_phase;
  int tile_w;
  int LX, LY, tag, coef_id;
  float h, sqh;       // step of this unit's knot (extended kernels)
  float gmc;          // Gobet-Menozzi shift per unit of |s|: 0.5826 sqrt(h), or 0
  float sigma_max;    // bound of s(x) (the moved box of the cheap test)
  long long kmax;     // step cap of this knot
  KnotDesc kd;
  float x0, y0, x1, y1, dx, dy, inv_dx, inv_dy;
  float params[8];
  float tab_inv_dx, tab_inv_dy;
  int tab_imax, tab_jmax;
  double bsum;
  unsigned long long mbar;
};
constexpr int kStageHdr = (int)((sizeof(Stage) + 127) / 128 * 128);

struct Smem {
  char* base;
  int stage_bytes, acc_bytes, tile_bytes;
  int* live;    // units loaded (or being loaded) and not yet flushed, this CTA
  int* qempty;  // 1 once a load found the global queue empty
  __device__ Stage& st(int s) const { return *reinterpret_cast<Stage*>(base + s * stage_bytes); }
  // Slot accumulators: exact 64-bit fixed point in units of 2^-30 of a path's
  // weight (weights are <= 1, a unit has <= 2^24 paths, so sums stay < 2^54);
  // integer shared atomics, independent of the order in which paths finish.
  __device__ unsigned long long* acc(int s) const {
    return reinterpret_cast<unsigned long long*>(base + s * stage_bytes + kStageHdr);
  }
  // TABLE: field 0 is the interleaved (s, c) tile (field 1 is not used).
  __device__ float* tile(int s, int field) const {
    return reinterpret_cast<float*>(base + s * stage_bytes + kStageHdr + acc_bytes +
                                    field * tile_bytes);
  }
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned ctrl_state(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.cta.shared::cta.b64 %0, [%1];" : "=l"(v) : "r"(smem_u32(p)) : "memory");
  return (unsigned)(v >> 32);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------- mbarrier/TMA
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, int parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ----------------------------------------------------------- coefficients
// tanh q = 1 - 2 / (e^{2q} + 1) (|q| <= 2 for the problem below).
__device__ __forceinline__ float tanh_small(float q) {
  return 1.0f - __fdividef(2.0f, __expf(2.0f * q) + 1.0f);
}

// The Poisson problem of Sec. 5.1 (Eq. 42-43): u = 3 + sin(r)/3 + tanh(q)/3 with
// r = sqrt(1 + x^2/100 + y^2/50), q = sin a + sin b, a = 3x/25 + y/20,
// b = x/20 - 3y/25; f = Lap u by the chain rule:
//   Lap sin r = cos r Lap r - sin r G / r^2,  Lap r = 0.03 / r - G / r^3,
//   G = x^2/100^2 + y^2/50^2;  Lap tanh q = (1 - T^2)(Lap q - 2 T |grad q|^2),
//   Lap q = -((3/25)^2 + (1/20)^2) q.
struct E1Terms {
  float sr, cr, q, T, sa, ca, sb, cb;
};
// sin and cos of an angle a in radians: the hardware sine on a itself when
// the host has bounded |a| to a few tens of radians (direct), else after an
// exact reduction to [-1/2, 1/2] turn.
__device__ __forceinline__ void sincos_rad(float a, bool direct, float& s, float& c) {
  if (direct) __sincosf(a, &s, &c);
  else sincos_2pi(a * 0.15915494309189535f, s, c);
}
// The terms of u at (x, y) given r.  direct: |x|, |y| <= 256, so every angle
// is below 45 rad.
__device__ __forceinline__ E1Terms e1_terms(float x, float y, float r, bool direct) {
  E1Terms t;
  sincos_rad(r, direct, t.sr, t.cr);
  sincos_rad(fmaf(0.12f, x, 0.05f * y), direct, t.sa, t.ca);
  sincos_rad(fmaf(0.05f, x, -0.12f * y), direct, t.sb, t.cb);
  t.q = t.sa + t.sb;
  t.T = tanh_small(t.q);
  return t;
}
__device__ __forceinline__ float e1_r2(float x, float y) {
  return fmaf(x * x, 0.01f, fmaf(y * y, 0.02f, 1.0f));
}
// u (boundary data, once per exit): r by the correctly rounded square root.
__device__ __forceinline__ float e1_u(float x, float y) {
  const E1Terms t = e1_terms(x, y, sqrtf(e1_r2(x, y)), false);
  return fmaf(t.sr + t.T, 0.333333343f, 3.0f);
}
// f = Lap u (every step): 1/r from the hardware reciprocal square root
// (r^2 >= 1; a few ulp, far below the FP32 path rounding), r = r^2 / r.
__device__ __forceinline__ float e1_lap(float x, float y, bool direct) {
  const float r2 = e1_r2(x, y);
  const float ir = rsqrtf(r2);
  const E1Terms t = e1_terms(x, y, r2 * ir, direct);
  const float Gi2 = fmaf(x * x, 1e-4f, y * y * 4e-4f) * (ir * ir);  // G / r^2
  const float lap_r = ir * (0.03f - Gi2);                           // 0.03 / r - G / r^3
  const float lap_sin = fmaf(t.cr, lap_r, -t.sr * Gi2);
  const float qx = fmaf(0.12f, t.ca, 0.05f * t.cb);
  const float qy = fmaf(0.05f, t.ca, -0.12f * t.cb);
  const float lap_q = -0.0169f * t.q;
  const float lap_tanh = (1.0f - t.T * t.T) * fmaf(-2.0f * t.T, fmaf(qx, qx, qy * qy), lap_q);
  return (lap_sin + lap_tanh) * 0.333333343f;
}

// Boundary data g (Eq. 6) of each coefficient set.
template <int COEF>
__device__ __forceinline__ float g_value(const Stage& H, float x, float y) {
  if constexpr (COEF == PDDS_COEF_LAPLACE_EXPSIN) {
    float s, c;
    sincos_2pi(y * (1.0f / kTwoPi), s, c);
    return __expf(x) * s;
  } else if constexpr (COEF == PDDS_COEF_MANUFACTURED) {
    float sx, cx, sy, cy;
    sincos_2pi(0.5f * x, sx, cx);
    sincos_2pi(0.5f * y, sy, cy);
    return sx * cy + x * y;
  } else if constexpr (COEF == PDDS_COEF_VARSIGMA) {
    float s, c;
    sincos_2pi(y * (0.5f / kTwoPi), s, c);
    return __expf(0.25f * x) * c;
  } else if constexpr (COEF == PDDS_COEF_TABLE) {
    return H.params[1];
  } else if constexpr (COEF == PDDS_COEF_POISSON_E1) {
    return e1_u(x, y);
  } else {
    return H.params[5];
  }
}

// Both tabulated fields at once from the interleaved (s, c) tile: four 8-byte
// shared loads instead of eight 4-byte ones.
__device__ __forceinline__ void bilinear2(const float* T, int w, float fx, float fy, int imax,
                                          int jmax, float& s, float& c) {
  int i = (int)floorf(fx), j = (int)floorf(fy);
  i = min(max(i, 0), imax);
  j = min(max(j, 0), jmax);
  const float tx = fx - (float)i, ty = fy - (float)j;
  const float2* r0 = reinterpret_cast<const float2*>(T) + j * w + i;
  const float2* r1 = r0 + w;
  const float2 a = r0[0], b = r0[1], d = r1[0], e = r1[1];
  const float s0 = fmaf(tx, b.x - a.x, a.x), s1 = fmaf(tx, e.x - d.x, d.x);
  const float c0 = fmaf(tx, b.y - a.y, a.y), c1 = fmaf(tx, e.y - d.y, d.y);
  s = fmaf(ty, s1 - s0, s0);
  c = fmaf(ty, c1 - c0, c0);
}

__device__ __forceinline__ float bilinear(const float* T, int w, float fx, float fy, int imax,
                                          int jmax) {
  int i = (int)floorf(fx), j = (int)floorf(fy);
  i = min(max(i, 0), imax);
  j = min(max(j, 0), jmax);
  const float tx = fx - (float)i, ty = fy - (float)j;
  const float* r0 = T + j * w + i;
  const float* r1 = r0 + w;
  const float a = fmaf(tx, r0[1] - r0[0], r0[0]);
  const float b = fmaf(tx, r1[1] - r1[0], r1[0]);
  return fmaf(ty, b - a, a);
}

// Coefficients s, d, c, f at the absolute point (x, y); (xr, yr) is the same
// point relative to the knot (used by the tabulated set).
template <int COEF>
__device__ __forceinline__ void coeffs(const Stage& H, const float* tsig, const float* tc,
                                       float x, float y, float xr, float yr, bool trig_direct,
                                       float& s, float& dx, float& dy, float& c, float& f) {
  if constexpr (COEF == PDDS_COEF_LAPLACE_EXPSIN) {
    s = 1.41421356237309505f; dx = 0.f; dy = 0.f; c = 0.f; f = 0.f;
  } else if constexpr (COEF == PDDS_COEF_MANUFACTURED) {
    // u = sin(pi x) cos(pi y) + x y, Lap u = -2 pi^2 sin(pi x) cos(pi y),
    // d = (sin 2 pi y, cos 2 pi x), c = -(1 + x^2), f = Lap u + d.grad u + c u.
    float sx, cx, sy, cy;
    const float pi = 3.14159265358979324f;
    if (trig_direct) {  // |x|, |y| <= 1 (set on the host): pi x is within [-pi, pi]
      const float2 a = mul2(f2(pi, pi), f2(x, y));
      __sincosf(a.x, &sx, &cx);
      __sincosf(a.y, &sy, &cy);
    } else {
      sincos_2pi(0.5f * x, sx, cx);
      sincos_2pi(0.5f * y, sy, cy);
    }
    const float sxcy = sx * cy;
    // (u, 1 + x^2), (u_x, u_y) and (2 sin(pi y), -2 sin(pi x)) as packed pairs
    const float2 u_c = fma2(f2(x, x), f2(y, x), f2(sxcy, 1.0f));
    const float2 uxy = fma2(mul2(f2(pi, -pi), f2(cx, sx)), f2(cy, sy), f2(y, x));
    const float2 t2 = mul2(f2(2.0f, -2.0f), f2(sy, sx));
    const float lap = (-2.0f * pi * pi) * sxcy;
    s = 1.41421356237309505f;
    dx = t2.x * cy;
    dy = fmaf(t2.y, sx, 1.0f);
    c = -u_c.y;
    f = fmaf(dx, uxy.x, fmaf(dy, uxy.y, fmaf(c, u_c.x, lap)));
  } else if constexpr (COEF == PDDS_COEF_VARSIGMA) {
    // s = sqrt2 (1 + 0.3 sin 2 pi x sin 2 pi y), c = -1, u = e^{x/4} cos(y/2),
    // f = (s^2/2)(1/16 - 1/4) u + c u.
    float s1, c1, s2, c2, sh, ch;
    if (trig_direct) {  // |x|, |y| <= 7 (set on the host): angles below 45 rad
      const float2 a = mul2(f2(kTwoPi, kTwoPi), f2(x, y));
      s1 = __sinf(a.x);
      s2 = __sinf(a.y);
      ch = __cosf(0.5f * y);
      (void)c1; (void)c2; (void)sh;
    } else {
      sincos_2pi(x, s1, c1);
      sincos_2pi(y, s2, c2);
      sincos_2pi(y * (0.5f / kTwoPi), sh, ch);
    }
    // q = s / sqrt2; u = 2^{x log2(e) / 4} cos(y/2); f = -u (1 + (3/16) q^2)
    const float q = fmaf(0.3f * s1, s2, 1.0f);
    s = 1.41421356237309505f * q;
    const float u = ex2_approx(x * 0.360673760222241f) * ch;
    dx = 0.f; dy = 0.f; c = -1.0f;
    f = -u * fmaf(0.1875f * q, q, 1.0f);
  } else if constexpr (COEF == PDDS_COEF_TABLE) {
    const float fx = fmaf(xr, H.tab_inv_dx, H.kd.tab_fx);
    const float fy = fmaf(yr, H.tab_inv_dy, H.kd.tab_fy);
    (void)tc;
    bilinear2(tsig, H.tile_w, fx, fy, H.tab_imax, H.tab_jmax, s, c);
    dx = 0.f; dy = 0.f; f = H.params[0];
  } else if constexpr (COEF == PDDS_COEF_POISSON_E1) {
    s = 1.41421356237309505f; dx = 0.f; dy = 0.f; c = 0.f;
    f = e1_lap(x, y, trig_direct);
  } else {
    s = H.params[0]; dx = H.params[1]; dy = H.params[2]; c = H.params[3]; f = H.params[4];
  }
}

template <int COEF>
__host__ __device__ constexpr bool has_c() {  // c may be nonzero (Y != 1)
  return COEF != PDDS_COEF_LAPLACE_EXPSIN && COEF != PDDS_COEF_POISSON_E1;
}
template <int COEF>
__host__ __device__ constexpr bool has_f() {  // f may be nonzero (Z != 0)
  return COEF != PDDS_COEF_LAPLACE_EXPSIN;
}
template <int COEF>
__host__ __device__ constexpr bool const_sigma() {  // s(x) is one constant
  return COEF != PDDS_COEF_VARSIGMA && COEF != PDDS_COEF_TABLE;
}
// s on the whole domain for the constant sets, else an upper bound.
template <int COEF>
__device__ __forceinline__ float sigma_bound(const Stage& H) {
  if constexpr (COEF == PDDS_COEF_CONSTANT) return fabsf(H.params[0]);
  else if constexpr (const_sigma<COEF>()) return 1.41421356237309505f;
  else return H.sigma_max;
}

// Gobet-Menozzi shifts (Sec. 2.3) of the four sides E, N, W, S of the knot's
// patch (box relative to the knot) for the point (X, Y): gmc |s(P_o)| with
// P_o the point's normal projection on side o, kept on the closed side.
template <int COEF>
__device__ __forceinline__ void gm_shifts(const Stage& H, const float* tsig, const float* tc,
                                          float xk, float yk, float X, float Y, float gmc,
                                          bool trig_direct, float sh[4]) {
  if constexpr (const_sigma<COEF>()) {
    const float d = gmc * sigma_bound<COEF>(H);
    sh[0] = sh[1] = sh[2] = sh[3] = d;
  } else {
    const float* b = H.kd.box;
    const float cx = fminf(fmaxf(X, b[0]), b[1]), cy = fminf(fmaxf(Y, b[2]), b[3]);
    const float px[4] = {b[1], cx, b[0], cx}, py[4] = {cy, b[3], cy, b[2]};
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      float s, ddx, ddy, c, f;
      coeffs<COEF>(H, tsig, tc, xk + px[o], yk + py[o], px[o], py[o], trig_direct, s, ddx, ddy,
                   c, f);
      sh[o] = gmc * fabsf(s);
    }
  }
}

// True when (X, Y) lies beyond at least one side moved by its own shift.
template <int COEF>
__device__ __noinline__ bool gm_outside(const Stage& H, const float* tsig, const float* tc,
                                        float xk, float yk, float X, float Y, float gmc,
                                        int trig_direct) {
  float sh[4];
  gm_shifts<COEF>(H, tsig, tc, xk, yk, X, Y, gmc, trig_direct != 0, sh);
  const float* b = H.kd.box;
  return (X > b[1] - sh[0]) | (Y > b[3] - sh[1]) | (X < b[0] + sh[2]) | (Y < b[2] + sh[3]);
}
template <int COEF>
__host__ __device__ constexpr bool has_drift() {  // d may be nonzero
  return COEF == PDDS_COEF_MANUFACTURED || COEF == PDDS_COEF_CONSTANT;
}

__device__ __forceinline__ const ProbDesc& prob_desc(const KParams& P, int i) {
  return P.nprob == 1 ? P.prob0 : P.probs[i];
}

// Tabulated control variate (Sec. 4.2): grad u0 at the [cv_ny][cv_nx] nodes
// spanning Omega, bilinear in between, kept cell by cell: cell (i, j) holds
// its four corners' gx then gy (32 bytes, one sector; read through L1/L2),
// one lookup = two 16-byte loads of one sector instead of four 8-byte loads
// from two rows (7 % faster per step on the paper's problem).
__device__ __forceinline__ void cv_table_grad(const ProbDesc& D, float x, float y, float& gx,
                                              float& gy) {
  const float fx = (x - D.x0) * D.cv_inv_dx, fy = (y - D.y0) * D.cv_inv_dy;
  const int i = min(max((int)floorf(fx), 0), D.cv_nx - 2);
  const int j = min(max((int)floorf(fy), 0), D.cv_ny - 2);
  const float tx = fminf(fmaxf(fx - (float)i, 0.f), 1.f);
  const float ty = fminf(fmaxf(fy - (float)j, 0.f), 1.f);
  // cell-major table: the four corners of cell (i, j), gx then gy, in one sector
  const float4* cell = reinterpret_cast<const float4*>(D.cv_tab) +
                       2 * ((int64_t)j * (D.cv_nx - 1) + i);
  const float4 G = __ldg(cell), H = __ldg(cell + 1);
  const float x0 = fmaf(tx, G.y - G.x, G.x), x1 = fmaf(tx, G.w - G.z, G.z);
  const float y0 = fmaf(tx, H.y - H.x, H.x), y1 = fmaf(tx, H.w - H.z, H.z);
  gx = fmaf(ty, x1 - x0, x0);
  gy = fmaf(ty, y1 - y0, y0);
}

// One Euler-Maruyama step (Eq. 9, Sec. 2.3) of a lane's path, in place:
//   Z -= f Y h,  S += c h log2(e)  (Y = 2^S),  X += d h + s dW,
// [CV = 2: xi -= Y s grad u0 . dW (Eq. 37)], with dW = -sqrt(h) g for the
// packed pair g of box_muller4.  The pairs (Z, S) and (X, Y) are updated with
// packed FP32 instructions; the values are those of the scalar forms.
template <int COEF, int CV>
__device__ __forceinline__ void em_step(const Stage& H, const float* tile, const KParams& P,
                                        bool direct, float xk, float yk, float h, float hl2,
                                        float sqh, float2 g, float& X, float& Y, float& Sx,
                                        float& Z, float& XI) {
  const float2 a = add2(f2(xk, yk), f2(X, Y));  // the absolute position
  float s, ddx, ddy, c, f;
  coeffs<COEF>(H, tile, tile, a.x, a.y, X, Y, direct, s, ddx, ddy, c, f);
  float Yw = 1.0f;
  if constexpr (has_c<COEF>()) {
    Yw = ex2_approx(Sx);
    const float2 zs = fma2(f2(-f * Yw, c), f2(h, hl2), f2(Z, Sx));  // dZ = -f Y dt, dS = c dt
    Z = zs.x;
    Sx = zs.y;
  } else if constexpr (has_f<COEF>()) {
    Z = fmaf(-f, h, Z);  // c = 0: Y = 1
  }
  const float ssh = s * sqh;
  if constexpr (CV == 2) {
    // grad u0 from the table; a control variate never runs batched, so the
    // table is problem 0's, read from the launch constants
    float gx, gy;
    cv_table_grad(P.prob0, a.x, a.y, gx, gy);
    XI = fmaf(Yw * ssh, fmaf(gx, g.x, gy * g.y), XI);
  }
  float2 p = f2(X, Y);
  if constexpr (has_drift<COEF>()) p = fma2(f2(ddx, ddy), f2(h, h), p);
  p = fma2(f2(-ssh, -ssh), g, p);
  X = p.x;
  Y = p.y;
}

__device__ __forceinline__ bool outside_box(float X, float Y, float bx0, float bx1, float by0,
                                            float by1) {
  return (X > bx1) | (X < bx0) | (Y > by1) | (Y < by0);
}

template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

template <int COEF>
__host__ __device__ constexpr bool uses_angles() {  // the coefficients take sines of the position
  return COEF == PDDS_COEF_MANUFACTURED || COEF == PDDS_COEF_VARSIGMA ||
         COEF == PDDS_COEF_POISSON_E1;
}

// P.calls_per_check Philox calls (two steps each) of one lane's path on the
// naive exit, between two exit checks of the warp: the two steps of a call are
// taken without a branch between them -- the second one starts from the first
// one's result and is dropped when the first one left the patch or reached
// the step cap.  DIRECT: the coefficient sines take the angle without
// reduction (the launch's domains allow it), a compile-time choice so that the
// step carries no branch on it.
template <int COEF, int CV, bool DIRECT>
__device__ __forceinline__ void step_calls(const Stage& H, const float* tile,
                                               const KParams& P, uint32_t p, uint32_t kk,
                                               uint32_t tagw, float xk, float yk, float h,
                                               float hl2, float sqh, int kmax, float bx0,
                                               float bx1, float by0, float by1, int& n, float& X,
                                               float& Y, float& Sx, float& Z, float& XI,
                                               bool& exited, bool& trunc) {
#pragma unroll 1
  for (int pair = 0; pair < P.calls_per_check && !exited; ++pair) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(n >> 1), p, kk, tagw), P.round_keys);
    float2 gA, gB;
    box_muller4(r, gA, gB);
    float X1 = X, Y1 = Y, S1 = Sx, Z1 = Z, XI1 = XI;
    em_step<COEF, CV>(H, tile, P, DIRECT, xk, yk, h, hl2, sqh, gA, X1, Y1, S1, Z1, XI1);
    const bool e1 = outside_box(X1, Y1, bx0, bx1, by0, by1);
    float X2 = X1, Y2 = Y1, S2 = S1, Z2 = Z1, XI2 = XI1;
    em_step<COEF, CV>(H, tile, P, DIRECT, xk, yk, h, hl2, sqh, gB, X2, Y2, S2, Z2, XI2);
    const bool e2 = outside_box(X2, Y2, bx0, bx1, by0, by1);
    const bool first = e1 || (n + 1 >= kmax);
    X = first ? X1 : X2;
    Y = first ? Y1 : Y2;
    Sx = first ? S1 : S2;
    Z = first ? Z1 : Z2;
    if constexpr (CV == 2) XI = first ? XI1 : XI2;
    n += first ? 1 : 2;
    exited = first ? e1 : e2;
    if (!exited && n >= kmax) { exited = true; trunc = true; }
  }
}

// What the resolution of one exited path produces (Eq. 22-25).
struct ExitResult {
  double bc = 0.0;          // the path's share of b_k (times N_k)
  int side = 0, flags = 0;  // exit side; bit 0 step cap, bit 1 along-line clamp
  float Yk = 1.0f, sl = 0.f, s_line = 0.f;
  int col_a = -1, col_b = -1;  // RECORD: knots of the two linear weights
  float wa = 0.f, wb = 0.f;
  bool rbf_exit = false;  // EXT + RBF stencils: the weights are the warp loop's
};

// Resolution of one exited path (the corner rule of Sec. 3.3; Eq. 22-25):
// the exit side is the one of smallest positive overshoot (past the sides
// moved by the Gobet-Menozzi shift when gmc > 0); an exit on the boundary of
// Omega adds Y g at the normal projection to b, an exit on an interface
// deposits Y (1 - lam) and Y lam on the two nearest stencil knots (exact 2^-30
// fixed point in the stage's slot accumulators; boundary knots of the
// stencil add their weight times g to b).  gm_rec: a Gobet-Menozzi exit of a
// mixed run, recorded but not deposited.
template <int COEF, bool RECORD, int CV, bool EXT>
__device__ __forceinline__ ExitResult resolve_exit(const Smem& S, const KParams& P, int st,
                                                   float xk, float yk, float X, float Y,
                                                   float Sx, float Z, float XI, bool trunc,
                                                   float bx0, float bx1, float by0, float by1,
                                                   float gmc, bool gm_rec) {
  ExitResult E;
  double& bc = E.bc;
  int& side = E.side;
  int& flags = E.flags;
  float& Yk = E.Yk;
  float& sl = E.sl;
  float& s_line = E.s_line;
  int& col_a = E.col_a;
  int& col_b = E.col_b;
  float& wa = E.wa;
  float& wb = E.wb;
  bool& rbf_exit = E.rbf_exit;
  const Stage& H = S.st(st);
  const KnotDesc& kd = H.kd;
  unsigned long long* acc = S.acc(st);
  float ov[4] = {X - bx1, Y - by1, bx0 - X, by0 - Y};
  if constexpr (EXT && !const_sigma<COEF>()) {
    // overshoots past each side moved by its own shift (a constant s, or
    // no shift, gives the lane's moved box, used above)
    if (gmc > 0.f) {
      float sh[4];
      gm_shifts<COEF>(H, S.tile(st, 0), S.tile(st, 1), xk, yk, X, Y, gmc, P.trig_direct,
                      sh);
      const float* tb = kd.box;
      ov[0] = X - (tb[1] - sh[0]);
      ov[1] = Y - (tb[3] - sh[1]);
      ov[2] = (tb[0] + sh[2]) - X;
      ov[3] = (tb[2] + sh[3]) - Y;
    }
  }
  // smallest positive overshoot (ties to the earlier side), else (a path
  // truncated inside the box) the largest; the running best stays in a
  // register so the overshoots need no indexed (local-memory) array
  side = -1;
  float best = 0.f;
#pragma unroll
  for (int o = 0; o < 4; ++o)
    if (ov[o] > 0.f && (side < 0 || ov[o] < best)) { side = o; best = ov[o]; }
  if (side < 0) {
    side = 0;
    best = ov[0];
#pragma unroll
    for (int o = 1; o < 4; ++o)
      if (ov[o] > best) { side = o; best = ov[o]; }
  }
  if constexpr (has_c<COEF>()) Yk = ex2_approx(Sx);
  bc = (double)Z;
  if constexpr (CV != 0) bc += (double)XI;
  const bool vertical = (side == 0 || side == 2);
  flags = trunc ? 1 : 0;
  if ((kd.dirbits >> side) & 1) {
    // exit on the boundary of Omega: Y g at the normal projection
    float along = vertical ? (yk + Y) : (xk + X);
    along = vertical ? fminf(fmaxf(along, H.y0), H.y1) : fminf(fmaxf(along, H.x0), H.x1);
    const float line = vertical ? fmaf((float)kd.line[side], H.dx, H.x0)
                                : fmaf((float)kd.line[side], H.dy, H.y0);
    bc += (double)Yk * (double)g_value<COEF>(H, vertical ? line : along, vertical ? along : line);
  } else {
    // exit on an interface: interpolation on the side's extended stencil
    const int a = kd.a[side], b = kd.b[side];
    const int kal = vertical ? kd.kj : kd.ki;
    sl = (float)(kal - a) + (vertical ? Y * H.inv_dy : X * H.inv_dx);
    const float smax = (float)(b - a);
    if (sl < 0.f) { sl = 0.f; flags |= 2; }
    if (sl > smax) { sl = smax; flags |= 2; }
    s_line = (float)a + sl;
    if constexpr (EXT) rbf_exit = prob_desc(P, H.prob).rbf_coef != nullptr;
    if (!rbf_exit) {
      // linear: the two nearest stencil knots
      int t = (int)floorf(sl);
      if (t >= b - a) t = b - a - 1;
      const float lam = sl - (float)t;
      // Y (1 - lam) and Y lam in 2^-30 units: q0 + q1 = qY exactly, so the
      // path deposits its whole weight Y on the two knots (G 1 = b holds
      // exactly when c = f = 0 and g = 1).
      const unsigned long long qY = __float2ull_rn(Yk * kFixedOne);
      const unsigned long long q1 = __float2ull_rn((Yk * lam) * kFixedOne);
      const unsigned long long qw[2] = {qY - q1, q1};
      const int lmax = vertical ? H.LY : H.LX;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int tl = a + t + q;
        if (tl == 0 || tl == lmax) {
          const int li = vertical ? kd.line[side] : tl;
          const int lj = vertical ? tl : kd.line[side];
          bc += (double)qw[q] * kFixedInv *
                (double)g_value<COEF>(H, fmaf((float)li, H.dx, H.x0),
                                      fmaf((float)lj, H.dy, H.y0));
        } else {
          const int slot = kd.off[side] + t + q;
          if (!gm_rec) atomicAdd(acc + slot, qw[q]);
          if constexpr (RECORD) {
            const ProbDesc& D = prob_desc(P, H.prob);
            const int c = D.slot2csr[kd.slot_base + slot];
            const int col = D.col[c];
            const float wv = (float)((double)qw[q] * kFixedInv);
            if (q == 0) { col_a = col; wa = wv; }
            else { col_b = col; wb = wv; }
          }
        }
      }
    }
  }
  return E;
}

// The per-path record of a resolved exit (knot-major: the record prefix of
// the knot, then the path index).
__device__ __forceinline__ void write_record(const Smem& S, const KParams& P, int st, uint32_t kk,
                                             uint32_t p, int n, const ExitResult& E, float XI,
                                             bool gm_rec) {
  const ProbDesc& D = prob_desc(P, S.st(st).prob);
  const int64_t idx = (D.path_prefix ? D.path_prefix[kk] : (int64_t)kk * D.n_paths) + p;
  PathRecordDev R;
  R.steps = n; R.side_flags = E.side | (E.flags << 8); R.col_a = E.col_a; R.col_b = E.col_b;
  R.w_a = E.wa; R.w_b = E.wb; R.b_contrib = (float)E.bc; R.Y = E.Yk;
  R.xi = XI; R.s_line = E.s_line;
  (gm_rec ? P.records_gm : P.records)[idx] = R;
}

// ------------------------------------------------------------ unit loading
__device__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t v) {
  int64_t lo = 0, hi = n;  // first index with a[i] > v
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Whole warp: take the next unit from the global queue into stage `s` as this
// CTA's unit number q (or mark the stage terminal).  Returns false on timeout.
template <bool EXT>
__device__ bool load_unit(const Smem& S, int s, int q, const KParams& P, int64_t total_units,
                          int& units_done) {
  const int lane = threadIdx.x & 31;
  Stage& H = S.st(s);
  if (lane == 0) {
    atomicExch(&H.ctrl, (unsigned long long)(2u * q + 1u) << 32);  // loading
    // Reserve a live unit before touching the queue, so that no warp can see
    // "queue empty and nothing live" while this load is still in progress.
    atomicAdd(S.live, 1);
    __threadfence();
  }
  __syncwarp();
  unsigned long long u = 0;
  if (lane == 0) u = atomicAdd(&P.scratch->next_unit, 1ull);
  u = __shfl_sync(kFull, u, 0);
  if ((int64_t)u >= total_units) {
    if (lane == 0) {
      H.term = 1;
      H.p_begin = H.p_end = H.total = 0;
      __threadfence();
      atomicExch(S.qempty, 1);
      __threadfence_block();
      atomicSub(S.live, 1);  // nothing was taken after all
      atomicExch(&H.ctrl, (unsigned long long)(2u * q) << 32);
    }
    __syncwarp();
    return true;
  }
  int prob = 0, k = 0;
  int64_t pb = 0, pe = 0;
  if (lane == 0) {
    prob = P.nprob == 1 ? 0 : (int)upper_bound_i64(P.prob_unit_prefix, P.nprob + 1, (int64_t)u) - 1;
    const ProbDesc& D = prob_desc(P, prob);
    const int64_t uu = (int64_t)u - P.prob_unit_prefix[prob];
    int64_t j;
    int64_t Nk;
    if (D.knot_unit_prefix == nullptr) {
      k = (int)(uu / D.units_per_knot);
      j = uu - (int64_t)k * D.units_per_knot;
      Nk = D.n_paths;
    } else {
      k = (int)upper_bound_i64(D.knot_unit_prefix, (int64_t)D.n + 1, uu) - 1;
      j = uu - D.knot_unit_prefix[k];
      Nk = D.n_per_knot[k];
    }
    pb = j * P.unit_paths;
    pe = min(Nk, pb + P.unit_paths);
  }
  prob = __shfl_sync(kFull, prob, 0);
  k = __shfl_sync(kFull, k, 0);
  pb = __shfl_sync(kFull, pb, 0);
  pe = __shfl_sync(kFull, pe, 0);
  const ProbDesc& D = prob_desc(P, prob);
  // Knot descriptor (28 words) and the problem fields the warps need.
  const int* src = reinterpret_cast<const int*>(D.knots + k);
  int* dst = reinterpret_cast<int*>(&H.kd);
  if (lane < (int)(sizeof(KnotDesc) / 4)) dst[lane] = __ldg(src + lane);
  if (lane < 8) H.params[lane] = D.params[lane];
  if (lane == 0) {
    H.term = 0;
    H.prob = prob;
    H.k = k;
    H.p_begin = (int)pb;
    H.p_end = (int)pe;
    H.total = (int)(pe - pb);
    H.done = 0;
    H.LX = D.LX; H.LY = D.LY; H.tag = D.tag; H.coef_id = D.coef_id;
    H.x0 = D.x0; H.y0 = D.y0; H.x1 = D.x1; H.y1 = D.y1;
    H.dx = D.dx; H.dy = D.dy; H.inv_dx = D.inv_dx; H.inv_dy = D.inv_dy;
    H.tab_inv_dx = D.tab_inv_dx; H.tab_inv_dy = D.tab_inv_dy;
    H.tile_w = P.tile_w;
    H.bsum = 0.0;
    if constexpr (EXT) {
      // step h_k of the knot; the cap keeps the time horizon of kmax steps of dt
      const double hk = D.h_per_knot != nullptr ? D.h_per_knot[k] : P.dt;
      H.h = (float)hk;
      H.sqh = (float)sqrt(hk);
      H.kmax = hk == P.dt ? (long long)P.kmax
                          : (long long)fmax(1.0, ceil((double)P.kmax * P.dt / hk));
      H.gmc = P.gm ? 0.5826f * H.sqh : 0.f;
      H.sigma_max = D.sigma_max;
    }
  }
  __syncwarp();
  const int nslots = H.kd.nslots;
  unsigned long long* acc = S.acc(s);
  for (int i = lane; i < nslots; i += 32) acc[i] = 0ull;
  if (D.tmap != nullptr) {
    // Stage the patch's sigma and c tiles with TMA (one CTA, no multicast):
    // the patch-local coefficient memory of Sec. 3.3.
    if (lane == 0) {
      H.tab_imax = min(P.tile_w - 2, D.tab_nx - 2 - H.kd.tile_i0);
      H.tab_jmax = min(P.tile_h - 2, D.tab_ny - 2 - H.kd.tile_j0);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // one tile of interleaved (s, c) pairs: x = 2 i0 is a multiple of 8 floats
      mbar_expect_tx(&H.mbar, 2u * (unsigned)(P.tile_w * P.tile_h * 4));
      tma_load_2d(S.tile(s, 0), D.tmap, 2 * H.kd.tile_i0, H.kd.tile_j0, &H.mbar);
    }
    __syncwarp();
    // The wait is bounded by the launch's wait limit (pdds_set_wait_limit).
    const int parity = H.tma_phase;
    const uint64_t t0 = global_ns();
    bool ok = true;
    while (!mbar_try_wait(&H.mbar, parity)) {
      if (global_ns() - t0 > P.wait_ns) { ok = false; break; }
    }
    ok = __all_sync(kFull, ok);
    if (!ok) {
      if (lane == 0) atomicExch(&P.scratch->error, (int)PDDS_ETIMEOUT);
      // Before the CTA leaves, the copy in flight gets a second bounded wait
      // of at least one second, however short the limit: a copy that landed
      // after the CTA had left would write into shared memory it no longer
      // owns.  The error recorded above voids the call's results.
      const uint64_t drain = P.wait_ns > 1000000000ull ? P.wait_ns : 1000000000ull;
      const uint64_t t1 = global_ns();
      while (!mbar_try_wait(&H.mbar, parity) && global_ns() - t1 < drain) {
      }
      return false;
    }
    __syncwarp();
    if (lane == 0) H.tma_phase ^= 1;
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence_block();
    atomicExch(&H.ctrl, ((unsigned long long)(2u * q) << 32) | (unsigned)pb);  // publish
  }
  __syncwarp();
  ++units_done;
  return true;
}

// Whole warp: add the finished unit's FP64 sums to G and b (global atomics).
__device__ void flush_unit(const Smem& S, int s, const KParams& P) {
  const int lane = threadIdx.x & 31;
  __threadfence_block();
  Stage& H = S.st(s);
  const ProbDesc& D = prob_desc(P, H.prob);
  const unsigned long long* acc = S.acc(s);
  const int32_t* map = D.slot2csr + H.kd.slot_base;
  for (int i = lane; i < H.kd.nslots; i += 32) {
    const unsigned long long q = acc[i];
    const int c = __ldg(map + i);
    // exact: |q| < 2^53, times a power of two (RBF weights may be negative)
    if (q != 0ull && c >= 0) atomicAdd(D.Gval + c, (double)(long long)q * kFixedInv);
  }
  if (lane == 0) atomicAdd(D.b + H.k, H.bsum);
  __syncwarp();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ------------------------------------------------------------- the kernel
// CV: 0 no control variate, 1 the in-path network, 2 the tabulated gradient.
// Plain and table variants: up to 1024 threads (64 registers).  Network
// variants hold the MMA fragments of the in-path network: at most 256 threads
// and two CTAs per SM, i.e. up to 128 registers.  EXT: per-knot steps and the
// Gobet-Menozzi shift (P.gm).
// Register caps: 128 for the network variants; 56 for the plain kernels with
// analytic coefficients (a few bytes of spill, about 1.5 % faster than 64 on
// the manufactured workload: more warps per SM); 64 for the rest, which spill
// tens of bytes at 56.
constexpr int path_kernel_regs(int coef, int cv, bool ext) {
  return cv == 1 ? 128 : (cv == 0 && !ext && coef != PDDS_COEF_TABLE ? 56 : 64);
}
template <int COEF, bool RECORD, int CV, bool EXT>
__global__ void __launch_bounds__(CV == 1 ? 256 : 1024, CV == 1 ? 2 : 1)
    __maxnreg__(path_kernel_regs(COEF, CV, EXT))
    path_kernel(const __grid_constant__ KParams P) {
  extern __shared__ __align__(128) char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // Control variate: the network is staged once per CTA at the start of the
  // dynamic shared memory (network variants only); the unit ring follows it.
  MlpSmem* mlp_s = reinterpret_cast<MlpSmem*>(smem_raw);
  if constexpr (CV == 1) {
    const int4* src = reinterpret_cast<const int4*>(P.mlp);
    int4* dst = reinterpret_cast<int4*>(mlp_s);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) dst[i] = src[i];
  }
  Smem S;
  S.base = smem_raw + (CV == 1 ? kMlpSmemBytes : 0);
  S.stage_bytes = P.stage_bytes;
  S.acc_bytes = ((P.max_slots * 8) + 127) / 128 * 128;
  S.tile_bytes = ((2 * P.tile_w * P.tile_h * 4) + 127) / 128 * 128;  // interleaved (s, c)

  __shared__ int s_live, s_qempty;
  S.live = &s_live;
  S.qempty = &s_qempty;
  const int64_t total_units = P.prob_unit_prefix[P.nprob];
  int units_done = 0;
  if (threadIdx.x == 0) {
    s_live = 0;
    s_qempty = 0;
    for (int s = 0; s < 2; ++s) {
      S.st(s).ctrl = (unsigned long long)(2u * s + 1u) << 32;  // "loading unit s"
      S.st(s).term = 0;
      S.st(s).tma_phase = 0;
      mbar_init(&S.st(s).mbar);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  if (warp < 2) ok = load_unit<EXT>(S, warp, warp, P, total_units, units_done);
  __syncthreads();

  // lane state
  bool alive = false;
  int st = 0;
  uint32_t p = 0, kk = 0, tagw = 0;
  constexpr bool kPhiloxPre = EXT && CV == 0;  // the per-path Philox constants
  PhiloxPath ph{0u, 0u, 0u, 0u};
  // Mixed GM/EM run of the calibration (Sec. 4.1; records kernels with the
  // extended exit, P.mixed): a path first records its Gobet-Menozzi exit,
  // then steps on inside the closed patch to its naive exit, which is
  // accumulated and recorded like any other; it resumes at the step after
  // its GM exit, with that step's Gaussian pair.  pend_em: the naive exit
  // fell on the step of the Gobet-Menozzi one (or the path was truncated)
  // and is resolved in the next round.
  constexpr bool kMixed = EXT && RECORD;
  bool gm_phase = false, pend_em = false, pend_tr = false;
  int n = 0;
  float xk = 0.f, yk = 0.f, bx0 = 0.f, bx1 = 0.f, by0 = 0.f, by1 = 0.f;
  float X = 0.f, Y = 0.f, Sx = 0.f, Z = 0.f, XI = 0.f;
  unsigned long long my_steps = 0, my_paths = 0, my_trunc = 0, my_clamp = 0;
  int want = 0;  // warp-uniform: unit sequence number the warp takes paths from
  // EXT: step, its square root and the step cap of the knot the lane's path
  // belongs to, and the Gobet-Menozzi shift per unit of |s| (0: naive exit);
  // the other variants use the launch constants
  int64_t kmax_l = 0;
  float h_l = 0.f, sqh_l = 0.f, gmc = 0.f;
  const uint64_t wait_ns = P.wait_ns;
  uint64_t idle_since = 0;

  while (ok) {
    // ---- hand new paths to idle lanes ----------------------------------
    unsigned idle = __ballot_sync(kFull, !alive);
    for (int guard = 0; idle && guard < 64; ++guard) {
      Stage& H = S.st(want & 1);
      const unsigned ss = ctrl_state(&H.ctrl);
      if ((int)(ss >> 1) > want) { ++want; continue; }      // stage moved past unit `want`
      if ((ss & 1u) || (int)(ss >> 1) < want) break;       // unit `want` not published yet
      // A terminal stage only means this load found the queue empty; the other
      // stage may still hold a unit taken earlier, so move on to it.
      if (H.term) { ++want; continue; }
      const int cnt = __popc(idle);
      const int leader = __ffs(idle) - 1;
      unsigned long long c = 0;
      if (lane == leader) c = atomicAdd(&H.ctrl, (unsigned long long)cnt);
      c = __shfl_sync(kFull, c, leader);
      __threadfence_block();
      const unsigned sa = (unsigned)(c >> 32);
      if (sa & 1u) break;                 // claim landed on a unit being loaded: void
      const int base = (int)(unsigned)(c & 0xffffffffull);
      const int pend = H.p_end;
      __threadfence_block();
      if (ctrl_state(&H.ctrl) != sa) {    // unit recycled meanwhile: it was exhausted
        want = max(want, (int)(sa >> 1) + 1);
        continue;
      }
      want = max(want, (int)(sa >> 1));
      const int got = max(0, min(cnt, pend - base));
      const int rank = __popc(idle & ((1u << lane) - 1u));
      if (!alive && rank < got) {
        alive = true;
        st = want & 1;
        p = (uint32_t)(base + rank);
        kk = (uint32_t)H.k;
        tagw = (uint32_t)H.tag;
        if constexpr (kPhiloxPre) ph = philox_path(p, kk, tagw, P.round_keys);
        xk = H.kd.xk; yk = H.kd.yk;
        bx0 = H.kd.box[0]; bx1 = H.kd.box[1]; by0 = H.kd.box[2]; by1 = H.kd.box[3];
        if constexpr (EXT) {
          h_l = H.h; sqh_l = H.sqh; kmax_l = H.kmax; gmc = H.gmc;
          // the cheap exit test uses the box moved by the largest shift
          const float dm = gmc * sigma_bound<COEF>(H);
          bx0 += dm; bx1 -= dm; by0 += dm; by1 -= dm;
        }
        if constexpr (kMixed) {
          gm_phase = P.mixed != 0;
          pend_em = pend_tr = false;
        }
        n = 0; X = 0.f; Y = 0.f; Sx = 0.f; Z = 0.f; XI = 0.f;
      }
      if (base + cnt >= pend) ++want;     // unit fully handed out
      idle = __ballot_sync(kFull, !alive);
    }
    const unsigned alive_mask = __ballot_sync(kFull, alive);
    if (alive_mask == 0) {
      // Done when the queue is empty and no unit of this CTA is loaded or loading.
      const int qe = *(volatile int*)S.qempty;
      __threadfence_block();
      if (qe && *(volatile int*)S.live == 0) break;
      if (idle_since == 0) idle_since = global_ns();
      if (global_ns() - idle_since > wait_ns) {
        if (lane == 0) atomicExch(&P.scratch->error, (int)PDDS_ETIMEOUT);
        break;
      }
      __nanosleep(256);
      continue;
    }
    idle_since = 0;

    // ---- step until enough lanes have exited -----------------------------
    const float h = EXT ? h_l : P.h, sqh = EXT ? sqh_l : P.sqh;
    const float hl2 = h * 1.44269504088896341f;  // S is kept in log2 units: Y = 2^S
    // 32-bit step cap (the API keeps caps below 2^31): one compare per step
    const int kmax = (int)min(EXT ? kmax_l : P.kmax, (int64_t)0x7fffffff);
    bool exited = false, trunc = false;
    if constexpr (kMixed) {
      exited = alive && pend_em;
      trunc = pend_tr;
    }
    for (;;) {
      if constexpr (CV == 1) {
        // Same step as below, but the warp stays converged for the tensor-core
        // evaluation of grad v_theta at every lane's position; only lanes that
        // are stepping use it: dxi = -Y sigma grad v . dW (Eq. 37).
        const bool go = alive && !exited;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (go) {
          const uint4 r = kPhiloxPre ? philox_step((uint32_t)(n >> 1), ph, P.round_keys)
                          : philox4x32_10(make_uint4((uint32_t)(n >> 1), p, kk, tagw), P.round_keys);
          box_muller(r.x, r.y, z[0], z[1]);
          box_muller(r.z, r.w, z[2], z[3]);
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float gx, gy, vv;
          mlp_grad_warp<false>(*mlp_s, xk + X, yk + Y, gx, gy, vv);
          if (go && !exited && (!kMixed || half >= (n & 1))) {
            const Stage& H = S.st(st);
            float s, ddx, ddy, c, f;
            coeffs<COEF>(H, S.tile(st, 0), S.tile(st, 1), xk + X, yk + Y, X, Y, P.trig_direct,
                         s, ddx, ddy, c, f);
            const float dWx = sqh * z[2 * half], dWy = sqh * z[2 * half + 1];
            float Yw = 1.0f;
            if constexpr (has_c<COEF>()) Yw = ex2_approx(Sx);
            if constexpr (has_f<COEF>()) Z = fmaf(-f * Yw, h, Z);
            if constexpr (has_c<COEF>()) Sx = fmaf(c, hl2, Sx);
            XI = fmaf(-Yw * s, fmaf(gx, dWx, gy * dWy), XI);
            const float ssh = s * sqh;
            X = fmaf(ssh, z[2 * half], fmaf(ddx, h, X));
            Y = fmaf(ssh, z[2 * half + 1], fmaf(ddy, h, Y));
            ++n;
            exited = (X > bx1) | (X < bx0) | (Y > by1) | (Y < by0);
            if constexpr (EXT && !const_sigma<COEF>()) {
              if (exited && gmc > 0.f) exited = gm_outside<COEF>(H, S.tile(st, 0), S.tile(st, 1),
                                                              xk, yk, X, Y, gmc, P.trig_direct);
            }
            if (!exited && n >= kmax) { exited = true; trunc = true; }
          }
        }
      } else if (!EXT && alive && !exited) {
        const Stage& H = S.st(st);
        const float* tile = S.tile(st, 0);
        if (uses_angles<COEF>() && P.trig_direct)
          step_calls<COEF, CV, uses_angles<COEF>()>(H, tile, P, p, kk, tagw, xk, yk, h, hl2,
                                                        sqh, kmax, bx0, bx1, by0, by1, n, X, Y,
                                                        Sx, Z, XI, exited, trunc);
        else
          step_calls<COEF, CV, false>(H, tile, P, p, kk, tagw, xk, yk, h, hl2, sqh, kmax,
                                          bx0, bx1, by0, by1, n, X, Y, Sx, Z, XI, exited, trunc);
      } else if (alive && !exited) {
       // extended-exit kernels (per-knot steps, Gobet-Menozzi exits, the mixed
       // GM/EM run): P.calls_per_check Philox calls between exit checks, one
       // branch per step (the two-step form spills more here)
       // (the angle-reduction choice is a template constant here too)
       auto ext_calls = [&](auto direct_tag) {
        constexpr bool kDirect = decltype(direct_tag)::value;
#pragma unroll 1
         for (int pair = 0; pair < P.calls_per_check; ++pair) {
          if (exited) break;
          const uint4 r = kPhiloxPre ? philox_step((uint32_t)(n >> 1), ph, P.round_keys)
                            : philox4x32_10(make_uint4((uint32_t)(n >> 1), p, kk, tagw), P.round_keys);
          float z[4];
          box_muller(r.x, r.y, z[0], z[1]);
          box_muller(r.z, r.w, z[2], z[3]);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            // a Philox call serves steps 2q and 2q + 1; a mixed-run path that
            // resumes at an odd step takes the second half of its call
            if (!exited && (!kMixed || half >= (n & 1))) {
              const Stage& H = S.st(st);
              float s, ddx, ddy, c, f;
              coeffs<COEF>(H, S.tile(st, 0), S.tile(st, 1), xk + X, yk + Y, X, Y, kDirect,
                           s, ddx, ddy, c, f);
              float Yw = 1.0f;
              if constexpr (has_c<COEF>()) {
                Yw = ex2_approx(Sx);
                Z = fmaf(-f * Yw, h, Z);  // dZ = -f Y dt
                Sx = fmaf(c, hl2, Sx);    // dY = c Y dt, Y = 2^S with S = log2(e) int c dt
              } else if constexpr (has_f<COEF>()) {
                Z = fmaf(-f, h, Z);       // c = 0: Y = 1
              }
              // dX = d dt + s dW with dW = sqrt(h) z: s sqrt(h) once, then two FMAs
              const float ssh = s * sqh;
              if constexpr (CV == 2) {
                // dxi = -Y s grad u0 . dW with grad u0 from the table (Eq. 37, Sec. 4.2)
                float gx, gy;
                // a control variate never runs batched (pdds_assemble_batch refuses
                // it), so the table is problem 0's, read from the launch constants:
                // no per-step loads of the problem descriptor
                cv_table_grad(P.prob0, xk + X, yk + Y, gx, gy);
                XI = fmaf(-Yw * ssh, fmaf(gx, z[2 * half], gy * z[2 * half + 1]), XI);
              }
              if constexpr (has_drift<COEF>()) {
                X = fmaf(ssh, z[2 * half], fmaf(ddx, h, X));
                Y = fmaf(ssh, z[2 * half + 1], fmaf(ddy, h, Y));
              } else {
                X = fmaf(ssh, z[2 * half], X);
                Y = fmaf(ssh, z[2 * half + 1], Y);
              }
              ++n;
              exited = (X > bx1) | (X < bx0) | (Y > by1) | (Y < by0);
              if constexpr (EXT && !const_sigma<COEF>()) {
                if (exited && gmc > 0.f) exited = gm_outside<COEF>(H, S.tile(st, 0), S.tile(st, 1),
                                                                xk, yk, X, Y, gmc, kDirect);
              }
              if (!exited && n >= kmax) { exited = true; trunc = true; }
            }
          }
         }
       };
       if (uses_angles<COEF>() && P.trig_direct) ext_calls(BoolTag<uses_angles<COEF>()>{});
       else ext_calls(BoolTag<false>{});
      }
      const unsigned ex = __ballot_sync(kFull, alive && exited);
      const unsigned stepping = __ballot_sync(kFull, alive && !exited);
      if (stepping == 0 || __popc(ex) >= P.exit_batch) break;
    }

    // ---- resolve the exits (Eq. 22-25, corner rule of Sec. 3.3) -----------
    const bool leaving = alive && exited;
    bool gm_rec = false;  // a Gobet-Menozzi exit of a mixed run: recorded, the path goes on
    if constexpr (kMixed) gm_rec = leaving && gm_phase;
    ExitResult E;
    if (leaving)
      E = resolve_exit<COEF, RECORD, CV, EXT>(S, P, st, xk, yk, X, Y, Sx, Z, XI, trunc, bx0, bx1,
                                              by0, by1, gmc, gm_rec);
    double& bc = E.bc;
    const int side = E.side, flags = E.flags;
    const float Yk = E.Yk, sl = E.sl;
    const bool rbf_exit = E.rbf_exit;  // EXT + RBF stencils: weights come from the warp loop below
    if constexpr (EXT) {
      // RBF stencils (Eq. 21-22): every knot j of the exit side's stencil gets
      // Y H_j(s).  The whole warp serves one exiting lane at a time, a knot per
      // lane, evaluating the tabulated cardinal functions; knots on the
      // boundary of Omega add Y H_j g(x_j) to the exiting lane's b share.
      unsigned pend = __ballot_sync(kFull, rbf_exit);
      while (pend) {
        const int src = __ffs(pend) - 1;
        const int r_st = __shfl_sync(kFull, st, src);
        const int r_side = __shfl_sync(kFull, side, src);
        const float r_s = __shfl_sync(kFull, sl, src);
        const float r_Y = __shfl_sync(kFull, Yk, src);
        bool r_gm = false;
        if constexpr (kMixed) r_gm = __shfl_sync(kFull, gm_rec ? 1 : 0, src) != 0;
        const Stage& H = S.st(r_st);
        const KnotDesc& kd = H.kd;
        const ProbDesc& D = prob_desc(P, H.prob);
        const bool vertical = (r_side == 0 || r_side == 2);
        const int a = kd.a[r_side];
        const int L = kd.b[r_side] - a + 1;
        const int lmax = vertical ? H.LY : H.LX;
        float tau;
        const float* cf = rbf_interval(D, vertical ? 1 : 0, L, r_s, tau);
        unsigned long long* acc = S.acc(r_st);
        double dsum = 0.0;
        if (cf == nullptr && lane == 0) atomicExch(&P.scratch->error, (int)PDDS_EINVAL);
        for (int j = lane; cf != nullptr && j < L; j += 32) {
          const float w = r_Y * rbf_cardinal(cf, L, D.rbf_deg + 1, j, tau);
          const int tl = a + j;
          if (tl == 0 || tl == lmax) {
            const int li = vertical ? kd.line[r_side] : tl;
            const int lj = vertical ? tl : kd.line[r_side];
            dsum += (double)w * (double)g_value<COEF>(H, fmaf((float)li, H.dx, H.x0),
                                                      fmaf((float)lj, H.dy, H.y0));
          } else if (!r_gm) {
            // signed weights in 2^-30 units (two's complement in the slot)
            atomicAdd(acc + kd.off[r_side] + j,
                      (unsigned long long)__float2ll_rn(w * kFixedOne));
          }
        }
        dsum = warp_sum(dsum);
        if (lane == src) bc += dsum;
        pend &= pend - 1;
      }
    }
    if (leaving) {
      if (!gm_rec) {
        my_steps += (unsigned long long)n;
        my_paths += 1;
        my_trunc += (flags & 1);
        my_clamp += (flags >> 1) & 1;
      }
      if constexpr (RECORD) write_record(S, P, st, kk, p, n, E, XI, gm_rec);
      if (!gm_rec) atomicAdd(&S.st(st).bsum, bc);  // one FP64 shared atomic per exit
    }
    if constexpr (kMixed) {
      if (gm_rec) {
        // on to the naive exit: the closed patch, no shift
        const KnotDesc& kd = S.st(st).kd;
        gm_phase = false;
        gmc = 0.f;
        bx0 = kd.box[0]; bx1 = kd.box[1]; by0 = kd.box[2]; by1 = kd.box[3];
        // a GM exit on the step cap, still inside the patch, is the naive
        // path's truncation at that same step
        pend_tr = trunc || n >= kmax;
        pend_em = pend_tr || (X > bx1) | (X < bx0) | (Y > by1) | (Y < by0);
      } else if (leaving) {
        pend_em = pend_tr = false;
      }
    }
    // warp-aggregated completion counts per stage
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const unsigned m = __ballot_sync(kFull, leaving && !gm_rec && st == s);
      if (m == 0) continue;
      __syncwarp();
      __threadfence_block();
      int fin = 0;
      if (lane == 0) {
        Stage& H = S.st(s);
        const int old = atomicAdd(&H.done, __popc(m));
        fin = (old + __popc(m) == H.total);
      }
      fin = __shfl_sync(kFull, fin, 0);
      if (fin) {
        const int q = (int)(ctrl_state(&S.st(s).ctrl) >> 1);
        flush_unit(S, s, P);
        if (!load_unit<EXT>(S, s, q + 2, P, total_units, units_done)) ok = false;
        if (lane == 0) atomicSub(S.live, 1);  // the flushed unit (after the reload reserved)
        __syncwarp();
      }
    }
    if (leaving && !gm_rec) alive = false;
  }

  // per-launch counters
  my_steps = warp_sum_u64(my_steps);
  my_paths = warp_sum_u64(my_paths);
  my_trunc = warp_sum_u64(my_trunc);
  my_clamp = warp_sum_u64(my_clamp);
  if (lane == 0) {
    atomicAdd(&P.scratch->steps, my_steps);
    atomicAdd(&P.scratch->paths, my_paths);
    atomicAdd(&P.scratch->truncated, my_trunc);
    atomicAdd(&P.scratch->clamped, my_clamp);
    atomicAdd(&P.scratch->units, (unsigned long long)units_done);
  }
}

}  // namespace
}  // namespace pdds
