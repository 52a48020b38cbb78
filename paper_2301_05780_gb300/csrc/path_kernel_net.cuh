// The path kernel with the in-path network control variate (Eq. 37; v_theta
// of Eq. 11, 38-39) on the fifth-generation tensor cores: the paths of a
// warpgroup (four warps, 128 lanes) step together, and at every step the
// gradient of v_theta at their 128 positions is one M = 128 tile:
//
//   layer 1 (FP32 SIMT)   a1 = W1 x + b1, h1 = SiLU(a1) -> BF16 A tile in shared
//                         memory (row = the thread's path), SiLU'(a1) -> TMEM
//   forward (tcgen05)     D = h1 W2^T   (M = 128, N = 64, K = 64; BF16, FP32 in TMEM)
//   output (FP32 SIMT)    g2 = w3 * SiLU'(D + b2) = dv/da2 -> the A tile (BF16)
//   backward (tcgen05)    D = g2 W2     (same TMEM columns)
//   input gradient        grad v = W1^T (D * SiLU'(a1))
//
// Thread t of a warpgroup owns TMEM lane t and row t of the tile.  One
// elected thread issues the MMAs (kind::f16, BF16 operands as in the
// warp-level routine of pdds_mlp.cuh) and commits them to the group's
// mbarrier; every wait on it is bounded.  The group's four warps meet at a
// named barrier before each product, and agree on leaving the step loop with
// a barrier reduction, so no warp ever waits at a barrier the others do not
// reach: every decision that ends a loop is taken for the whole group.
//
// Everything else -- the unit ring, the claim of paths, the Philox stream
// and Box-Muller (one call per two steps), the EM update, the exit test and
// its resolution -- is the warp-level code of path_kernel.cuh, unchanged, so
// the estimator is the CV = 1 kernel's: only the rounding of the network's
// products differs.
#pragma once
#include "path_kernel.cuh"
#include "tc_sm103.cuh"

namespace pdds {
namespace {

constexpr int kNetRows = 128;  // paths per warpgroup = MMA M
constexpr int kNetH = kMlpHidden;

// The network as the tensor cores read it (per CTA), and the warpgroup's A
// tile.  BF16 tiles are K-major with the 128-byte swizzle: one 128-byte
// row per point (64 BF16), 8-row groups 1024 bytes apart, the 16-byte chunk c
// of row r at chunk position c ^ (r % 8).
struct alignas(1024) NetSmem {
  uint16_t B1[kNetH * kNetH];  // W2 as N = out x K = in
  uint16_t B2[kNetH * kNetH];  // W2^T as N = in x K = out
  uint16_t A[kNetRows * kNetH];
  unsigned long long mbar;
  unsigned tmem, tmem_s1;  // TMEM: the products (64 columns), 2 SiLU'(a1) as BF16 pairs (32)
};
// + alignment slack: the dynamic shared memory is aligned by hand
constexpr int kNetSmemBytes = (int)((sizeof(NetSmem) + 1024 + 127) / 128 * 128);

// The network's FP32 vectors, halved (W1[:, 0]/2, W1[:, 1]/2, b1/2, b2/2,
// w3/2; the SiLU algebra below works with a/2), as a kernel parameter: every
// thread reads the same value at the same time, so they are served from the
// constant bank instead of shared memory.
struct NetWeights {
  float w1x[kNetH], w1y[kNetH], b1[kNetH], b2[kNetH], w3[kNetH];
};

__device__ __forceinline__ int net_chunk(int r, int c) {
  return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
}
__device__ __forceinline__ int net_elem(int r, int k) { return net_chunk(r, k >> 3) + ((k & 7) << 1); }

// Named barriers 1 and 2 (0 is __syncthreads), immediate IDs: a barrier ID in
// a register makes the compiler reserve all sixteen of the CTA's barriers.
__device__ __forceinline__ void group_bar(int g) {
  if (g == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
  else asm volatile("bar.sync 2, 128;" ::: "memory");
}
// The group's OR / AND of a predicate (a barrier with reduction: every thread
// of the group gets the same value).
template <int ID>
__device__ __forceinline__ bool bar_red_or(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(ID)
      : "memory");
  return r != 0;
}
template <int ID>
__device__ __forceinline__ bool bar_red_and(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " bar.red.and.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(ID)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool group_any(int g, bool v) {
  return g == 0 ? bar_red_or<1>(v) : bar_red_or<2>(v);
}
__device__ __forceinline__ bool group_all(int g, bool v) {
  return g == 0 ? bar_red_and<1>(v) : bar_red_and<2>(v);
}

// D (TMEM columns [d, d + 64)) = A B^T: four K-steps of 16 BF16 (32 bytes
// inside the 128-byte swizzle atom).
__device__ __forceinline__ void net_mma(unsigned d, const uint16_t* A, const uint16_t* B) {
  constexpr uint32_t idesc = tc::idesc_bf16(kNetRows, kNetH);
  const unsigned a = tc::smem_addr(A), b = tc::smem_addr(B);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    tc::mma_bf16(d, tc::sdesc_k128(a + kk * 32), tc::sdesc_k128(b + kk * 32), idesc, kk > 0);
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) { return pack_bf16x2(lo, hi); }

// Bounded wait for phase `parity` of an MMA mbarrier: one try before the
// clock is read (a product is usually done by then).
__device__ __forceinline__ bool net_wait(unsigned long long* bar, unsigned parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, (int)parity)) return true;
  return tc::mbar_wait(bar, parity, limit_ns);
}

// SiLU through t = tanh(a/2), for a pair of units on the packed FP32 pipe:
// with a' = a/2 (the network's weights and biases halved, an exact scaling),
//   SiLU(a) = a (1 + t)/2 = a' (1 + t),
//   SiLU'(a) = (1 + t)/2 + a (1 - t^2)/4 = (1 + t + a' (1 - t^2)) / 2.
__device__ __forceinline__ float2 tanh2(float2 a) { return f2(tanh_approx(a.x), tanh_approx(a.y)); }
__device__ __forceinline__ float2 one_minus_sq(float2 t) {
  return fma2(t, f2(-t.x, -t.y), f2(1.0f, 1.0f));
}
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// grad v_theta at the thread's point (x, y), in two parts so that the caller
// can work while the forward product runs: net_grad_start (layer 1, then one
// thread issues the forward product) and net_grad_finish.  Whole warpgroup
// (all 128 threads of the CTA, converged per warp; g names its barrier).  tm:
// the 64 TMEM columns of the products, ts: the 32 columns of 2 SiLU'(a1) as
// BF16 pairs, tl: the warp's TMEM lane offset.  phase: the mbarrier parity,
// flipped twice by net_grad_finish, whose wait_ns bounds each wait for a
// product.  The SIMT parts work on unit pairs (f32x2).
__device__ __forceinline__ void net_grad_start(NetSmem& N, const NetWeights& W, int g, int t,
                                               unsigned tm, unsigned ts, unsigned tl, float x,
                                               float y) {
  uint16_t* const A = N.A;
  char* const Ab = reinterpret_cast<char*>(A);
  __syncwarp();  // the tcgen05 loads and stores below are warp-aligned
  // layer 1: h1 into row t of the A tile, SiLU'(a1) into TMEM
  const float2 xx = f2(x, x), yy = f2(y, y);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float d[16];
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      uint32_t hp[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = 16 * q + 8 * c2 + 2 * j;
        const float2 a = fma2(ld2(&W.w1x[u]), xx, fma2(ld2(&W.w1y[u]), yy, ld2(&W.b1[u])));  // a1/2
        const float2 th = tanh2(a);
        const float2 h = fma2(a, th, a);                                               // SiLU(a1)
        const float2 s = add2(fma2(a, one_minus_sq(th), th), f2(1.0f, 1.0f));          // 2 SiLU'(a1)
        hp[j] = bf16x2(h.x, h.y);
        d[8 * c2 + 2 * j] = s.x;
        d[8 * c2 + 2 * j + 1] = s.y;
      }
      *reinterpret_cast<uint4*>(Ab + net_chunk(t, 2 * q + c2)) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
    }
    uint32_t dp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) dp[j] = bf16x2(d[2 * j], d[2 * j + 1]);
    tc::tmem_st8u(ts + tl + 8 * q, dp);
  }
  tc::st_wait();
  tc::fence_async_smem();
  tc::fence_before();
  group_bar(g);
  if (t == 0) {
    tc::fence_after();
    net_mma(tm, A, N.B1);
    tc::commit(&N.mbar);
  }
}

// Second part of the evaluation (whole warpgroup): wait for the forward
// product, then layer 2, the backward product and the input gradient.
// Returns false if a wait ran out (results void).
__device__ __forceinline__ bool net_grad_finish(NetSmem& N, const NetWeights& W, int g, int t,
                                                unsigned tm, unsigned ts, unsigned tl,
                                                unsigned& phase,
                                                uint64_t wait_ns, float& gx, float& gy) {
  uint16_t* const A = N.A;
  char* const Ab = reinterpret_cast<char*>(A);
  bool ok = net_wait(&N.mbar, phase, wait_ns);
  phase ^= 1u;
  tc::fence_after();
  // dv/da2 = w3 SiLU'(a2) into the A tile (the forward product has read it)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a2[16];
    tc::tmem_ld16(tm + tl + 16 * q, a2);
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      uint32_t ep[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = 16 * q + 8 * c2 + 2 * j;
        // a2/2: the forward product runs on W2/2
        const float2 a = add2(f2(a2[8 * c2 + 2 * j], a2[8 * c2 + 2 * j + 1]), ld2(&W.b2[o]));
        const float2 th = tanh2(a);
        const float2 w = ld2(&W.w3[o]);  // w3/2
        const float2 e = fma2(w, fma2(a, one_minus_sq(th), th), w);  // w3 SiLU'(a2)
        ep[j] = bf16x2(e.x, e.y);
      }
      *reinterpret_cast<uint4*>(Ab + net_chunk(t, 2 * q + c2)) = make_uint4(ep[0], ep[1], ep[2], ep[3]);
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  group_bar(g);
  if (t == 0) {
    tc::fence_after();
    net_mma(tm, A, N.B2);
    tc::commit(&N.mbar);
  }
  ok = net_wait(&N.mbar, phase, wait_ns) && ok;
  phase ^= 1u;
  tc::fence_after();
  // grad v = W1^T (dv/dh1 * SiLU'(a1)) = (W1/2)^T (dv/dh1 * 2 SiLU'(a1)), even
  // and odd units summed apart
  float2 sx = f2(0.f, 0.f), sy = f2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float dh[16], s1[16];
    uint32_t sp[8];
    tc::tmem_ld16(tm + tl + 16 * q, dh);
    tc::tmem_ld8u(ts + tl + 8 * q, sp);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      s1[2 * j] = __uint_as_float(sp[j] << 16);
      s1[2 * j + 1] = __uint_as_float(sp[j] & 0xffff0000u);
    }
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
      const int u = 16 * q + j;
      const float2 r = mul2(f2(dh[j], dh[j + 1]), f2(s1[j], s1[j + 1]));
      sx = fma2(ld2(&W.w1x[u]), r, sx);
      sy = fma2(ld2(&W.w1y[u]), r, sy);
    }
  }
  gx = sx.x + sx.y;
  gy = sy.x + sy.y;
  return ok;
}

// One warpgroup (128 threads) per CTA; TMEM: 64 columns for the products and
// 32 for 2 SiLU'(a1) as BF16 pairs (the rounding the warp-level routine gives
// it too), so five CTAs per SM fit in TMEM, registers (96) and shared memory.
template <int COEF, bool RECORD, bool EXT>
__global__ void __launch_bounds__(kNetRows, 5)
    path_kernel_net(const __grid_constant__ KParams P, const __grid_constant__ NetWeights W) {
  extern __shared__ __align__(128) char smem_raw[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int g = 0, t = tid;  // one warpgroup per CTA (named barrier 1)
  // 1024-byte aligned by an offset from the shared array itself, so that the
  // compiler keeps every access in the shared state space
  char* const nbase = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  NetSmem& N = *reinterpret_cast<NetSmem*>(nbase);
  // the staged network (MlpSmem image): W2 / 2 (forward: the product gives
  // a2/2, exactly) and W2^T into the swizzled B tiles (the FP32 layers come
  // as the kernel parameter W)
  {
    const MlpSmem& M = *reinterpret_cast<const MlpSmem*>(P.mlp);
    const uint16_t* w2 = reinterpret_cast<const uint16_t*>(&M.W2[0][0]);
    for (int i = tid; i < kNetH * kNetH; i += blockDim.x) {
      const int o = i / kNetH, u = i % kNetH;
      const uint16_t w = w2[o * kW2Pitch + u];
      const uint16_t wh = (uint16_t)(bf16x2(0.5f * __uint_as_float((uint32_t)w << 16), 0.f) & 0xffffu);
      *reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(N.B1) + net_elem(o, u)) = wh;
      *reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(N.B2) + net_elem(u, o)) = w;
    }
  }
  Smem S;
  S.base = nbase + sizeof(NetSmem);
  S.stage_bytes = P.stage_bytes;
  S.acc_bytes = ((P.max_slots * 8) + 127) / 128 * 128;
  S.tile_bytes = ((2 * P.tile_w * P.tile_h * 4) + 127) / 128 * 128;

  __shared__ int s_live, s_qempty;
  S.live = &s_live;
  S.qempty = &s_qempty;
  const int64_t total_units = P.prob_unit_prefix[P.nprob];
  int units_done = 0;
  if (tid == 0) {
    s_live = 0;
    s_qempty = 0;
    for (int s = 0; s < 2; ++s) {
      S.st(s).ctrl = (unsigned long long)(2u * s + 1u) << 32;  // "loading unit s"
      S.st(s).term = 0;
      S.st(s).tma_phase = 0;
      mbar_init(&S.st(s).mbar);
    }
    tc::mbar_init(&N.mbar);
  }
  if (warp == 0) {
    tc::tmem_alloc_more(&N.tmem, 64u);
    tc::tmem_alloc(&N.tmem_s1, 32u);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  bool ok = true;
  if (warp < 2) ok = load_unit<EXT>(S, warp, warp, P, total_units, units_done);
  __syncthreads();
  const unsigned tm = N.tmem, ts = N.tmem_s1;
  const unsigned tl = (unsigned)((warp & 3) * 32) << 16;
  unsigned phase = 0;

  // lane state (as in path_kernel)
  bool alive = false;
  int st = 0;
  uint32_t p = 0, kk = 0, tagw = 0;
  int n = 0;
  float xk = 0.f, yk = 0.f, bx0 = 0.f, bx1 = 0.f, by0 = 0.f, by1 = 0.f;
  float X = 0.f, Y = 0.f, Sx = 0.f, Z = 0.f, XI = 0.f;
  unsigned long long my_steps = 0, my_paths = 0, my_trunc = 0, my_clamp = 0;
  int want = 0;
  // EXT: the knot's step, its square root, step cap and Gobet-Menozzi shift
  // per unit of |s|; the mixed GM/EM run of the calibration (records kernels
  // with the extended exit) as in path_kernel
  constexpr bool kMixed = EXT && RECORD;
  bool gm_phase = false, pend_em = false, pend_tr = false;
  int64_t kmax_l = 0;
  float h_l = 0.f, sqh_l = 0.f, gmc = 0.f;
  const uint64_t wait_ns = P.wait_ns;
  // a product takes microseconds; its wait gets the launch's limit, but never
  // less than a second, so that no MMA can still be running when the kernel
  // gives up and releases its tensor memory
  const uint64_t mma_wait_ns = wait_ns > 1000000000ull ? wait_ns : 1000000000ull;
  uint64_t idle_since = 0;

  for (;;) {
    // every exit from this loop is decided for the whole group
    if (!group_all(g, ok)) break;
    // ---- hand new paths to idle lanes (per warp, never waits) --------------
    unsigned idle = __ballot_sync(kFull, !alive);
    for (int guard = 0; idle && guard < 64; ++guard) {
      Stage& H = S.st(want & 1);
      const unsigned ss = ctrl_state(&H.ctrl);
      if ((int)(ss >> 1) > want) { ++want; continue; }
      if ((ss & 1u) || (int)(ss >> 1) < want) break;
      if (H.term) { ++want; continue; }
      const int cnt = __popc(idle);
      const int leader = __ffs(idle) - 1;
      unsigned long long c = 0;
      if (lane == leader) c = atomicAdd(&H.ctrl, (unsigned long long)cnt);
      c = __shfl_sync(kFull, c, leader);
      __threadfence_block();
      const unsigned sa = (unsigned)(c >> 32);
      if (sa & 1u) break;
      const int base = (int)(unsigned)(c & 0xffffffffull);
      const int pend = H.p_end;
      __threadfence_block();
      if (ctrl_state(&H.ctrl) != sa) {
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
      if (base + cnt >= pend) ++want;
      idle = __ballot_sync(kFull, !alive);
    }
    if (!group_any(g, alive)) {
      // no path in the whole group: done once the queue is empty and no unit
      // of this CTA is loaded or loading, else wait (bounded) for a unit
      const int qe = *(volatile int*)S.qempty;
      __threadfence_block();
      const bool fin = qe && *(volatile int*)S.live == 0;
      if (group_all(g, fin)) break;
      if (idle_since == 0) idle_since = global_ns();
      if (group_any(g, global_ns() - idle_since > wait_ns)) {
        if (t == 0) atomicExch(&P.scratch->error, (int)PDDS_ETIMEOUT);
        break;
      }
      __nanosleep(256);
      continue;
    }
    idle_since = 0;

    // ---- step until a warp of the group has gathered enough exits ---------
    const float h = EXT ? h_l : P.h, sqh = EXT ? sqh_l : P.sqh;
    const float hl2 = h * 1.44269504088896341f;
    const int kmax = (int)min(EXT ? kmax_l : P.kmax, (int64_t)0x7fffffff);
    bool exited = false, trunc = false;
    if constexpr (kMixed) {
      exited = alive && pend_em;
      trunc = pend_tr;
    }
    for (;;) {
      const bool go = alive && !exited;
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (go) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(n >> 1), p, kk, tagw), P.round_keys);
        box_muller(r.x, r.y, z[0], z[1]);
        box_muller(r.z, r.w, z[2], z[3]);
      }
      // one copy of the network code for both steps of the Philox call
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const float za = half ? z[2] : z[0], zb = half ? z[3] : z[1];
        // the network at the step's starting point; while the forward product
        // runs, the step itself (the path does not depend on the network)
        net_grad_start(N, W, g, t, tm, ts, tl, xk + X, yk + Y);
        // a Philox call serves steps 2q and 2q + 1; a mixed-run path that
        // resumes at an odd step takes the second half of its call
        const bool stepping_now = go && !exited && (!kMixed || half >= (n & 1));
        float fac = 0.f, dWx = 0.f, dWy = 0.f;
        if (stepping_now) {
          const Stage& H = S.st(st);
          float s, ddx, ddy, c, f;
          coeffs<COEF>(H, S.tile(st, 0), S.tile(st, 1), xk + X, yk + Y, X, Y, P.trig_direct,
                       s, ddx, ddy, c, f);
          dWx = sqh * za;
          dWy = sqh * zb;
          float Yw = 1.0f;
          if constexpr (has_c<COEF>()) Yw = ex2_approx(Sx);
          if constexpr (has_f<COEF>()) Z = fmaf(-f * Yw, h, Z);
          if constexpr (has_c<COEF>()) Sx = fmaf(c, hl2, Sx);
          fac = -Yw * s;
          const float ssh = s * sqh;
          X = fmaf(ssh, za, fmaf(ddx, h, X));
          Y = fmaf(ssh, zb, fmaf(ddy, h, Y));
          ++n;
          exited = (X > bx1) | (X < bx0) | (Y > by1) | (Y < by0);
          if constexpr (EXT && !const_sigma<COEF>()) {
            if (exited && gmc > 0.f)
              exited = gm_outside<COEF>(H, S.tile(st, 0), S.tile(st, 1), xk, yk, X, Y, gmc,
                                        P.trig_direct);
          }
          if (!exited && n >= kmax) { exited = true; trunc = true; }
        }
        float gx, gy;
        if (!net_grad_finish(N, W, g, t, tm, ts, tl, phase, mma_wait_ns, gx, gy)) ok = false;
        // dxi = -Y s grad v . dW at the step's starting point (Eq. 37)
        if (stepping_now) XI = fmaf(fac, fmaf(gx, dWx, gy * dWy), XI);
      }
      const unsigned ex = __ballot_sync(kFull, alive && exited);
      const unsigned stepping = __ballot_sync(kFull, alive && !exited);
      if (group_any(g, stepping == 0 || __popc(ex) >= P.exit_batch || !ok)) break;
    }
    if (!ok && t == 0) atomicExch(&P.scratch->error, (int)PDDS_ETIMEOUT);

    // ---- resolve the exits (Eq. 22-25, corner rule of Sec. 3.3) -----------
    const bool leaving = alive && exited;
    bool gm_rec = false;  // a Gobet-Menozzi exit of a mixed run: recorded, the path goes on
    if constexpr (kMixed) gm_rec = leaving && gm_phase;
    ExitResult E;
    if (leaving)
      E = resolve_exit<COEF, RECORD, 1, EXT>(S, P, st, xk, yk, X, Y, Sx, Z, XI, trunc, bx0, bx1,
                                               by0, by1, gmc, gm_rec);
    if constexpr (EXT) {
      // RBF stencils (Eq. 21-22): the warp serves one exiting lane at a time,
      // a stencil knot per lane (as in path_kernel)
      unsigned pend = __ballot_sync(kFull, E.rbf_exit);
      while (pend) {
        const int src = __ffs(pend) - 1;
        const int r_st = __shfl_sync(kFull, st, src);
        const int r_side = __shfl_sync(kFull, E.side, src);
        const float r_s = __shfl_sync(kFull, E.sl, src);
        const float r_Y = __shfl_sync(kFull, E.Yk, src);
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
          const int tl2 = a + j;
          if (tl2 == 0 || tl2 == lmax) {
            const int li = vertical ? kd.line[r_side] : tl2;
            const int lj = vertical ? tl2 : kd.line[r_side];
            dsum += (double)w * (double)g_value<COEF>(H, fmaf((float)li, H.dx, H.x0),
                                                      fmaf((float)lj, H.dy, H.y0));
          } else if (!r_gm) {
            atomicAdd(acc + kd.off[r_side] + j, (unsigned long long)__float2ll_rn(w * kFixedOne));
          }
        }
        dsum = warp_sum(dsum);
        if (lane == src) E.bc += dsum;
        pend &= pend - 1;
      }
    }
    if (leaving) {
      if (!gm_rec) {
        my_steps += (unsigned long long)n;
        my_paths += 1;
        my_trunc += (E.flags & 1);
        my_clamp += (E.flags >> 1) & 1;
      }
      if constexpr (RECORD) write_record(S, P, st, kk, p, n, E, XI, gm_rec);
      if (!gm_rec) atomicAdd(&S.st(st).bsum, E.bc);
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
    // warp-aggregated completion counts per stage; the warp that finishes a
    // unit flushes it and loads the next one (bounded waits only)
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
        if (lane == 0) atomicSub(S.live, 1);
        __syncwarp();
      }
    }
    if (leaving && !gm_rec) alive = false;
  }

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
  // TMEM back once every warp is done with it
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(N.tmem, 64u);
    tc::tmem_dealloc(N.tmem_s1, 32u);
  }
}

}  // namespace
}  // namespace pdds
