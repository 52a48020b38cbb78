// Launch plumbing of the persistent path kernel: per-knot unit and record
// prefixes, the per-problem unit prefix, the finalize kernel (Eq. 24-25) and
// the dispatch to the kernel variants, which are instantiated in
// pdds_path_{em,cv,cvt,ext,ext_cv,ext_cvt}.cu so that they compile in parallel.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "pdds.h"
#include "pdds_internal.h"
#include "path_kernel.cuh"

namespace pdds {
namespace {

// ------------------------------------------------------ prefix / finalize
// A budget outside [0, 2^31) counts as no paths (the knot keeps row e_k).
__device__ __forceinline__ int64_t checked_budget(int64_t v, bool& bad) {
  if (v < 0 || v > 0x7fffffffll) { bad = true; return 0; }
  return v;
}

// Single block: units and records before each knot (exclusive prefix sums).
// An invalid budget is skipped and recorded as PDDS_EINVAL in *err.
__global__ void unit_prefix_kernel(const int64_t* __restrict__ N, int64_t n, int64_t C,
                                   int64_t* __restrict__ up, int64_t* __restrict__ pp,
                                   int32_t* __restrict__ err) {
  __shared__ int64_t su[1024], sp[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (n + T - 1) / T;
  const int64_t lo = min(n, t * per), hi = min(n, lo + per);
  int64_t a = 0, b = 0;
  bool bad = false;
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t v = checked_budget(N[i], bad);
    a += (v + C - 1) / C;
    b += v;
  }
  if (bad) atomicExch(err, (int32_t)PDDS_EINVAL);
  su[t] = a; sp[t] = b;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const int64_t va = t >= o ? su[t - o] : 0, vb = t >= o ? sp[t - o] : 0;
    __syncthreads();
    su[t] += va; sp[t] += vb;
    __syncthreads();
  }
  a = su[t] - a; b = sp[t] - b;  // exclusive
  for (int64_t i = lo; i < hi; ++i) {
    up[i] = a; pp[i] = b;
    const int64_t v = checked_budget(N[i], bad);
    a += (v + C - 1) / C; b += v;
  }
  if (t == T - 1) { up[n] = su[t]; pp[n] = sp[t]; }
}

// Units of each problem before it (exclusive prefix over problems).
__global__ void prob_prefix_kernel(const ProbDesc* probs, ProbDesc single, int nprob, int64_t* out) {
  int64_t acc = 0;
  out[0] = 0;
  for (int i = 0; i < nprob; ++i) {
    const ProbDesc& D = nprob == 1 && probs == nullptr ? single : probs[i];
    acc += D.knot_unit_prefix ? D.knot_unit_prefix[D.n] : (int64_t)D.n * D.units_per_knot;
    out[i + 1] = acc;
  }
}

// One warp per row: G_kk = 1, G_kj = -sum/N_k, b_k = sum/N_k (Eq. 24-25).
__global__ void finalize_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                double* __restrict__ val, double* __restrict__ b,
                                const int64_t* __restrict__ N, int64_t Nu, int64_t n) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const int64_t Nk = N ? N[k] : Nu;
  const double inv = Nk > 0 ? 1.0 / (double)Nk : 0.0;  // no paths: row e_k, b_k = 0
  for (int q = row_ptr[k] + lane; q < row_ptr[k + 1]; q += 32)
    val[q] = (col[q] == (int32_t)k) ? 1.0 : -val[q] * inv;
  if (lane == 0) b[k] *= inv;
}

}  // namespace

// Kernel variants, one translation unit each (pdds_path_em.cu, ...): no
// control variate / in-path network / tabulated gradient, each with and
// without the extended exit (per-knot steps, Gobet-Menozzi shift, RBF
// stencils).  nullptr: no such variant.
void* path_kernel_em(int coef, bool rec);
void* path_kernel_cv(int coef, bool rec);
void* path_kernel_cvt(int coef, bool rec);
void* path_kernel_ext(int coef, bool rec);
void* path_kernel_ext_cv(int coef, bool rec);
void* path_kernel_ext_cvt(int coef, bool rec);
void* path_kernel_net_tc(int coef, bool rec);      // cv 3: the network on tcgen05 (pdds_path_net.cu)
void* path_kernel_net_ext_tc(int coef, bool rec);  // the same with the extended exit

namespace {
void* pick(int coef, bool rec, int cv, bool ext) {
  if (ext) {
    if (cv == 3) return path_kernel_net_ext_tc(coef, rec);
    if (cv == 1) return path_kernel_ext_cv(coef, rec);
    if (cv == 2) return path_kernel_ext_cvt(coef, rec);
    return path_kernel_ext(coef, rec);
  }
  if (cv == 1) return path_kernel_cv(coef, rec);
  if (cv == 2) return path_kernel_cvt(coef, rec);
  if (cv == 3) return path_kernel_net_tc(coef, rec);
  return path_kernel_em(coef, rec);
}
}  // namespace

bool path_kernel_has_cv(int coef) { return pick(coef, false, 1, false) != nullptr; }

cudaError_t launch_path_kernel(int coef, bool rec, int cv, bool ext, const KParams& kp, int grid,
                               int block, size_t smem, cudaStream_t stream) {
  void* fn = pick(coef, rec, cv, ext);
  if (!fn) return cudaErrorInvalidValue;
  void* args[] = {const_cast<KParams*>(&kp)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
}

cudaError_t path_kernel_occupancy(int coef, bool rec, int cv, bool ext, int block, size_t smem,
                                  int* ctas) {
  void* fn = pick(coef, rec, cv, ext);
  if (!fn) return cudaErrorInvalidValue;
  if (cv != 3) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, block, smem);
  // The tcgen05 network kernel: the occupancy query answers one CTA per SM
  // for it, while registers, shared memory (large carve-out) and tensor
  // memory admit five (measured: several 128-thread CTAs per SM run more than
  // twice as fast as one), so the count is taken from those three limits.
  cudaFuncAttributes fa;
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  const int regs = (fa.numRegs + 7) / 8 * 8;  // allocated per warp in 256-register steps
  const int by_regs = regs_sm / (regs * block);
  const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + (size_t)smem_res);
  const int by_tmem = 512 / 96;  // 64 + 32 TMEM columns per 128-thread CTA
  *ctas = std::max(0, std::min(std::min(by_regs, by_smem), by_tmem));
  return cudaSuccess;
}

cudaError_t set_path_kernel_smem(int coef, bool rec, int cv, bool ext, size_t smem) {
  void* fn = pick(coef, rec, cv, ext);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the tcgen05 network kernel (~55 KB per CTA) needs the large shared-memory
  // carve-out for two CTAs per SM
  if (e == cudaSuccess && cv == 3)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_unit_prefix(const int64_t* N, int64_t n, int64_t C, int64_t* up, int64_t* pp,
                               int32_t* err, cudaStream_t stream) {
  unit_prefix_kernel<<<1, 1024, 0, stream>>>(N, n, C, up, pp, err);
  return cudaGetLastError();
}

cudaError_t launch_prob_prefix_single(const ProbDesc& D, int64_t* out, cudaStream_t stream) {
  prob_prefix_kernel<<<1, 1, 0, stream>>>(nullptr, D, 1, out);
  return cudaGetLastError();
}

cudaError_t launch_prob_prefix(const ProbDesc* probs, int nprob, int64_t* out, cudaStream_t stream) {
  prob_prefix_kernel<<<1, 1, 0, stream>>>(probs, ProbDesc{}, nprob, out);
  return cudaGetLastError();
}

__global__ void cv_cells_kernel(const float* __restrict__ nodes, int nx, int ny,
                                float* __restrict__ cells) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)(nx - 1) * (ny - 1);
  if (c >= ncell) return;
  const int i = (int)(c % (nx - 1)), j = (int)(c / (nx - 1));
  const float2* n2 = reinterpret_cast<const float2*>(nodes);
  const float2 a = n2[(int64_t)j * nx + i], b = n2[(int64_t)j * nx + i + 1];
  const float2 d0 = n2[(int64_t)(j + 1) * nx + i], d1 = n2[(int64_t)(j + 1) * nx + i + 1];
  float4* o = reinterpret_cast<float4*>(cells) + 2 * c;
  o[0] = make_float4(a.x, b.x, d0.x, d1.x);
  o[1] = make_float4(a.y, b.y, d0.y, d1.y);
}

cudaError_t launch_cv_cells(const float* nodes, int nx, int ny, float* cells, cudaStream_t s) {
  const int64_t ncell = (int64_t)(nx - 1) * (ny - 1);
  cv_cells_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(nodes, nx, ny, cells);
  return cudaGetLastError();
}

// Samples of the boundary data g (Eq. 6) at the midpoints of n equal
// intervals of each side of Omega (E, N, W, S), evaluated as the path kernel
// evaluates g at an exit on the boundary.
struct Params8 {
  float v[8];
};
template <int COEF>
__global__ void boundary_samples_kernel(float x0, float x1, float y0, float y1, int n, Params8 prm,
                                        float* __restrict__ xy, float* __restrict__ g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * (int64_t)n) return;
  const int side = (int)(i / n);
  const float t = ((float)(i % n) + 0.5f) / (float)n;
  const float ax = fmaf(t, x1 - x0, x0), ay = fmaf(t, y1 - y0, y0);
  const float x = side == 0 ? x1 : side == 2 ? x0 : ax;
  const float y = side == 1 ? y1 : side == 3 ? y0 : ay;
  Stage H;  // g reads only the set's constants
  for (int q = 0; q < 8; ++q) H.params[q] = prm.v[q];
  xy[2 * i] = x;
  xy[2 * i + 1] = y;
  g[i] = g_value<COEF>(H, x, y);
}

cudaError_t launch_boundary_samples(int coef, const double dom[4], const double params[8], int n,
                                    float* xy, float* g, cudaStream_t s) {
  Params8 prm;
  for (int q = 0; q < 8; ++q) prm.v[q] = (float)params[q];
  const float x0 = (float)dom[0], x1 = (float)dom[1], y0 = (float)dom[2], y1 = (float)dom[3];
  const unsigned blocks = (unsigned)((4 * (int64_t)n + 255) / 256);
  switch (coef) {
    case PDDS_COEF_LAPLACE_EXPSIN:
      boundary_samples_kernel<0><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    case PDDS_COEF_MANUFACTURED:
      boundary_samples_kernel<1><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    case PDDS_COEF_VARSIGMA:
      boundary_samples_kernel<2><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    case PDDS_COEF_TABLE:
      boundary_samples_kernel<3><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    case PDDS_COEF_CONSTANT:
      boundary_samples_kernel<4><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    case PDDS_COEF_POISSON_E1:
      boundary_samples_kernel<5><<<blocks, 256, 0, s>>>(x0, x1, y0, y1, n, prm, xy, g); break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t stage_header_bytes() { return (size_t)kStageHdr; }

cudaError_t launch_finalize(const int32_t* row_ptr, const int32_t* col, double* val, double* b,
                            const int64_t* N, int64_t Nu, int64_t n, cudaStream_t stream) {
  const int threads = 256;
  const int64_t blocks = (n * 32 + threads - 1) / threads;
  finalize_kernel<<<(unsigned)blocks, threads, 0, stream>>>(row_ptr, col, val, b, N, Nu, n);
  return cudaGetLastError();
}

}  // namespace pdds

