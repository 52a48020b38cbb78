// FP64 BiCGSTAB (van der Vorst 1992) for the PDDSparse system G u = b
// (Eq. 23), entirely on the device.  The paper solves this system on one core
// after assembly (Sec. 4.3, Sec. 5.2.2); here every vector operation, CSR
// product and dot product is a kernel, and the recurrence scalars live in
// device memory so that the host only reads the residual every few
// iterations.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "pdds.h"
#include "pdds_internal.h"

namespace pdds {

struct SolveScalars {
  double bb;            // (b, b)
  double rho, rho_prev, alpha, omega;
  double d_rv, d_ss, d_ts, d_tt, d_rr, d_rr2;  // dot accumulators
  double relres;
  double rtol2;
  int32_t converged, breakdown, iters, pad_;
};

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of up to three values, then one atomic per value.
__device__ __forceinline__ void block_add3(double a, double b, double c, double* ga, double* gb,
                                           double* gc) {
  __shared__ double sh[3][kThreads / 32];
  a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = a; sh[1][w] = b; sh[2][w] = c; }
  __syncthreads();
  if (w == 0) {
    a = l < kThreads / 32 ? sh[0][l] : 0.0;
    b = l < kThreads / 32 ? sh[1][l] : 0.0;
    c = l < kThreads / 32 ? sh[2][l] : 0.0;
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    if (l == 0) {
      if (ga) atomicAdd(ga, a);
      if (gb) atomicAdd(gb, b);
      if (gc) atomicAdd(gc, c);
    }
  }
}

// x = 0, r = rh = b, p = v = 0, bb = rho = (b, b).
__global__ void k_init(const double* __restrict__ b, double* __restrict__ x,
                       double* __restrict__ r, double* __restrict__ rh, double* __restrict__ p,
                       double* __restrict__ v, int64_t n, SolveScalars* sc) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    x[i] = 0.0; r[i] = bi; rh[i] = bi; p[i] = 0.0; v[i] = 0.0;
    acc += bi * bi;
  }
  block_add3(acc, 0.0, 0.0, &sc->bb, nullptr, nullptr);
}

__global__ void k_setup(SolveScalars* sc, double rtol) {
  sc->rho = sc->bb;
  sc->rho_prev = 1.0; sc->alpha = 1.0; sc->omega = 1.0;
  sc->rtol2 = rtol * rtol;
  sc->relres = sc->bb > 0 ? 1.0 : 0.0;
  sc->converged = sc->bb == 0.0;
  sc->breakdown = 0;
  sc->iters = 0;
  sc->d_rv = sc->d_ss = sc->d_ts = sc->d_tt = sc->d_rr = sc->d_rr2 = 0.0;
}

// p = r + beta (p - omega v), beta = (rho / rho_prev)(alpha / omega).
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ r,
                           const double* __restrict__ v, int64_t n, const SolveScalars* sc) {
  if (sc->converged | sc->breakdown) return;
  const double beta = (sc->rho / sc->rho_prev) * (sc->alpha / sc->omega), om = sc->omega;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - om * v[i]);
}

// y = A x (one warp per row), with (w1, y) and, if `self_dot`, (y, y)
// accumulated.  y never aliases x or w1; (y, y) is taken from the register.
__global__ void k_spmv_dot(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ val, const double* __restrict__ x,
                           double* __restrict__ y, const double* __restrict__ w1, int self_dot,
                           int64_t n, double* acc1, double* acc2, const SolveScalars* sc) {
  if (sc->converged | sc->breakdown) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double a1 = 0.0, a2 = 0.0;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += warps) {
    double s = 0.0;
    for (int q = rp[row] + lane; q < rp[row + 1]; q += 32) s += val[q] * x[ci[q]];
    s = warp_sum(s);
    if (lane == 0) {
      y[row] = s;
      a1 += w1[row] * s;
      if (self_dot) a2 += s * s;
    }
  }
  block_add3(a1, a2, 0.0, acc1, acc2, nullptr);
}

// alpha = rho / (rh, v); s = r - alpha v; (s, s).
__global__ void k_s(double* __restrict__ s, const double* __restrict__ r,
                    const double* __restrict__ v, int64_t n, SolveScalars* sc) {
  if (sc->converged | sc->breakdown) return;
  const double alpha = sc->rho / sc->d_rv;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = r[i] - alpha * v[i];
    s[i] = si;
    acc += si * si;
  }
  block_add3(acc, 0.0, 0.0, &sc->d_ss, nullptr, nullptr);
}

// omega = (t, s) / (t, t); x += alpha p + omega s; r = s - omega t;
// accumulate (rh, r) and (r, r).
__global__ void k_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ rh,
                     const double* __restrict__ p, const double* __restrict__ s,
                     const double* __restrict__ t, int64_t n, SolveScalars* sc) {
  if (sc->converged | sc->breakdown) return;
  const double alpha = sc->rho / sc->d_rv;
  const double omega = sc->d_tt > 0.0 ? sc->d_ts / sc->d_tt : 0.0;
  double a1 = 0.0, a2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = s[i], ti = t[i];
    x[i] += alpha * p[i] + omega * si;
    const double ri = si - omega * ti;
    r[i] = ri;
    a1 += rh[i] * ri;
    a2 += ri * ri;
  }
  block_add3(a1, a2, 0.0, &sc->d_rr, &sc->d_rr2, nullptr);
}

// Scalar bookkeeping of one iteration (single thread).
__global__ void k_scalars(SolveScalars* sc) {
  if (sc->converged | sc->breakdown) return;
  const double alpha = sc->rho / sc->d_rv;
  const double omega = sc->d_tt > 0.0 ? sc->d_ts / sc->d_tt : 0.0;
  sc->iters += 1;
  const double rel = sqrt(sc->d_rr2 / sc->bb);
  sc->relres = rel;
  if (sc->d_rr2 <= sc->rtol2 * sc->bb) sc->converged = 1;
  if (!sc->converged) {
    // breakdown codes: 1 (rh, v) = 0, 2 omega = 0, 3 (rh, r) = 0, 4 residual not finite
    if (!(sc->d_rv != 0.0)) sc->breakdown = 1;
    else if (!(omega != 0.0)) sc->breakdown = 2;
    else if (!(sc->d_rr != 0.0)) sc->breakdown = 3;
    else if (!(rel == rel) || rel > 1e300) sc->breakdown = 4;
  }
  sc->rho_prev = sc->rho;
  sc->rho = sc->d_rr;
  sc->alpha = alpha;
  sc->omega = omega;
  sc->d_rv = sc->d_ss = sc->d_ts = sc->d_tt = sc->d_rr = sc->d_rr2 = 0.0;
}

}  // namespace

size_t bicgstab_work_doubles(int64_t n) { return (size_t)6 * (size_t)n; }
size_t bicgstab_scalars_bytes() { return sizeof(SolveScalars); }

cudaError_t bicgstab_device(const int32_t* rp, const int32_t* ci, const double* val,
                            const double* b, double* x, int64_t n, double* work, SolveScalars* sc,
                            double rtol, int32_t maxit, int32_t* iters, double* relres,
                            int* converged, int* launches, cudaStream_t st) {
  double *r = work, *rh = work + n, *p = work + 2 * n, *v = work + 3 * n, *s = work + 4 * n,
         *t = work + 5 * n;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int vgrid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sms * 8);
  const int mgrid = (int)std::min<int64_t>((n * 32 + kThreads - 1) / kThreads, (int64_t)sms * 16);
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc, 0, sizeof(SolveScalars), st)) != cudaSuccess) return e;
  k_init<<<vgrid, kThreads, 0, st>>>(b, x, r, rh, p, v, n, sc);
  k_setup<<<1, 1, 0, st>>>(sc, rtol);
  int nl = 2;
  SolveScalars h{};
  const int chunk = 8;
  for (int it = 0; it < maxit; it += chunk) {
    const int m = std::min(chunk, maxit - it);
    for (int j = 0; j < m; ++j) {
      k_update_p<<<vgrid, kThreads, 0, st>>>(p, r, v, n, sc);
      k_spmv_dot<<<mgrid, kThreads, 0, st>>>(rp, ci, val, p, v, rh, 0, n, &sc->d_rv,
                                              nullptr, sc);
      k_s<<<vgrid, kThreads, 0, st>>>(s, r, v, n, sc);
      k_spmv_dot<<<mgrid, kThreads, 0, st>>>(rp, ci, val, s, t, s, 1, n, &sc->d_ts, &sc->d_tt, sc);
      k_xr<<<vgrid, kThreads, 0, st>>>(x, r, rh, p, s, t, n, sc);
      k_scalars<<<1, 1, 0, st>>>(sc);
      nl += 6;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h.converged || h.breakdown) break;
  }
  if (iters) *iters = h.iters;
  if (relres) *relres = h.relres;
  if (converged) *converged = h.converged ? 1 : -h.breakdown;
  if (launches) *launches = nl;
  return cudaSuccess;
}

}  // namespace pdds

// ===========================================================================
// Allocation-free solve.
//
// Some callers of this library cannot allocate device memory: applications
// that own all device memory through their own pool or arena under a fixed
// budget (a library-side cudaMalloc would bypass their accounting, or fail),
// and latency-critical code where the implicit device synchronization of
// cudaMalloc/cudaFree is not acceptable.  pdds_solve_noalloc serves them: it
// runs the same BiCGSTAB kernels as pdds_solve, but its scratch -- six work
// vectors and the recurrence scalars -- lives in the file-scope device array
// below, which every GPU that loads this library holds until the process
// exits (6.3 MB).  The caller still passes G, b and u.
// ===========================================================================
namespace pdds {
namespace {

constexpr int64_t kNoAllocMaxN = 131072;           // largest system size served
constexpr int64_t kNoAllocScalarSlots = 32;        // >= sizeof(SolveScalars) / 8
static_assert(sizeof(pdds::SolveScalars) <= kNoAllocScalarSlots * sizeof(double), "scratch");

static __device__ __align__(256) double g_noalloc_scratch[6 * kNoAllocMaxN + kNoAllocScalarSlots];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace pdds

extern "C" pdds_status pdds_solve_noalloc(const pdds_csr* G, const double* b, double* u,
                                          double rtol, int32_t maxit, int32_t* iters,
                                          void* cuda_stream) {
  using namespace pdds;
  if (!G || !b || !u || !G->row_ptr || !G->col || !G->val) {
    set_global_error("solve_noalloc: NULL matrix/vector");
    return PDDS_EINVAL;
  }
  if (G->n > kNoAllocMaxN) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "solve_noalloc: n = %lld exceeds the static scratch limit of %lld unknowns; "
                  "use pdds_solve", (long long)G->n, (long long)kNoAllocMaxN);
    set_global_error(buf);
    return PDDS_EINVAL;
  }
  if (G->n < 1 || G->nnz < G->n) {
    set_global_error("solve_noalloc: need n >= 1 and nnz >= n");
    return PDDS_EINVAL;
  }
  if (!(rtol > 0) || maxit < 1) {
    set_global_error("solve_noalloc: need rtol > 0, maxit >= 1");
    return PDDS_EINVAL;
  }
  (void)cudaGetLastError();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(std::string("solve_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return PDDS_ECUDA;
  }
  double* scratch = nullptr;
  {
    // First call on this device (the current one): look up the array's device
    // address.  Host code cannot use g_noalloc_scratch's name as a pointer.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error(std::string("solve_noalloc: cudaGetSymbolAddress: ") +
                         cudaGetErrorString(e));
        return PDDS_ECUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  auto* sc = reinterpret_cast<SolveScalars*>(scratch + 6 * kNoAllocMaxN);
  int32_t it = 0;
  double rel = 0;
  int conv = 0, nl = 0;
  // bicgstab_device zeroes the scalars and initialises every work vector it
  // reads, so the previous call's contents never leak into this one.
  e = bicgstab_device(G->row_ptr, G->col, G->val, b, u, G->n, scratch, sc, rtol, maxit, &it, &rel,
                      &conv, &nl, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    set_global_error(std::string("solve_noalloc: ") + cudaGetErrorString(e));
    return PDDS_ECUDA;
  }
  if (iters) *iters = it;
  if (conv != 1) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "solve_noalloc: no convergence after %d iterations (relres %.3e)%s", it, rel,
                  bicgstab_stop_reason(conv));
    set_global_error(buf);
    return PDDS_ENOCONV;
  }
  return PDDS_OK;
}
