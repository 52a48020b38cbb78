// Calibration of the PDDSparse production run (arXiv 2301.05780, Sec. 4.1-4.2).
//
// calib_moments_kernel: per knot, the moments of the "mixed GM/EM" scores.
//   The naive and the Gobet-Menozzi pass of the path kernel use the same Philox
//   counters, so path p of knot k follows one trajectory in both: the GM pass
//   records it at the first step beyond a moved patch side, the naive pass at
//   the first step outside the patch -- the two exits of one mixed path.  With
//   the warm-up nodal solution u0 as patch data, a score is
//     phi = b_contrib - xi + w_a u0[col_a] + w_b u0[col_b]
//   (the path's share of b without the control variate, plus its weights on
//   the stencil knots applied to u0: the same row as G's).  One warp per knot
//   sums, in FP64 and in a fixed order,
//     N, sum d, sum d^2, sum phi_GM, sum phi_GM^2, sum xi, sum xi^2, sum phi_GM xi
//   with d = phi_EM - phi_GM and xi taken at the GM exit.
//
// plan_kernel: Eq. 40-41 per knot (h_i and N_i for accuracy eps).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdds_internal.h"
#include "pdds_rbf.cuh"

namespace pdds {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNMom = 8;

// phi of one path.  Linear stencils: the record's two weights.  RBF stencils
// (D.rbf_coef set): Y H_j(s_line) on every unknown knot j of the exit side's
// stencil (boundary knots are already in b_contrib), from the same tables the
// path kernel used.
__device__ __forceinline__ double score(const PathRecordDev& r, const double* __restrict__ u0,
                                        const ProbDesc& D, const KnotDesc& kd) {
  double phi = (double)r.b_contrib - (double)r.xi;
  if (r.col_a >= 0) phi += (double)r.w_a * u0[r.col_a];
  if (r.col_b >= 0) phi += (double)r.w_b * u0[r.col_b];
  const int side = r.side_flags & 0xFF;
  if (D.rbf_coef != nullptr && !((kd.dirbits >> side) & 1)) {
    const bool vertical = (side == 0 || side == 2);
    const int a = kd.a[side];
    const int L = kd.b[side] - a + 1;
    float tau;
    const float* cf = rbf_interval(D, vertical ? 1 : 0, L, r.s_line - (float)a, tau);
    const int32_t* map = D.slot2csr + kd.slot_base + kd.off[side];
    double acc = 0.0;
    for (int j = 0; cf != nullptr && j < L; ++j) {
      const int c = map[j];
      if (c < 0) continue;
      acc += (double)(r.Y * rbf_cardinal(cf, L, D.rbf_deg + 1, j, tau)) * u0[D.col[c]];
    }
    phi += acc;
  }
  return phi;
}

__global__ void calib_moments_kernel(const PathRecordDev* __restrict__ em,
                                     const PathRecordDev* __restrict__ gm,
                                     const int64_t* __restrict__ path_prefix, int64_t n_paths,
                                     const double* __restrict__ u0, int64_t n,
                                     double* __restrict__ mom, const ProbDesc D) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const int64_t beg = path_prefix ? path_prefix[k] : k * n_paths;
  const int64_t end = path_prefix ? path_prefix[k + 1] : beg + n_paths;
  double m[kNMom] = {0, 0, 0, 0, 0, 0, 0, 0};
  const KnotDesc& kd = D.knots[k];
  for (int64_t i = beg + lane; i < end; i += 32) {
    const PathRecordDev a = em[i];
    const PathRecordDev b = gm[i];
    const double pe = score(a, u0, D, kd), pg = score(b, u0, D, kd), x = (double)b.xi;
    const double d = pe - pg;
    m[1] += d;
    m[2] += d * d;
    m[3] += pg;
    m[4] += pg * pg;
    m[5] += x;
    m[6] += x * x;
    m[7] += pg * x;
  }
#pragma unroll
  for (int j = 1; j < kNMom; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m[j] += __shfl_xor_sync(kFull, m[j], o);
  if (lane == 0) {
    m[0] = (double)(end - beg);
#pragma unroll
    for (int j = 0; j < kNMom; ++j) mom[k * kNMom + j] = m[j];
  }
}

// Eq. 40-41 for one knot, in the order the formulas are written (no fused
// multiply-add can form: no product feeds an addition directly).
__global__ void plan_kernel(const double* __restrict__ mom, int64_t n, double eps, double h0,
                            double h0p, int64_t n_job, double* __restrict__ h_out,
                            int64_t* __restrict__ n_out, double* __restrict__ diag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* m = mom + i * kNMom;
  const double N = m[0];
  const double gap = N > 0 ? m[1] / N : 0.0;
  double var = 0.0, vx = 0.0, cov = 0.0;
  if (N > 1) {
    var = (m[4] - m[3] * m[3] / N) / (N - 1.0);
    vx = (m[6] - m[5] * m[5] / N) / (N - 1.0);
    cov = (m[7] - m[3] * m[5] / N) / (N - 1.0);
  }
  if (var < 0) var = 0;
  double rho2 = (var > 0 && vx > 0) ? cov * cov / (var * vx) : 0.0;
  if (rho2 > 1.0) rho2 = 1.0;
  double h = h0;  // Eq. 40: the GM bias at h0' is bounded by |gap| / 2 (Eq. 35)
  if (gap != 0.0) {
    const double hb = 2.0 * h0p * eps / (3.0 * fabs(gap));
    if (hb < h) h = hb;
  }
  // Eq. 41: (2/3) eps = 2 sqrt(V (1 - rho^2) / N), rounded to k N_job, k >= 1
  const double nraw = 9.0 * var * (1.0 - rho2) / (eps * eps);
  double kj = rint(nraw / (double)n_job);
  if (!(kj >= 1.0)) kj = 1.0;  // also a NaN variance: one job
  // N_i stays a valid budget: at most the largest multiple of N_job below 2^31
  const double kcap = floor(2147483647.0 / (double)n_job);
  if (kj > kcap) kj = kcap;
  h_out[i] = h;
  n_out[i] = (int64_t)kj * n_job;
  if (diag) {
    diag[3 * i] = gap;
    diag[3 * i + 1] = var;
    diag[3 * i + 2] = rho2;
  }
}

}  // namespace

cudaError_t launch_calib_moments(const PathRecordDev* rec_em, const PathRecordDev* rec_gm,
                                 const int64_t* path_prefix, int64_t n_paths, const double* u0,
                                 int64_t n, double* moments, const ProbDesc& D,
                                 cudaStream_t stream) {
  const int threads = 256;
  const int64_t blocks = (n * 32 + threads - 1) / threads;
  calib_moments_kernel<<<(unsigned)blocks, threads, 0, stream>>>(rec_em, rec_gm, path_prefix,
                                                                   n_paths, u0, n, moments, D);
  return cudaGetLastError();
}

cudaError_t launch_plan(const double* moments, int64_t n, double eps, double h0, double h0p,
                        int64_t n_job, double* h_out, int64_t* n_out, double* diag,
                        cudaStream_t stream) {
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  plan_kernel<<<(unsigned)blocks, threads, 0, stream>>>(moments, n, eps, h0, h0p, n_job, h_out,
                                                          n_out, diag);
  return cudaGetLastError();
}

}  // namespace pdds
