// In-path network control variate on the fifth-generation tensor cores
// (path_kernel_net, naive EM exit; the extended-exit variants are in
// pdds_path_net_ext.cu): the analytic sets used with a learned v_theta and
// the constant set, as in pdds_path_cv.cu.
#include "path_kernel_net.cuh"

namespace pdds {
namespace {
template <int COEF, bool REC>
void* ptr() {
  return reinterpret_cast<void*>(&path_kernel_net<COEF, REC, false>);
}
}  // namespace

void* path_kernel_net_tc(int coef, bool rec) {
  switch (coef) {
    case PDDS_COEF_LAPLACE_EXPSIN:
      return rec ? ptr<0, true>() : ptr<0, false>();
    case PDDS_COEF_MANUFACTURED:
      return rec ? ptr<1, true>() : ptr<1, false>();
    case PDDS_COEF_CONSTANT:
      return rec ? ptr<4, true>() : ptr<4, false>();
    case PDDS_COEF_POISSON_E1:
      return rec ? ptr<5, true>() : ptr<5, false>();
    default:
      return nullptr;
  }
}

size_t net_smem_bytes() { return (size_t)kNetSmemBytes; }

// w: host array of the network's FP32 vectors, W1[:, 0], W1[:, 1], b1, b2, w3
// (64 each), passed halved, by value, as the kernel's second parameter.
void* path_kernel_net_ext_tc(int coef, bool rec);  // pdds_path_net_ext.cu

cudaError_t launch_path_kernel_net(int coef, bool rec, bool ext, const KParams& kp,
                                   const float* w, int grid, int block, size_t smem,
                                   cudaStream_t stream) {
  void* fn = ext ? path_kernel_net_ext_tc(coef, rec) : path_kernel_net_tc(coef, rec);
  if (!fn) return cudaErrorInvalidValue;
  NetWeights W;
  for (int u = 0; u < kNetH; ++u) {
    W.w1x[u] = 0.5f * w[u];
    W.w1y[u] = 0.5f * w[kNetH + u];
    W.b1[u] = 0.5f * w[2 * kNetH + u];
    W.b2[u] = 0.5f * w[3 * kNetH + u];
    W.w3[u] = 0.5f * w[4 * kNetH + u];
  }
  void* args[] = {const_cast<KParams*>(&kp), &W};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
}

}  // namespace pdds
