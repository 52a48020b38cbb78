// In-path network control variate on the fifth-generation tensor cores
// (path_kernel_net, naive EM exit): the analytic sets used with a learned
// v_theta and the constant set, as in pdds_path_cv.cu.
#include "path_kernel_net.cuh"

namespace pdds {
namespace {
template <int COEF, bool REC>
void* ptr() {
  return reinterpret_cast<void*>(&path_kernel_net<COEF, REC>);
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

}  // namespace pdds
