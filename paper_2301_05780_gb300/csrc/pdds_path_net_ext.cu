// In-path network control variate on the fifth-generation tensor cores with
// the extended exit (per-knot steps, Gobet-Menozzi shift, RBF stencils, the
// mixed GM/EM run of the calibration): path_kernel_net<COEF, REC, true>.
#include "path_kernel_net.cuh"

namespace pdds {
namespace {
template <int COEF, bool REC>
void* ptr() {
  return reinterpret_cast<void*>(&path_kernel_net<COEF, REC, true>);
}
}  // namespace

void* path_kernel_net_ext_tc(int coef, bool rec) {
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

}  // namespace pdds
