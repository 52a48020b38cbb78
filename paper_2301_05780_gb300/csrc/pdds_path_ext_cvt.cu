// Extended-exit path-kernel variants with the tabulated gradient of u0
// (the production runs of the calibrated pipeline: per-knot h_k,
// Gobet-Menozzi shift, RBF stencils, xi of Eq. 37 from the table).
#include "path_kernel.cuh"

namespace pdds {
namespace {
template <int COEF, bool REC>
void* ptr() {
  return reinterpret_cast<void*>(&path_kernel<COEF, REC, 2, true>);
}
}  // namespace

void* path_kernel_ext_cvt(int coef, bool rec) {
  switch (coef) {
    case PDDS_COEF_LAPLACE_EXPSIN:
      return rec ? ptr<0, true>() : ptr<0, false>();
    case PDDS_COEF_MANUFACTURED:
      return rec ? ptr<1, true>() : ptr<1, false>();
    case PDDS_COEF_VARSIGMA:
      return rec ? ptr<2, true>() : ptr<2, false>();
    case PDDS_COEF_TABLE:
      return rec ? ptr<3, true>() : ptr<3, false>();
    case PDDS_COEF_CONSTANT:
      return rec ? ptr<4, true>() : ptr<4, false>();
    case PDDS_COEF_POISSON_E1:
      return rec ? ptr<5, true>() : ptr<5, false>();
    default:
      return nullptr;
  }
}

}  // namespace pdds
