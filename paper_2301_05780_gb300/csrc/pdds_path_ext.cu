// Extended-exit path-kernel variants: per-knot steps h_k, the
// Gobet-Menozzi shift of the patch sides (Sec. 2.3) and RBF stencils.
#include "path_kernel.cuh"

namespace pdds {
namespace {
template <int COEF, bool REC>
void* ptr() {
  return reinterpret_cast<void*>(&path_kernel<COEF, REC, 0, true>);
}
}  // namespace

void* path_kernel_ext(int coef, bool rec) {
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
