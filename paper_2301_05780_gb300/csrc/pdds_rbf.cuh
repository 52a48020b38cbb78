// Device evaluation of the tabulated RBF cardinal functions (see pdds_rbf.cpp):
// H_j on lattice interval t of an L-point stencil is a Chebyshev series in
// tau = 2 (s - t) - 1, coefficients at cf[(t (P1) + n) L + j], n < P1.
#pragma once
#include <stdint.h>

#include "pdds_internal.h"

namespace pdds {

// Start of interval t's coefficients for an L-point stencil of orientation o
// (0: line along x, 1: line along y), and tau for the coordinate s (lattice
// spacings from the stencil's first knot, 0 <= s <= L - 1).  nullptr when no
// table exists for that length (the caller then deposits nothing and reports).
__device__ __forceinline__ const float* rbf_interval(const ProbDesc& D, int o, int L, float s,
                                                     float& tau) {
  tau = 0.f;
  if (L < 2 || L > D.rbf_lmax) return nullptr;
  const int64_t off = D.rbf_off[(int64_t)o * (D.rbf_lmax + 1) + L];
  if (off < 0) return nullptr;
  int t = (int)floorf(s);
  t = max(0, min(t, L - 2));
  tau = fmaf(2.0f, s - (float)t, -1.0f);
  const int P1 = D.rbf_deg + 1;
  return D.rbf_coef + off + (int64_t)t * P1 * L;
}

// H_j(tau) by Clenshaw's recurrence.
__device__ __forceinline__ float rbf_cardinal(const float* cf, int L, int P1, int j, float tau) {
  float b1 = 0.f, b2 = 0.f;
  const float t2 = 2.0f * tau;
  for (int n = P1 - 1; n >= 1; --n) {
    const float v = fmaf(t2, b1, __ldg(cf + (int64_t)n * L + j) - b2);
    b2 = b1;
    b1 = v;
  }
  return fmaf(tau, b1, __ldg(cf + j) - b2);
}

}  // namespace pdds
