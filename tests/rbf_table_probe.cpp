// Test driver (CPU): builds the library's RBF cardinal-function tables with
// pdds::rbf_build_tables and evaluates them the way the path kernel does
// (Clenshaw on the [interval][coefficient][knot] layout), printing H_j(s)
// for the stencils and points read from stdin:
//   input : c_lat  then lines "L s"  (orientation 0)
//   output: for each line, L values H_0..H_{L-1}
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "pdds_internal.h"

int main() {
  double c;
  if (std::scanf("%lf", &c) != 1) return 2;
  std::vector<std::pair<int, double>> q;
  int L;
  double s;
  while (std::scanf("%d %lf", &L, &s) == 2) q.push_back({L, s});
  std::vector<int> lengths[2];
  for (auto& p : q) {
    bool seen = false;
    for (int v : lengths[0]) seen |= (v == p.first);
    if (!seen) lengths[0].push_back(p.first);
  }
  const double c_lat[2] = {c, c};
  pdds::RbfTables T;
  std::string err;
  if (!pdds::rbf_build_tables(lengths, c_lat, T, err)) {
    std::printf("error %s\n", err.c_str());
    return 1;
  }
  std::printf("degree %d err %.3e\n", T.degree, T.max_err);
  const int P1 = T.degree + 1;
  for (auto& p : q) {
    const int Ls = p.first;
    const int64_t off = T.offset[Ls];
    int t = (int)std::floor(p.second);
    if (t > Ls - 2) t = Ls - 2;
    if (t < 0) t = 0;
    const float tau = 2.0f * (float)(p.second - t) - 1.0f;
    const float* cf = T.coef.data() + off + (int64_t)t * P1 * Ls;
    for (int j = 0; j < Ls; ++j) {
      float b1 = 0.f, b2 = 0.f;
      for (int n = P1 - 1; n >= 1; --n) {
        const float v = std::fma(2.0f * tau, b1, cf[(int64_t)n * Ls + j] - b2);
        b2 = b1;
        b1 = v;
      }
      std::printf("%.9e ", (double)std::fma(tau, b1, cf[j] - b2));
    }
    std::printf("\n");
  }
  std::printf("shape %.12e\n", pdds::rbf_shape_for_cond(q.empty() ? 2 : q[0].first, 1e10));
  return 0;
}
