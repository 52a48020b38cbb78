// Cardinal-function tables of the 1-D inverse-multiquadric RBF interpolation
// on patch-side stencils (arXiv 2301.05780: Sec. 2.1, Eq. 1-5; Eq. 21-22).
//
// A stencil is m equispaced lattice points of one interface line, so in
// lattice units its cardinal functions depend only on m and on the shape
// parameter measured in lattice spacings, c_lat:
//   H(z) = Phi^{-1} phi(z),  Phi_ij = phi_c(|i - j|),  phi(z)_i = phi_c(|z - i|),
//   phi_c(r) = 1 / sqrt(r^2 + c^2)          (Eq. 3, read with + c^2).
// For every stencil length that occurs, H_0..H_{m-1} are computed in FP64 on
// each lattice interval [t, t+1] at Chebyshev points and stored as Chebyshev
// coefficients (FP32, laid out [t][n][j]) of one common degree, chosen as the smallest of
// 7, 11, 15, 19, 23 whose truncation error is below 2e-7 of max |H|; the
// path kernel evaluates them with Clenshaw's recurrence at every interface
// exit.  The spectral condition number of Phi sets c when the caller gives
// none (the paper fixes it at O(1e10), Sec. 5.1): power iteration for the
// largest eigenvalue, inverse iteration with a Cholesky factor for the
// smallest, bisection on log c.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pdds_internal.h"

namespace pdds {
namespace {

constexpr double kPi = 3.14159265358979323846;

inline double imq(double r, double c) { return 1.0 / std::sqrt(r * r + c * c); }

void phi_matrix(int m, double c, std::vector<double>& A) {
  A.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = imq((double)(i - j), c);
}

// Lower Cholesky factor in place (row-major, upper part ignored).
bool cholesky(int m, std::vector<double>& A) {
  for (int j = 0; j < m; ++j) {
    double d = A[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * m + k] * A[(size_t)j * m + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
      A[(size_t)i * m + j] = v / d;
    }
  }
  return true;
}

void chol_solve(int m, const std::vector<double>& L, double* x) {
  for (int i = 0; i < m; ++i) {
    double v = x[i];
    for (int k = 0; k < i; ++k) v -= L[(size_t)i * m + k] * x[k];
    x[i] = v / L[(size_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < m; ++k) v -= L[(size_t)k * m + i] * x[k];
    x[i] = v / L[(size_t)i * m + i];
  }
}

// Spectral condition number of the SPD Phi(m, c); < 0 if not SPD numerically.
double cond_spd(int m, double c) {
  std::vector<double> A, L;
  phi_matrix(m, c, A);
  L = A;
  if (!cholesky(m, L)) return -1.0;
  std::vector<double> x(m), y(m);
  // largest eigenvalue: power iteration from the all-ones vector (Perron)
  for (int i = 0; i < m; ++i) x[i] = 1.0 / std::sqrt((double)m);
  double lmax = 0;
  for (int it = 0; it < 500; ++it) {
    double nrm = 0;
    for (int i = 0; i < m; ++i) {
      double v = 0;
      for (int j = 0; j < m; ++j) v += A[(size_t)i * m + j] * x[j];
      y[i] = v;
      nrm += v * v;
    }
    nrm = std::sqrt(nrm);
    const double prev = lmax;
    lmax = nrm;
    for (int i = 0; i < m; ++i) x[i] = y[i] / nrm;
    if (it > 10 && std::fabs(lmax - prev) <= 1e-14 * lmax) break;
  }
  // smallest eigenvalue: inverse iteration (alternating start so that it is
  // not orthogonal to the oscillating eigenvector)
  for (int i = 0; i < m; ++i) x[i] = ((i & 1) ? -1.0 : 1.0) / std::sqrt((double)m) * (1.0 + 0.01 * i);
  double mu = 0;
  for (int it = 0; it < 500; ++it) {
    y = x;
    chol_solve(m, L, y.data());
    double nrm = 0;
    for (double v : y) nrm += v * v;
    nrm = std::sqrt(nrm);
    const double prev = mu;
    mu = nrm;  // ~ 1 / lambda_min
    for (int i = 0; i < m; ++i) x[i] = y[i] / nrm;
    if (it > 10 && std::fabs(mu - prev) <= 1e-13 * mu) break;
  }
  return lmax * mu;
}

}  // namespace

double rbf_shape_for_cond(int m, double cond) {
  double lo = 1e-3, hi = 1e2;
  for (int it = 0; it < 200 && hi / lo > 1.0 + 1e-10; ++it) {
    const double mid = std::sqrt(lo * hi);
    const double k = cond_spd(m, mid);
    if (k >= 0 && k < cond) lo = mid; else hi = mid;
  }
  return std::sqrt(lo * hi);
}

double rbf_cond(int m, double c_lat) { return cond_spd(m, c_lat); }

bool rbf_build_tables(const std::vector<int> lengths[2], const double c_lat[2], RbfTables& T,
                      std::string& err) {
  const int kMaxDeg = 23;
  const int K = kMaxDeg + 1;
  T.lmax = 0;
  for (int o = 0; o < 2; ++o)
    for (int L : lengths[o]) T.lmax = std::max(T.lmax, L);
  // FP64 Chebyshev coefficients of degree kMaxDeg for every (orientation, L)
  struct Full {
    int o, L;
    std::vector<double> a;  // [(t * L + j) * K + n]
  };
  std::vector<Full> full;
  double hmax = 1.0;
  std::vector<double> tk(K);
  for (int k = 0; k < K; ++k) tk[k] = std::cos(kPi * (k + 0.5) / K);
  for (int o = 0; o < 2; ++o)
    for (int L : lengths[o]) {
      if (L < 2) continue;
      const double c = c_lat[o];
      std::vector<double> Lf;
      phi_matrix(L, c, Lf);
      if (!cholesky(L, Lf)) {
        err = "rbf: interpolation matrix not positive definite in FP64 (shape parameter too large)";
        return false;
      }
      Full F{o, L, std::vector<double>((size_t)(L - 1) * L * K)};
      std::vector<double> vals((size_t)K * L), h(L);
      for (int t = 0; t < L - 1; ++t) {
        for (int k = 0; k < K; ++k) {
          const double z = t + 0.5 * (tk[k] + 1.0);
          for (int i = 0; i < L; ++i) h[i] = imq(z - i, c);
          chol_solve(L, Lf, h.data());
          for (int j = 0; j < L; ++j) {
            vals[(size_t)k * L + j] = h[j];
            hmax = std::max(hmax, std::fabs(h[j]));
          }
        }
        for (int j = 0; j < L; ++j)
          for (int nn = 0; nn < K; ++nn) {
            double s = 0;
            for (int k = 0; k < K; ++k)
              s += vals[(size_t)k * L + j] * std::cos(kPi * nn * (k + 0.5) / K);
            F.a[((size_t)t * L + j) * K + nn] = (nn == 0 ? 1.0 : 2.0) * s / K;
          }
      }
      full.push_back(std::move(F));
    }
  // common degree: smallest candidate whose coefficient tail is small enough
  const int cands[] = {7, 11, 15, 19, 23};
  T.degree = kMaxDeg;
  for (int d : cands) {
    double worst = 0;
    for (const Full& F : full)
      for (size_t q = 0; q < F.a.size() / K; ++q) {
        double tail = 0;
        for (int nn = d + 1; nn < K; ++nn) tail += std::fabs(F.a[q * K + nn]);
        worst = std::max(worst, tail);
      }
    if (worst <= 2e-7 * hmax || d == kMaxDeg) {
      T.degree = d;
      T.max_err = worst;
      break;
    }
  }
  // device layout per table: [t][n][j] (interval, coefficient, stencil knot),
  // so that the lanes of a warp, one knot each, read consecutive words
  const int P1 = T.degree + 1;
  T.offset.assign(2 * (size_t)(T.lmax + 1), -1);
  T.coef.clear();
  for (const Full& F : full) {
    T.offset[(size_t)F.o * (T.lmax + 1) + F.L] = (int64_t)T.coef.size();
    for (int t = 0; t < F.L - 1; ++t)
      for (int nn = 0; nn < P1; ++nn)
        for (int j = 0; j < F.L; ++j)
          T.coef.push_back((float)F.a[((size_t)t * F.L + j) * K + nn]);
  }
  T.hmax = hmax;
  return true;
}

}  // namespace pdds
