// Host-side dense linear algebra shared by the C-ABI front ends (dqmc_api.cu,
// dqmc_su2_api.cu): the symmetric eigendecomposition of the hopping matrix and
// the exponentials exp(t K) built from it (Sec. 3.1, Op_set).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace dqmc {
namespace host {

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition A = V diag(w) V^T (host, FP64): Jacobi
// rotations with the classical threshold strategy (Rutishauser), sweeping the
// upper triangle until every off-diagonal element is below the threshold.
// ---------------------------------------------------------------------------
inline void symmetric_eigen(int n, const std::vector<double>& A_in, std::vector<double>& w, std::vector<double>& V) {
  std::vector<double> a(A_in);
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
  double scale = 0.0;
  for (double x : a) scale = std::max(scale, std::fabs(x));
  if (scale == 0.0) scale = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(at(i, j)));
    if (off <= 1e-17 * scale) break;
    const double thresh = (sweep < 4) ? 0.2 * off : 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(p, q);
        if (std::fabs(apq) <= thresh || apq == 0.0) continue;
        // tangent t of the rotation angle that annihilates a_pq: the smaller
        // root of t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq)
        const double theta = 0.5 * (at(q, q) - at(p, p)) / apq;
        double t;
        if (std::fabs(theta) > 1e150) {
          t = 0.5 / theta;
        } else {
          t = 1.0 / (std::fabs(theta) + std::sqrt(1.0 + theta * theta));
          if (theta < 0.0) t = -t;
        }
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < n; ++k) {
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double& vkp = V[(size_t)k * n + p];
          double& vkq = V[(size_t)k * n + q];
          const double x = vkp, y = vkq;
          vkp = c * x - s * y;
          vkq = s * x + c * y;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = at(i, i);
}

// exp(t K) through the eigendecomposition of K.
inline std::vector<double> expm_symmetric(int n, const std::vector<double>& w, const std::vector<double>& V, double t) {
  std::vector<double> E((size_t)n * n, 0.0);
  std::vector<double> ex(n);
  for (int k = 0; k < n; ++k) ex[k] = std::exp(t * w[k]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += V[(size_t)i * n + k] * ex[k] * V[(size_t)j * n + k];
      E[(size_t)i * n + j] = acc;
    }
  return E;
}

}  // namespace host
}  // namespace dqmc
