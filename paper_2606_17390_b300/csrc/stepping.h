// Host-side arithmetic of the load-step predictor (internal; no CUDA).
#pragma once

#include <algorithm>
#include <cmath>

namespace hfe {

// Extrapolated predictor (Sec. 2.2, automatic time stepping): the Lagrange weights at the
// load factor t_new of the stored converged solutions t_hist[0] (newest), t_hist[1], ...;
// up to min(n_stored, max_order) points are used (max_order 2: linear, 3: quadratic), and
// points closer than 1e-12 in the load factor lower the order.  Returns the number of points
// used: 1 means no extrapolation (w = {1, 0, 0}).
inline int extrapolation_weights(const double* t_hist, int n_stored, int max_order, double t_new, double w[3]) {
  int k = std::min(std::min(n_stored, max_order), 3);
  auto close = [](double a, double b) { return std::fabs(a - b) <= 1e-12 * std::max(1.0, std::fabs(a)); };
  if (k == 3 && (close(t_hist[0], t_hist[2]) || close(t_hist[1], t_hist[2]))) k = 2;
  if (k >= 2 && close(t_hist[0], t_hist[1])) k = 1;
  if (k < 1) k = 1;
  w[0] = 1.0;
  w[1] = w[2] = 0.0;
  if (k == 1) return 1;
  for (int i = 0; i < k; ++i) {
    double l = 1.0;
    for (int j = 0; j < k; ++j)
      if (j != i) l *= (t_new - t_hist[j]) / (t_hist[i] - t_hist[j]);
    w[i] = l;
  }
  return k;
}

}  // namespace hfe
