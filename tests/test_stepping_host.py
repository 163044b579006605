"""The extrapolated predictor's weights (csrc/stepping.h, compiled here by the host C++
compiler without CUDA): Lagrange weights through the newest 2 or 3 stored load factors
reproduce every polynomial of degree below the number of points used (so a solution linear
or quadratic in the load factor is predicted exactly), fewer stored solutions or points
closer than 1e-12 lower the order, and one point gives no extrapolation."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_17390_b300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "stepping.h"
int main(int argc, char** argv) {
  double t[3] = {atof(argv[1]), atof(argv[2]), atof(argv[3])};
  double w[3];
  int k = hfe::extrapolation_weights(t, atoi(argv[4]), atoi(argv[5]), atof(argv[6]), w);
  printf("%d %.17g %.17g %.17g\n", k, w[0], w[1], w[2]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def weights(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("stepping")
    (d / "driver.cpp").write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(d / "driver.cpp"), "-o", str(exe)], check=True)

    def f(t_hist, n_stored, max_order, t_new):
        t = list(t_hist) + [0.0] * (3 - len(t_hist))
        out = subprocess.run([str(exe)] + [repr(float(x)) for x in t] + [str(n_stored), str(max_order), repr(t_new)],
                             check=True, capture_output=True, text=True).stdout.split()
        return int(out[0]), np.array([float(x) for x in out[1:]])
    return f


@pytest.mark.parametrize("t_hist,t_new", [((0.5, 0.4, 0.3), 0.6), ((1.0, 0.75, 0.25), 1.1),
                                          ((0.6, 1.0, 0.5), 0.3)])   # the last: unloading after a reversal
def test_polynomials_reproduced(weights, t_hist, t_new):
    th = np.array(t_hist)
    for max_order, degree in ((2, 1), (3, 2)):
        k, w = weights(th, 3, max_order, t_new)
        assert k == max_order and abs(w.sum() - 1.0) < 1e-14
        rng = np.random.default_rng(degree)
        for _ in range(3):
            c = rng.standard_normal(degree + 1)
            p = np.polynomial.polynomial.polyval
            assert abs(w[:k] @ p(th[:k], c) - p(t_new, c)) < 1e-12 * (1 + abs(p(t_new, c)))


def test_order_lowered_by_history_and_close_points(weights):
    assert weights((0.5, 0.4, 0.3), 1, 3, 0.6) == (1, pytest.approx([1.0, 0.0, 0.0]))   # only the state
    k, w = weights((0.5, 0.4, 0.3), 2, 3, 0.6)                                         # two stored: linear
    assert k == 2 and w == pytest.approx([2.0, -1.0, 0.0])
    k, w = weights((0.5, 0.4, 0.4 + 1e-14), 3, 3, 0.6)                                  # third point too close
    assert k == 2
    k, w = weights((0.5, 0.5 + 1e-14, 0.3), 3, 3, 0.6)                                  # two newest coincide
    assert k == 1 and w == pytest.approx([1.0, 0.0, 0.0])
