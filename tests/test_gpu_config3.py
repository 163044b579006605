"""Config 3's gradient check on config 3's own problem, reduced: the perforated plate at
24 x 12 x 2 (the same GRF recipe, correlation length scaled with the grid), Swift hardening,
all 20 load steps, the nine uniform parameters (F, G, H, L, M, N, K, eps0, n) at the seeded
+-20 % evaluation point, and the noisy target u_true + N(0, (1e-3 max|u|)^2) with u_true the
oracle's forward at the true parameters (Sec. 2.3, Eq. dR_u, Eq. main_grad, Algorithm
adjoint_ad; Algorithm finite_difference).

* The GPU adjoint (FP64 forward; mixed forward with the FP64 refinement of each step) against
  the oracle's FP64 adjoint: 1e-6 relative (norm, and per component above 1e-3 of the
  largest).
* The GPU FP64 adjoint against central differences of J with a relative step of 1e-6 per
  parameter (two GPU FP64 forwards each, Newton to 1e-12): compared as theta_i dJ/dtheta_i,
  1e-4 relative in norm (the differences carry ~1e-10 relative noise of J over 2e-6)."""
import numpy as np
import pytest

from oracle import solver
from paper_2606_17390_b300 import hfe, inputs

pytestmark = pytest.mark.gpu

NX, NY, NZ = 24, 12, 2
IDX = np.arange(2, 11)                     # F, G, H, L, M, N, K, eps0, n in theta's order
FP64 = dict(newton_rtol=1e-12, pcg_rtol=1e-13)


@pytest.fixture(scope="module")
def config3_oracle():
    mesh, bc, mat, ts = inputs.config3_problem(NX, NY, NZ)
    th_true = mat.theta_vector()
    u_true, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_true), ts, rtol=1e-13)
    u_gt = u_true + inputs.noise(u_true.shape, 1e-3 * np.abs(u_true).max())
    th = inputs.perturbed_theta(th_true)
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    assert 0 < infos[-1]["plastic"] < 8 * mesh.n_el
    g = solver.adjoint(prob, ts, us, hs, u_gt)
    return mesh, bc, mat, ts, u_gt, th, g, solver.objective(us, u_gt)


def _check(g, go, tol):
    assert np.linalg.norm(g - go) < tol * np.linalg.norm(go), (g, go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    assert np.all(np.abs(g[big] - go[big]) < tol * np.abs(go[big]) + 1e-12 * np.abs(go).max()), (g, go)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config3_gradient_vs_oracle_adjoint(config3_oracle, precision):
    mesh, bc, mat, ts, u_gt, th, go, Jo = config3_oracle
    opts = FP64 if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, **opts) as s:
        J, g, st = s.adjoint(ts, u_gt)
    assert abs(J - Jo) < 1e-8 * Jo
    _check(g[0][IDX], go[IDX], 1e-6)


def test_config3_gradient_vs_central_differences(config3_oracle):
    mesh, bc, mat, ts, u_gt, th, go, Jo = config3_oracle
    h = 1e-6
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, **FP64) as s:
        J, g, _ = s.adjoint(ts, u_gt)
        d_adj = th[IDX] * g[0][IDX]
        d_fd = np.empty(IDX.size)
        for k, i in enumerate(IDX):
            Jpm = []
            for sgn in (1.0, -1.0):
                tp = th.copy()
                tp[i] *= 1.0 + sgn * h
                s.set_material(tp, mat.Theta)
                s.set_state(None, None)
                u, _ = s.forward(ts)
                Jpm.append(float(np.sum((u - u_gt) ** 2)))
            d_fd[k] = (Jpm[0] - Jpm[1]) / (2.0 * h)
    assert np.linalg.norm(d_fd - d_adj) < 1e-4 * np.linalg.norm(d_adj), (d_fd, d_adj)
    big = np.abs(d_adj) > 1e-2 * np.abs(d_adj).max()
    assert np.all(np.abs(d_fd[big] - d_adj[big]) < 1e-3 * np.abs(d_adj[big])), (d_fd, d_adj)
