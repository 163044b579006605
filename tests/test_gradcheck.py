"""The finite-difference gradient check (Alg. finite_difference and E_FD,check of Sec. 3.2)
driven by the oracle's forward solve against the oracle's adjoint: the error against the
step size has the paper's V shape (truncation at large h, rounding and solver tolerance at
small h) and its minimum is at the adjoint-accuracy level."""
import dataclasses

import numpy as np

from oracle import solver
from paper_2606_17390_b300 import gradcheck
from tests.test_oracle_global import _tiny_inverse_problem


def test_fd_check_v_shape_against_oracle_adjoint():
    prob, ts, u_gt = _tiny_inverse_problem()
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    g = solver.adjoint(prob, ts, us, hs, u_gt)
    idx = np.array([8, 9])                                   # sigma0, Q (Voce)

    def J(theta):
        u, _, _ = solver.forward(dataclasses.replace(prob, theta=theta), ts, rtol=1e-13)
        return solver.objective(u, u_gt)

    steps = gradcheck.PAPER_STEPS[::2]                       # 1e-1, 1e-3, ..., 1e-11
    res, ref = gradcheck.fd_check(J, g[idx], prob.theta, steps=steps, index=idx, scale=np.abs(prob.theta[idx]))
    assert ref == gradcheck.PAPER_DIRECTION * g[idx].sum()
    E = np.array([r["E"] for r in res])
    k = int(E.argmin())
    assert E[k] < 1e-5 * abs(ref), (E, ref)
    assert 0 < k < len(E) - 1 and E[0] > 10 * E[k] and E[-1] > 10 * E[k], E


def test_fd_gradient_of_a_quadratic_is_exact():
    """J = 1/2 theta^T A theta + b^T theta: central differences are exact up to rounding for
    any h, and the check against the exact gradient is at rounding level."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((4, 4))
    A = A @ A.T
    b = rng.standard_normal(4)
    th = rng.standard_normal(4)

    def J(t):
        return 0.5 * t @ A @ t + b @ t

    g = A @ th + b
    assert np.allclose(gradcheck.fd_gradient(J, th, 1e-3), g, rtol=0, atol=1e-9)
    res, ref = gradcheck.fd_check(J, g, th, steps=(1e-1, 1e-2, 1e-3))
    assert all(r["E"] < 1e-10 for r in res)
