"""Inverse identification (L-BFGS-B over normalised parameters, the paper's Sec. 4 set-up):
the normalisation round trip and its worked initial value (CPU), and recovery of Voce
hardening parameters from a noiseless target on a small box (GPU)."""
import numpy as np
import pytest

from paper_2606_17390_b300 import inverse


def test_normalisation_round_trip_and_paper_initial_guess():
    # Sec. 4 (C1): theta_min = [140, 300, 3, 0.9, 0.9, 0.9], theta_ref = [40, 300, 2, 0.8, 0.8,
    # 0.8], rho_i = 0.2 -> theta = (rho + 1) theta_ref / 2 + theta_min
    tmin = np.array([140.0, 300.0, 3.0, 0.9, 0.9, 0.9])
    tref = np.array([40.0, 300.0, 2.0, 0.8, 0.8, 0.8])
    th = inverse.denormalize(np.full(6, 0.2), tmin, tref)
    assert np.allclose(th, [164.0, 480.0, 4.2, 1.38, 1.38, 1.38], rtol=0, atol=1e-12)
    assert np.allclose(inverse.normalize(th, tmin, tref), 0.2, rtol=0, atol=1e-14)
    assert np.allclose(inverse.denormalize(-1.0, tmin, tref), tmin)
    assert np.allclose(inverse.denormalize(1.0, tmin, tref), tmin + tref)


def test_warm_start_rule():
    # Sec. 3.6: the previous pass is reused when every parameter moved by less than 10 %
    prev = np.array([150.0, 120.0, 12.0, 0.0])
    assert not inverse.warm_start_applies(prev, None)
    assert inverse.warm_start_applies(prev, prev)
    assert inverse.warm_start_applies(prev * [1.09, 0.92, 1.0, 1.0], prev)
    assert not inverse.warm_start_applies(prev * [1.1, 1.0, 1.0, 1.0], prev)      # exactly 10 %
    assert not inverse.warm_start_applies(prev * [1.0, 1.0, 0.85, 1.0], prev)
    assert not inverse.warm_start_applies(prev + [0.0, 0.0, 0.0, 1e-9], prev)     # from 0
    assert inverse.warm_start_applies(np.full((3, 2), 1.05), np.ones((3, 2)))    # per element


@pytest.mark.gpu
def test_identify_voce_parameters_noiseless():
    from oracle import solver
    from paper_2606_17390_b300 import hfe, inputs
    mesh = inputs.box_mesh(4, 2, 1, 4.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.12, 0.02, 0.0))
    mat = inputs.config1_material()
    th_true = mat.theta_vector()
    ts = inputs.load_factors(4)
    u_gt, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_true), ts, rtol=1e-13)
    idx = np.array([8, 9, 10])                      # sigma0, Q, b
    tmin, tref = 0.5 * th_true[idx], th_true[idx]   # bounds theta_true x [0.5, 1.5]
    th0 = th_true.copy()
    th0[idx] = inverse.denormalize(np.full(3, 0.2), tmin, tref)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th0, newton_rtol=1e-12, pcg_rtol=1e-13) as s:
        # w scales J(theta0) to O(1): the L-BFGS-B stopping tests are absolute below |J| = 1
        res = inverse.identify(s, ts, u_gt, th0, idx, tmin, tref, w=1e6)
    assert res.J < 1e-8 * res.history[0][0], (res.J, res.history[0][0], res.message)
    assert np.allclose(res.theta[idx], th_true[idx], rtol=1e-4), (res.theta[idx], th_true[idx], res.message)
