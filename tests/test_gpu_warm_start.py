"""Warm start of the load steps (hfe_set_warm_start, Sec. 3.6): a pass started from the record
of a pass at the same parameters reproduces it bit for bit without a Newton correction; a pass
started from the record of nearby parameters converges to the oracle's forward at the new
parameters (FP64 1e-10, mixed 1e-5 relative in displacement) and its adjoint gradient to the
oracle's (1e-6); record slots of other load factors are not used; the inverse loop with the
10 % rule recovers the same parameters as without it."""
import numpy as np
import pytest

from oracle import solver
from paper_2606_17390_b300 import hfe, inputs, inverse

pytestmark = pytest.mark.gpu

FP64 = dict(newton_rtol=1e-12, pcg_rtol=1e-13)
TOL_U = {"fp64": 1e-10, "mixed": 1e-5}


def _problem():
    """A clamped 4x2x1 box pulled along x and y, config 1's Voce material rotated by 30 degrees
    about z, four load steps (plastic from the second)."""
    mesh = inputs.box_mesh(4, 2, 1, 4.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.08, 0.02, 0.0))
    mat = inputs.config1_material()
    a = np.deg2rad(30.0)
    mat.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    return mesh, bc, mat, inputs.load_factors(4)


def _perturbed(th, rel, seed):
    rng = np.random.default_rng(seed)
    return th * (1 + rel * rng.uniform(-1, 1, th.size))


def _axes(mat):
    return np.asarray(mat.Theta, dtype=np.float64)


def test_same_parameters_bit_identical_without_newton_corrections():
    mesh, bc, mat, ts = _problem()
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", **FP64) as s:
        s.set_warm_start("record")
        u0, st0 = s.forward(ts)
        assert st0["warm_steps"] == 0 and st0["newton_iters"] > 0 and st0["plastic_gps"] > 0
        s.set_warm_start("use")
        s.set_state(None, None)
        u1, st1 = s.forward(ts)
    assert st1["warm_steps"] == len(ts) and st1["warm_retries"] == 0
    assert st1["newton_iters"] == 0 and st1["pcg_iters"] == 0
    assert np.array_equal(u0, u1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nearby_parameters_match_oracle(precision):
    mesh, bc, mat, ts = _problem()
    th_a = mat.theta_vector()
    th_b = _perturbed(th_a, 0.05, 11)
    us, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_b), ts, rtol=1e-13)
    opts = FP64 if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th_a, **opts) as s:
        s.set_warm_start("record")
        s.forward(ts)
        s.set_material(th_b, _axes(mat))
        s.set_state(None, None)
        s.set_warm_start("use")
        u, st = s.forward(ts)
    assert st["warm_steps"] == len(ts) and st["warm_retries"] == 0
    for n in range(len(ts)):
        assert np.abs(u[n] - us[n]).max() < TOL_U[precision] * np.abs(us[n]).max(), n


def test_small_change_takes_no_more_newton_iterations_than_cold():
    """Late in an inverse loop the parameters move little: from the record of a pass at
    parameters 1e-3 away the warm pass needs at most the cold pass's Newton iterations."""
    mesh, bc, mat, ts = _problem()
    th_a = mat.theta_vector()
    th_b = _perturbed(th_a, 1e-3, 12)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th_a, **FP64) as s:
        s.set_warm_start("record")
        s.forward(ts)
        s.set_material(th_b, _axes(mat))
        s.set_state(None, None)
        s.set_warm_start("use")
        uw, stw = s.forward(ts)
        s.set_warm_start("off")
        s.set_state(None, None)
        uc, stc = s.forward(ts)
    assert stw["warm_steps"] == len(ts) and stc["warm_steps"] == 0
    assert stw["newton_iters"] <= stc["newton_iters"], (stw["newton_iters"], stc["newton_iters"])
    assert np.abs(uw - uc).max() < 1e-10 * np.abs(uc).max()


def test_other_load_factors_start_cold():
    mesh, bc, mat, ts = _problem()
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", **FP64) as s:
        s.set_warm_start("record")
        s.forward(ts)                         # slots at 0.25, 0.5, 0.75, 1.0
        s.set_warm_start("use")
        s.set_state(None, None)
        t2 = inputs.load_factors(2)           # 0.5, 1.0 at slots 0 and 1
        u2, st2 = s.forward(t2)
        s.set_warm_start("off")
        s.set_state(None, None)
        u2c, st2c = s.forward(t2)
        s.set_warm_start("use")               # the record was freed: nothing to start from
        s.set_state(None, None)
        _, st3 = s.forward(t2)
    assert st2["warm_steps"] == 0 and st3["warm_steps"] == 0
    assert np.array_equal(u2, u2c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_from_warm_start_matches_oracle(precision):
    mesh, bc, mat, ts = _problem()
    th_true = mat.theta_vector()
    u_gt, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_true), ts, rtol=1e-13)
    rng = np.random.default_rng(4)
    u_gt = u_gt + 1e-3 * np.abs(u_gt).max() * rng.standard_normal(u_gt.shape)
    th = _perturbed(th_true, 0.1, 5)
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    go, Jo = solver.adjoint(prob, ts, us, hs, u_gt), solver.objective(us, u_gt)
    opts = FP64 if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=_perturbed(th, 0.05, 6), **opts) as s:
        s.set_warm_start("record")
        s.adjoint(ts, u_gt)
        s.set_material(th, _axes(mat))
        s.set_warm_start("use")
        J, g, st = s.adjoint(ts, u_gt)
    assert st["warm_steps"] == len(ts)
    assert abs(J - Jo) < 1e-8 * Jo
    g = g[0]
    assert np.linalg.norm(g - go) < 1e-6 * np.linalg.norm(go), (g, go)


def test_identify_with_warm_start():
    from paper_2606_17390_b300.inverse import denormalize
    mesh = inputs.box_mesh(4, 2, 1, 4.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.12, 0.02, 0.0))
    mat = inputs.config1_material()
    th_true = mat.theta_vector()
    ts = inputs.load_factors(4)
    u_gt, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_true), ts, rtol=1e-13)
    idx = np.array([8, 9, 10])
    tmin, tref = 0.5 * th_true[idx], th_true[idx]
    th0 = th_true.copy()
    th0[idx] = denormalize(np.full(3, 0.2), tmin, tref)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th0, **FP64) as s:
        res = inverse.identify(s, ts, u_gt, th0, idx, tmin, tref, w=1e6, warm_start=True)
    assert res.warm_passes > 0
    assert res.J < 1e-8 * res.history[0][0], (res.J, res.message)
    assert np.allclose(res.theta[idx], th_true[idx], rtol=1e-4), (res.theta[idx], res.message)


def test_record_grows_and_keeps_its_slots():
    """A longer pass grows the record (reallocated, the recorded slots copied over): after a
    2-step pass to (0.5, 1.0) a 4-step pass to (0.5, 1.0, 1.25, 1.5) starts its first two steps
    from the slots recorded before the growth - converged at their first sweep, bit-identical
    to the 2-step pass - and the last two cold; a repeat of the 4-step pass starts warm at
    every step and repeats it bit for bit."""
    mesh, bc, mat, _ = _problem()
    t2, t4 = np.array([0.5, 1.0]), np.array([0.5, 1.0, 1.25, 1.5])
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", **FP64) as s:
        s.set_warm_start("use")
        u2, st_a = s.forward(t2)
        s.set_state(None, None)
        u4, st_b = s.forward(t4)
        s.set_state(None, None)
        u4w, st_c = s.forward(t4)
    assert st_a["warm_steps"] == 0 and st_b["warm_steps"] == 2 and st_b["warm_retries"] == 0
    assert np.array_equal(u4[:2], u2)
    assert st_c["warm_steps"] == 4 and st_c["newton_iters"] == 0
    assert np.array_equal(u4w, u4)
