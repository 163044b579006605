"""Full forward solves on the GPU (load steps, global Newton, block-CSR assembly, PCG) vs the
FP64 oracle on the same seeded inputs.  Tolerances: FP64 path 1e-10 relative in displacement
(max over dofs / max |u| per step); mixed path 1e-5 in displacement and 1e-4 in von Mises
stress (max |dvm| / max vm)."""
import numpy as np
import pytest

from oracle import material, solver
from paper_2606_17390_b300 import hfe, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def config0_oracle():
    mesh, bc, mat, ts = inputs.config0_problem()
    prob = solver.from_inputs(mesh, bc, mat)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-12)
    return mesh, bc, mat, ts, us, hs, infos


@pytest.fixture(scope="module")
def plate_oracle():
    mesh, bc, mat, ts = inputs.config1_problem(nx=24, ny=12, nz=2, n_steps=6)
    prob = solver.from_inputs(mesh, bc, mat)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-12)
    return mesh, bc, mat, ts, us, hs, infos


def _per_step_rel(u, uo):
    return max(np.abs(u[n] - uo[n]).max() / np.abs(uo[n]).max() for n in range(len(uo)))


def _vm_rel(sig, sig_o):
    vm = material.von_mises(sig.reshape(-1, 3, 3) if sig.ndim == 3 else _sym(sig))
    vmo = material.von_mises(sig_o.reshape(-1, 3, 3))
    return np.abs(vm - vmo).max() / vmo.max()


def _sym(s6):
    return material.sym(s6)


# initial guess of each step: 1 tangent predictor, 0 previous displacement, 2 (default) / 3
# linear / quadratic extrapolation through the last converged steps
PREDICTORS = [1, 0, 2, 3]


@pytest.mark.parametrize("predictor", PREDICTORS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config0_forward(config0_oracle, precision, predictor):
    mesh, bc, mat, ts, uo, ho, infos = config0_oracle
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, predictor=predictor, **opts) as s:
        sig = np.empty((mesh.n_el * 8, 6))
        hist = np.empty((7, mesh.n_el * 8))
        u, st = s.forward(ts, sigma_out=sig, hist_out=hist)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert _per_step_rel(u, uo) < tol
    assert _vm_rel(sig, infos[-1]["sigma"]) < (1e-10 if precision == "fp64" else 1e-4)
    assert np.abs(hist[6] - ho[-1][..., 6].ravel()).max() < (1e-12 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("predictor", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plate_forward(plate_oracle, precision, predictor):
    mesh, bc, mat, ts, uo, ho, infos = plate_oracle
    assert 0 < infos[-1]["plastic"] < 8 * mesh.n_el      # heterogeneous elastic/plastic mix
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, predictor=predictor, **opts) as s:
        sig = np.empty((mesh.n_el * 8, 6))
        u, st = s.forward(ts, sigma_out=sig)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert _per_step_rel(u, uo) < tol, _per_step_rel(u, uo)
    assert _vm_rel(sig, infos[-1]["sigma"]) < (1e-9 if precision == "fp64" else 1e-4)


def test_spmv_and_solve_consistent():
    """SpMV with symmetric Dirichlet elimination against scipy on the exported block-CSR
    matrix (perforated plate), and PCG solves with the elastic tangent (u = 0, positive
    definite) on a clamped cube; the mixed solve's true residual is bounded by the FP32
    matrix (kappa * eps_32), so its bound is looser."""
    from tests._helpers import bsr_to_csr
    plate = inputs.config1_problem(nx=16, ny=8, nz=2, n_steps=4)
    cube = inputs.config2_problem(n=6)
    for (mesh, bc, mat, ts), check_solve in ((plate, False), (cube, True)):
        for precision, tol_mv, tol_x in (("fp64", 1e-12, 1e-10), ("mixed", 1e-6, 1e-4)):
            with hfe.from_inputs(mesh, bc, mat, precision=precision) as s:
                s.sweep(np.zeros(mesh.n_dof), 0.0)
                rowptr, cols, vals = s.get_bsr()
                K = bsr_to_csr(rowptr, cols, vals, mesh.n_nodes)
                free = np.ones(mesh.n_dof, bool)
                free[bc.dof] = False
                x = np.random.default_rng(0).standard_normal(mesh.n_dof)
                y = s.spmv(x)
                xm = np.where(free, x, 0.0)
                y_ref = np.where(free, K @ xm, x)
                assert np.abs(y - y_ref).max() < tol_mv * np.abs(y_ref).max()
                if not check_solve:
                    continue
                b = np.where(free, np.random.default_rng(1).standard_normal(mesh.n_dof), 0.0)
                dx, st = s.solve(b)
                assert st["pcg_iters"] > 0
                res = np.where(free, K @ np.where(free, dx, 0.0), 0.0) - b
                assert np.linalg.norm(res) < tol_x * np.linalg.norm(b)
                assert np.all(dx[~free] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_and_chunked_cg_agree(precision):
    """The one-launch CG (grid barriers) and the chunked CG (CUDA-graph chunks, host checks)
    run the same iteration: elastic solves on a clamped cube at 40^3 (the FP64 matrix, 141 MB,
    takes the HBM-streaming register budget, the FP32 one the L2-resident one) and a
    three-step forward on a reduced perforated plate."""
    cube = inputs.config2_problem(n=40)
    mesh, bc, mat, _ = cube
    b = np.random.default_rng(1).standard_normal(mesh.n_dof)
    b[bc.dof] = 0.0
    xs, its = [], []
    for pers in (1, 0):
        with hfe.from_inputs(mesh, bc, mat, precision=precision, pcg_persistent=pers) as s:
            s.sweep(np.zeros(mesh.n_dof), 0.0)
            x, st = s.solve(b)
        xs.append(x)
        its.append(st["pcg_iters"])
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.abs(xs[0] - xs[1]).max() <= tol * np.abs(xs[1]).max()
    assert abs(its[0] - its[1]) <= max(2, its[1] // 50), its
    mesh, bc, mat, ts = inputs.config1_problem(nx=16, ny=8, nz=2, n_steps=20)
    us = []
    for pers in (1, 0):
        with hfe.from_inputs(mesh, bc, mat, precision=precision, pcg_persistent=pers) as s:
            u, _ = s.forward(ts[:3])
        us.append(u)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert _per_step_rel(us[0], us[1]) < tol


def test_adaptive_stepping_closed_form_and_restore():
    """Adaptive load stepping: on the homogeneous config-0 problem (here stretched to 25 %)
    the solution at the requested load factors is the uniaxial closed form whatever substeps
    are taken, so two requested steps (10 %, 25 %) with newton_maxit = 3, which forces
    rejected attempts and substeps, must still match it to 1e-10 (FP64); without adaptive
    stepping the same run fails and leaves the stored state at the last converged step."""
    from tests.test_oracle_global import _uniaxial_closed_form
    mesh, _, mat, _ = inputs.config0_problem()
    bc = inputs.roller_uniaxial_bcs(mesh, 0.25, axis=0)
    ts = np.array([0.4, 1.0])
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13, newton_maxit=3)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", **opts) as s:
        u, st = s.forward(ts)
    assert st["cutbacks"] > 0 and st["substeps"] > 2, st
    for k, t in enumerate(ts):
        uex = _uniaxial_closed_form(5.0 * t, mesh)[0]      # closed form written for 0.05 t
        assert np.abs(u[k] - uex).max() < 1e-10 * np.abs(uex).max()
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", adaptive=0, **opts) as s:
        u1, _ = s.forward(np.array([0.001]))       # a small elastic first step converges
        with pytest.raises(hfe.HfeError):
            s.forward(ts[1:])
        u_after, _ = s.get_state()
        assert s.get_load() == pytest.approx(0.001)
    assert np.array_equal(u_after, u1[0])


def test_adaptive_stepping_plate_in_few_steps():
    """The perforated plate at 100 x 50 x 2 in 10 requested steps: without adaptive stepping
    the second step fails; with it the run completes through substeps and the final state is
    in equilibrium (residual of the committed state below the Newton tolerance)."""
    mesh, bc, mat, ts = inputs.config3_problem(100, 50, 2, n_steps=10)
    with hfe.from_inputs(mesh, bc, mat, precision="mixed") as s:
        u, st = s.forward(ts)
        assert st["steps_done"] == 10 and st["substeps"] >= 10
        rn = np.empty(1)
        s.sweep(u[-1], 1.0, tangent=False, rnorm_out=rn)
    assert np.isfinite(u).all()
    # out-of-balance force of the committed state: Newton-tolerance level, against
    # reaction forces of order E * 2 % * 100 mm^2 = 1.4e5 N
    assert rn[0] < 1.0, rn


@pytest.mark.parametrize("predictor", PREDICTORS)
def test_unloading_step_matches_oracle(predictor):
    """Load factors need not increase: tension to 5 %, then back to 3 % (beyond the elastic
    range 2 sigma_y / E, so the unloading yields in reverse), against the oracle's forward on
    the same factors (FP64 1e-10); the extrapolations then point the wrong way at the reversal."""
    mesh, bc, mat, _ = inputs.config0_problem(n=2)
    ts = np.array([0.5, 1.0, 0.6])
    us, hs, _ = solver.forward(solver.from_inputs(mesh, bc, mat), ts, rtol=1e-13)
    assert np.abs(hs[3][..., 6] - hs[2][..., 6]).max() > 0.0           # reverse plastic flow
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", newton_rtol=1e-12, pcg_rtol=1e-13,
                         predictor=predictor) as s:
        u, st = s.forward(ts)
    assert _per_step_rel(u, us) < 1e-10


def test_extrapolation_history_restarts_after_set_state():
    """Quadratic extrapolation over two passes of the same loading on one handle: the second
    pass (after hfe_set_state) starts from the stored state alone, so it repeats the first
    bit for bit; options.predictor outside 0-3 is refused at hfe_create."""
    mesh, bc, mat, ts = inputs.config0_problem(n=3, n_steps=5)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", predictor=3) as s:
        u1, st1 = s.forward(ts)
        s.set_state(None, None)
        u2, st2 = s.forward(ts)
    assert np.array_equal(u1, u2) and st1["newton_iters"] == st2["newton_iters"]
    with pytest.raises(hfe.HfeError):
        hfe.from_inputs(mesh, bc, mat, precision="fp64", predictor=4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_voce_homogeneous_closed_form(precision):
    """Voce hardening through the whole GPU forward: the config-0 cube with roller BCs and
    config 1's Voce material (sigma0 = 150, Q = 120, b = 12), 10 steps to 5 %, against the
    uniaxial closed form eps11 = sigma_y(alpha)/E + alpha (Eq. Hard, reading R1), which the
    test writes out itself: FP64 1e-10, mixed 1e-5 in displacement; alpha 1e-12 / 1e-6."""
    from tests.test_oracle_global import _uniaxial_closed_form, config0_voce_problem
    mesh, bc, mat, ts = config0_voce_problem()
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, **opts) as s:
        hist = np.empty((7, mesh.n_el * 8))
        u, st = s.forward(ts, hist_out=hist)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for k, t in enumerate(ts):
        uex = _uniaxial_closed_form(t, mesh, "voce")[0]
        assert np.abs(u[k] - uex).max() < tol * np.abs(uex).max(), (k, precision)
    a = _uniaxial_closed_form(ts[-1], mesh, "voce")[1]
    assert np.abs(hist[6] - a).max() < (1e-12 if precision == "fp64" else 1e-6) * max(a, 1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plate_50x25x2_all_steps_vs_stored_oracle(precision):
    """The perforated plate at 50 x 25 x 2 over all 20 Voce load steps against the oracle's
    forward solve stored by tests/golden/make_plate_forward_50x25x2.py (per step: u at 600
    seeded dofs and max |u|; after the last step von Mises at 1,000 seeded Gauss points and
    the maximum).  FP64 1e-10 in displacement, mixed 1e-5 in displacement and 1e-4 in von
    Mises stress, relative to the step's maximum."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "plate_forward_50x25x2.npz"))
    mesh, bc, mat, ts = inputs.config1_problem(nx=50, ny=25, nz=2, n_steps=20)
    assert mesh.n_el == int(g["n_el"]) and mesh.n_dof == int(g["n_dof"])
    assert np.array_equal(np.asarray(ts), g["ts"])
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, **opts) as s:
        sig = np.empty((mesh.n_el * 8, 6))
        u, st = s.forward(ts, sigma_out=sig)
    assert st["steps_done"] == 20
    err_u = max(np.abs(u[n][g["dofs"]] - g["u_sample"][n]).max() / g["u_max"][n] for n in range(20))
    err_umax = np.abs(np.abs(u).max(axis=1) - g["u_max"]).max() / g["u_max"].max()
    vm = material.von_mises(_sym(sig))
    err_vm = max(np.abs(vm[g["gps"]] - g["vm_sample"]).max(), abs(vm.max() - float(g["vm_max"]))) / float(g["vm_max"])
    tol_u = 1e-10 if precision == "fp64" else 1e-5
    assert err_u < tol_u and err_umax < tol_u, (err_u, err_umax)
    assert err_vm < (1e-9 if precision == "fp64" else 1e-4), err_vm
