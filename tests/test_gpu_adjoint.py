"""GPU discrete adjoint (hfe_adjoint and the torch.autograd.Function around it) against the
FP64 oracle's adjoint on the same seeded inverse problem: gradients to 1e-6 relative
(||dg|| / ||g||, and per component where |g_i| > 1e-3 max |g|), uniform and per-element
parameters, FP64 and mixed forward (the mixed forward ends each step with an FP64 Newton
iteration), history checkpointing with recompute (ckpt_every = 2) equal to full storage."""
import numpy as np
import pytest
import torch

from oracle import solver
from paper_2606_17390_b300 import hfe, inputs
from paper_2606_17390_b300.autograd import misfit

pytestmark = pytest.mark.gpu


def _problem(per_element=False, rotated=True):
    mesh = inputs.box_mesh(4, 2, 1, 4.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.08, 0.02, 0.0))
    mat = inputs.config1_material()
    if rotated:
        a = np.deg2rad(30.0)
        mat.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    th_true = mat.theta_vector()
    ts = inputs.load_factors(4)
    u_gt, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, th_true), ts, rtol=1e-13)
    rng = np.random.default_rng(4)
    u_gt = u_gt + 1e-3 * np.abs(u_gt).max() * rng.standard_normal(u_gt.shape)
    th = th_true * (1 + 0.1 * rng.uniform(-1, 1, 11))
    if per_element:
        th = th[None, :] * (1 + 0.05 * rng.uniform(-1, 1, (mesh.n_el, 11)))
    return mesh, bc, mat, ts, u_gt, th


@pytest.fixture(scope="module")
def oracle_uniform():
    mesh, bc, mat, ts, u_gt, th = _problem()
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    assert sum(i["plastic"] for i in infos) > 0
    g = solver.adjoint(prob, ts, us, hs, u_gt)
    return mesh, bc, mat, ts, u_gt, th, g, solver.objective(us, u_gt)


def _check(g, go, tol=1e-6):
    assert np.linalg.norm(g - go) < tol * np.linalg.norm(go), (g, go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    assert np.all(np.abs(g[big] - go[big]) < tol * np.abs(go[big]) + 1e-12 * np.abs(go).max()), (g, go)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_uniform_vs_oracle(oracle_uniform, precision):
    mesh, bc, mat, ts, u_gt, th, go, Jo = oracle_uniform
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, **opts) as s:
        J, g, st = s.adjoint(ts, u_gt)
    assert abs(J - Jo) < 1e-8 * Jo
    _check(g[0], go)
    # iteration counters: the reverse pass solves once per step; only the mixed forward
    # ends its steps with the FP64 refinement
    assert st["reverse_pcg_iters"] >= len(ts)
    assert (st["refine_pcg_iters"] > 0) == (precision == "mixed")
    assert st["pcg_iters"] >= st["reverse_pcg_iters"] + st["refine_pcg_iters"]


def test_adjoint_checkpoint_recompute_matches_full_storage(oracle_uniform):
    mesh, bc, mat, ts, u_gt, th, go, Jo = oracle_uniform
    out = []
    for k in (1, 2, 3):
        with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, ckpt_every=k, newton_rtol=1e-12,
                             pcg_rtol=1e-13) as s:
            out.append(s.adjoint(ts, u_gt)[1])
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_after_forward_repeats_a_fresh_handle(oracle_uniform, precision):
    """hfe_adjoint restarts from the zero state: after a forward (or another adjoint) on the
    same handle its forward pass starts like a fresh handle's - the extrapolated predictor
    does not reach back to the previous pass's solutions - so the results are bit-identical."""
    mesh, bc, mat, ts, u_gt, th, go, Jo = oracle_uniform
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, **opts) as s:
        J0, g0, st0 = s.adjoint(ts, u_gt)
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, **opts) as s:
        s.forward(ts)
        J1, g1, st1 = s.adjoint(ts, u_gt)
        J2, g2, st2 = s.adjoint(ts, u_gt)
    assert J1 == J0 and J2 == J0 and np.array_equal(g1, g0) and np.array_equal(g2, g0)
    assert st1["newton_iters"] == st0["newton_iters"] == st2["newton_iters"]


def test_adjoint_per_element_vs_oracle():
    mesh, bc, mat, ts, u_gt, th = _problem(per_element=True)
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    go = solver.adjoint(prob, ts, us, hs, u_gt, per_element=True)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, newton_rtol=1e-12, pcg_rtol=1e-13) as s:
        J, g, st = s.adjoint(ts, u_gt)
    assert g.shape == go.shape
    assert np.linalg.norm(g - go) < 1e-6 * np.linalg.norm(go)


def test_autograd_function(oracle_uniform):
    mesh, bc, mat, ts, u_gt, th, go, Jo = oracle_uniform
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, newton_rtol=1e-12, pcg_rtol=1e-13) as s:
        theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
        J = misfit(theta, s, ts, u_gt)
        (2.0 * J).backward()
    assert abs(J.item() - Jo) < 1e-8 * Jo
    _check(theta.grad.numpy() / 2.0, go)


def _config4_target(mesh, ts):
    """A seeded synthetic target field (no arithmetic of the method): a uniform stretch along
    x growing with the load factor plus noise."""
    rng = np.random.default_rng(3)
    u = np.stack([0.02 * mesh.X[:, 0], -0.003 * (mesh.X[:, 1] - 25.0), np.zeros(mesh.n_nodes)], 1).ravel()
    return np.stack([t * u + 1e-4 * rng.standard_normal(u.size) for t in ts])


def test_config4_remesh_per_element_vs_oracle():
    """Config 4's per-element F, G, H, sigma0 fields on the 40 x 20 x 2 re-mesh of the plate,
    evaluated at the spatially uniform mean parameters, three load steps of five: the GPU
    adjoint (FP64 and mixed forward) against the oracle's per-element adjoint."""
    mesh, bc, mat, th_true, ts = inputs.config4_problem(40, 20, 2, n_steps=5)
    ts = ts[:3]
    th = np.tile(mat.theta_vector(), (mesh.n_el, 1))
    u_gt = _config4_target(mesh, ts)
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    assert sum(i["plastic"] for i in infos) > 0
    go = solver.adjoint(prob, ts, us, hs, u_gt, per_element=True)
    for precision in ("fp64", "mixed"):
        opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
        with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, **opts) as s:
            J, g, st = s.adjoint(ts, u_gt)
        assert abs(J - solver.objective(us, u_gt)) < 1e-8 * J
        assert g.shape == go.shape
        assert np.linalg.norm(g - go) < 1e-6 * np.linalg.norm(go), (precision, np.linalg.norm(g - go) / np.linalg.norm(go))


def test_config4_reduced_directional_fd_and_checkpoints():
    """Config 4 on an 80 x 40 x 2 mesh of the plate (the true per-element fields perturbed
    by a seeded +-5 %): the adjoint gradient along a seeded random direction against central
    differences of J with the FP64 forward (relative step 1e-6), and checkpointing every 4
    steps equal bit for bit to storing every step (8 load steps)."""
    mesh, bc, mat, th_true, ts = inputs.config4_problem(80, 40, 2, n_steps=20)
    rng = np.random.default_rng(11)
    th = th_true * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, th_true.shape))
    u_gt = _config4_target(mesh, ts[:8])
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, **opts) as s:
        J, g, _ = s.adjoint(ts[:4], u_gt[:4])
    v = np.zeros_like(th)
    v[:, [2, 3, 4, 8]] = rng.standard_normal((mesh.n_el, 4))
    d = v * th
    h = 1e-6
    Jpm = []
    for sgn in (1.0, -1.0):
        with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th + sgn * h * d, **opts) as s:
            u, _ = s.forward(ts[:4])
        Jpm.append(float(np.sum((u - u_gt[:4]) ** 2)))
    fd = (Jpm[0] - Jpm[1]) / (2.0 * h)
    ad = float(np.sum(g * d))
    assert abs(fd - ad) < 1e-4 * abs(ad), (fd, ad)
    for precision in ("fp64", "mixed"):
        out = []
        for k in (1, 4):
            o = dict(opts) if precision == "fp64" else {}
            with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, ckpt_every=k, **o) as s:
                out.append(s.adjoint(ts[:8], u_gt)[1])
        assert np.array_equal(out[0], out[1]), precision


def test_adjoint_through_adaptive_substeps():
    """On the homogeneous config-0 problem (stretched to 25 %) J depends only on the
    displacements at the requested load factors, which do not depend on the substeps, so the
    discrete adjoint through whatever substeps adaptive stepping takes (newton_maxit = 3
    forces them) must equal the oracle's adjoint with plain steps."""
    mesh, _, mat, _ = inputs.config0_problem()
    bc = inputs.roller_uniaxial_bcs(mesh, 0.25, axis=0)
    ts = np.array([0.4, 1.0])
    th = mat.theta_vector() * (1 + 0.05 * np.random.default_rng(2).uniform(-1, 1, 11))
    th[0:2] = mat.theta_vector()[0:2]
    rng = np.random.default_rng(5)
    u_gt = 0.01 * rng.standard_normal((2, mesh.n_dof))
    prob = solver.from_inputs(mesh, bc, mat, th)
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    go = solver.adjoint(prob, ts, us, hs, u_gt)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, newton_rtol=1e-12, pcg_rtol=1e-13,
                         newton_maxit=3) as s:
        J, g, st = s.adjoint(ts, u_gt)
    assert st["cutbacks"] > 0
    assert abs(J - solver.objective(us, u_gt)) < 1e-9 * J
    _check(g[0], go)


def test_gradcheck_tool_on_the_gpu_path(oracle_uniform):
    """gradcheck.objective drives the GPU forward: its J equals hfe_adjoint's J, and the
    finite-difference check of the GPU adjoint gradient along D (relative steps) has its
    minimum below 1e-5 of g.D and a larger error at both ends of the step range."""
    from paper_2606_17390_b300 import gradcheck
    mesh, bc, mat, ts, u_gt, th, go, Jo = oracle_uniform
    idx = np.array([8, 9])
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, newton_rtol=1e-13, pcg_rtol=1e-14) as s:
        Ja, g, _ = s.adjoint(ts, u_gt)
        J = gradcheck.objective(s, ts, u_gt)
        assert abs(J(th) - Ja) <= 1e-12 * Ja
        res, ref = gradcheck.fd_check(J, g[0][idx], th, steps=gradcheck.PAPER_STEPS[::2], index=idx,
                                      scale=np.abs(th[idx]))
    E = np.array([r["E"] for r in res])
    k = int(E.argmin())
    assert E[k] < 1e-5 * abs(ref) and E[0] > E[k] and E[-1] > E[k], (E, ref)
