"""The oracle's discrete adjoint with the Barlat Yld2004-18p model (App. D applied to the
8-unknown closest-point projection, parameters c' (9), c'' (9), E, nu and the hardening
parameters): the parameter columns of the local update against central differences of the
update (elastic and plastic points), and the global gradient against the direct
(forward-mode) sensitivity and against central differences of the misfit over the oracle's
forward solve, on a rotated anisotropic box with elastic, mixed and plastic load steps."""
import numpy as np
import pytest

from oracle import barlat as BA
from oracle import solver
from paper_2606_17390_b300 import inputs

A30 = np.deg2rad(30.0)
THETA = np.array([[np.cos(A30), -np.sin(A30), 0], [np.sin(A30), np.cos(A30), 0], [0, 0, 1.0]])


def _q0():
    m = inputs.barlat_verification_material()
    th = inputs.config0_material().theta_vector()
    model = BA.Barlat(m.c1, m.c2, m.m, THETA)
    return BA.params(model, th[0], th[1], (th[8], th[9], th[10])), m.m


def _local(q, m):
    model, E, nu, h = BA.unpack(q, m, THETA)
    return BA.local(model, E, nu, "swift", h)


def test_parameter_columns_vs_central_differences():
    q, m = _q0()
    rng = np.random.default_rng(2)
    eps = rng.standard_normal((12, 6)) * 0.003 * np.linspace(0.05, 1.5, 12)[:, None]   # elastic to plastic
    epn = rng.standard_normal((12, 6)) * 4e-4
    epn[:, :3] -= epn[:, :3].mean(axis=1, keepdims=True)          # plastic strain deviatoric
    alpn = rng.uniform(0, 0.01, 12)
    out = _local(q, m)(eps, epn, alpn, derivatives=True, param_derivatives=True)
    assert out["plastic"].any() and (~out["plastic"]).any() and out["converged"].all()
    dz = out["dz"][:, :, 13:]
    assert dz.shape == (12, 13, BA.N_PARAMS)
    for j in range(BA.N_PARAMS):
        hj = 1e-6 * max(abs(q[j]), 1e-2)
        qp, qm = q.copy(), q.copy()
        qp[j] += hj
        qm[j] -= hj
        zp = _local(qp, m)(eps, epn, alpn, derivatives=False)["z"]
        zm = _local(qm, m)(eps, epn, alpn, derivatives=False)["z"]
        fd = (zp - zm) / (2 * hj)
        scale = np.abs(fd).max() + np.abs(dz[:, :, j]).max() + 1e-30
        assert np.abs(fd - dz[:, :, j]).max() < 2e-5 * scale, j


@pytest.fixture(scope="module")
def barlat_inverse_problem():
    q, m = _q0()
    mesh = inputs.box_mesh(3, 2, 1, 3.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.012, 0.004, 0.0))
    mat = inputs.config1_material()
    ts = inputs.load_factors(3)

    def prob_of(qq):
        p = solver.from_inputs(mesh, bc, mat)
        p.local = _local(qq, m)
        return p
    u_gt, _, _ = solver.forward(prob_of(q), ts, rtol=1e-13)
    rng = np.random.default_rng(4)
    u_gt = u_gt + 1e-3 * np.abs(u_gt).max() * rng.standard_normal(u_gt.shape)
    q_eval = q * (1 + 0.03 * rng.uniform(-1, 1, q.size))
    return prob_of, q_eval, ts, u_gt, mesh


def test_barlat_adjoint_equals_direct_and_fd(barlat_inverse_problem):
    prob_of, q_eval, ts, u_gt, mesh = barlat_inverse_problem
    P = prob_of(q_eval)
    us, hs, infos = solver.forward(P, ts, rtol=1e-13)
    plastic = [i["plastic"] for i in infos]
    assert plastic[0] < 8 * mesh.n_el and plastic[-1] > 0       # elastic points and plastic ones
    g = solver.adjoint(P, ts, us, hs, u_gt)
    assert g.shape == (BA.N_PARAMS,)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(BA.N_PARAMS) * np.abs(q_eval)
    d_dir = solver.direct_sensitivity(P, ts, us, hs, u_gt, v)
    assert abs(d_dir - g @ v) < 1e-10 * np.abs(g * v).sum()
    h = 1e-6
    Jp = solver.objective(solver.forward(prob_of(q_eval + h * v), ts, rtol=1e-13)[0], u_gt)
    Jm = solver.objective(solver.forward(prob_of(q_eval - h * v), ts, rtol=1e-13)[0], u_gt)
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - g @ v) < 1e-6 * abs(g @ v), (fd, g @ v)


def test_models_without_parameter_derivatives_are_refused(barlat_inverse_problem):
    prob_of, q_eval, ts, u_gt, _ = barlat_inverse_problem
    P = prob_of(q_eval)
    P.local = lambda eps, epn, alpn, derivatives=True: None       # no n_params attribute
    with pytest.raises(NotImplementedError):
        solver.adjoint(P, ts, np.zeros((len(ts), P.n_dof)), None, u_gt)
