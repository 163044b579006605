"""GPU Gauss-point sweep vs the FP64 oracle, element by element through the C ABI.

Each case builds a seeded state (mesh, displacement, history, material), runs one sweep on
the GPU in FP64 and in mixed precision, and compares the assembled internal force R, the
assembled tangent K (exported block-CSR) and the trial history with the oracle's.  Cases:
mixed elastic/plastic states on a distorted mesh whose element count leaves a ragged CTA tail,
exactly repeated principal stretches (homogeneous uniaxial state), rotated material axes,
per-element parameters, Voce and Swift hardening, the zero state."""
import numpy as np
import pytest

from oracle import element, solver
from paper_2606_17390_b300 import hfe, inputs
from tests._helpers import bsr_to_csr, hist_oracle_to_soa, mixed_state, rel_inf

pytestmark = pytest.mark.gpu

# mixed: FP32 kinematics and FP32 history storage (eps_p, alpha); the history bound matches
# the 1e-5 displacement tolerance of the mixed path
TOL = {"fp64": dict(R=1e-11, K=1e-9, h=1e-12), "mixed": dict(R=2e-5, K=1e-4, h=1e-5)}


def _oracle(mesh, u, hist, theta, hardening, Theta):
    es = element.element_sweep(mesh.X, mesh.conn.astype(np.int64), u, hist, theta, hardening, Theta)
    prob = solver.Problem(X=mesh.X, conn=mesh.conn.astype(np.int64), fixed_dof=np.zeros(0, np.int64),
                          fixed_val=np.zeros(0), theta=theta, hardening=hardening)
    return solver.assemble_R(prob, es["Re"]), solver.assemble_K(prob, es["Ke"]), es


def _gpu(mesh, u, hist, theta, hardening, Theta, precision, **opts):
    with hfe.Solver(mesh.X, mesh.conn, np.zeros(0, np.int64), np.zeros(0), theta, hardening, Theta,
                    precision=precision, **opts) as s:
        s.set_state(np.zeros(mesh.n_dof), hist_oracle_to_soa(hist))
        Ht = np.empty((7, mesh.n_gp if hasattr(mesh, "n_gp") else 8 * mesh.n_el))
        R, _, st = s.sweep(u, 1.0, tangent=True, hist_out=Ht)
        rowptr, cols, vals = s.get_bsr()
        K = bsr_to_csr(rowptr, cols, vals, mesh.n_nodes)
        return R, K, Ht, st


def _compare(mesh, u, hist, theta, hardening, Theta=None, min_plastic=0.05, max_plastic=0.95):
    Ro, Ko, es = _oracle(mesh, u, hist, theta, hardening, Theta)
    frac = es["gp"]["plastic"].mean()
    assert min_plastic <= frac <= max_plastic, frac
    ho = hist_oracle_to_soa(es["h_new"])
    for prec in ("fp64", "mixed"):
        R, K, Ht, st = _gpu(mesh, u, hist, theta, hardening, Theta, prec)
        tol = TOL[prec]
        assert st["local_fail"] == 0
        assert abs(st["plastic_gps"] - es["gp"]["plastic"].sum()) <= (0 if prec == "fp64" else 2)
        assert rel_inf(R, Ro) < tol["R"], (prec, rel_inf(R, Ro))
        dK = (K - Ko).tocsr()
        kerr = np.abs(dK.data).max() / np.abs(Ko.data).max() if dK.nnz else 0.0
        assert kerr < tol["K"], (prec, kerr)
        herr = np.abs(Ht - ho).max() / max(np.abs(ho[:6]).max(), 1e-12)
        assert herr < tol["h"], (prec, herr)


@pytest.mark.parametrize("hardening", ["swift", "voce"])
def test_sweep_mixed_state_distorted_ragged(hardening):
    mesh = inputs.distorted_box_mesh(4, seed=3, amp=0.2)
    keep = np.arange(mesh.n_el) != 5              # 63 elements: ragged tail, uneven colours
    mesh = inputs.Mesh(X=mesh.X, conn=mesh.conn[keep])
    mat = inputs.config0_material() if hardening == "swift" else inputs.config1_material()
    u, hist = mixed_state(mesh, 11)
    _compare(mesh, u, hist, mat.theta_vector(), hardening)


def test_sweep_rotated_axes_per_element_theta():
    mesh = inputs.distorted_box_mesh(3, seed=4, amp=0.15)
    mat = inputs.config1_material()
    rng = np.random.default_rng(2)
    theta = mat.theta_vector()[None, :] * (1 + 0.15 * rng.uniform(-1, 1, (mesh.n_el, 11)))
    a = np.deg2rad(37.0)
    c, s_ = np.cos(a), np.sin(a)
    Theta = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1.0]]) @ np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)],
                                                                         [0, np.sin(0.3), np.cos(0.3)]])
    u, hist = mixed_state(mesh, 21)
    _compare(mesh, u, hist, theta, "voce", Theta)


def test_sweep_repeated_principal_stretches():
    """Homogeneous uniaxial stretch on a regular mesh: C = diag(a, b, b) at every point."""
    mesh = inputs.box_mesh(3, 2, 2)
    X = mesh.X
    u = np.stack([0.02 * X[:, 0], -0.006 * X[:, 1], -0.006 * X[:, 2]], 1).ravel()
    hist = np.zeros((mesh.n_el, 8, 7))
    _compare(mesh, u, hist, inputs.config0_material().theta_vector(), "swift", min_plastic=1.0, max_plastic=1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_slab_launch_order(precision):
    """Launches ordered by slabs of K rows (options.assembly_l2_bytes small enough for many
    slabs on this mesh, each colour of a slab a launch of a few elements): K, R and the trial
    history match the oracle as in colour order, and match the colour-order sweep up to the
    order of the additions (the history bit for bit)."""
    mesh = inputs.distorted_box_mesh(6, seed=12, amp=0.2)
    mat = inputs.config1_material()
    u, hist = mixed_state(mesh, 31)
    Ro, Ko, es = _oracle(mesh, u, hist, mat.theta_vector(), "voce", None)
    with hfe.Solver(mesh.X, mesh.conn, np.zeros(0, np.int64), np.zeros(0), mat.theta_vector(), "voce",
                    precision=precision, assembly_l2_bytes=6000) as s:
        info = s.info()
    assert info["n_slabs"] > 10 and info["n_launches"] > info["n_slabs"]
    runs = {b: _gpu(mesh, u, hist, mat.theta_vector(), "voce", None, precision, assembly_l2_bytes=b) for b in (0, 6000)}
    tol = TOL[precision]
    R, K, Ht, st = runs[6000]
    assert st["local_fail"] == 0 and 0.05 < es["gp"]["plastic"].mean() < 0.95
    assert rel_inf(R, Ro) < tol["R"]
    assert np.abs((K - Ko).tocsr().data).max() / np.abs(Ko.data).max() < tol["K"]
    R0, K0, Ht0, _ = runs[0]
    assert np.array_equal(Ht, Ht0)
    assert rel_inf(R, R0) < (1e-13 if precision == "fp64" else 1e-12)
    assert np.abs((K - K0).tocsr().data).max() / np.abs(K0.data).max() < (1e-13 if precision == "fp64" else 2e-6)


def test_sweep_zero_state_is_linear_elastic():
    mesh = inputs.box_mesh(2, 2, 2)
    u = np.zeros(mesh.n_dof)
    hist = np.zeros((mesh.n_el, 8, 7))
    _compare(mesh, u, hist, inputs.config0_material().theta_vector(), "swift", min_plastic=0.0, max_plastic=0.0)


# relative distances delta of the trial phi from the yield value: |phi^2 - phi_y^2| ~ 2|delta|
# phi_y^2, so +-2e-6 and +-4e-6 lie inside the mixed path's FP64 band (1e-5) and +-1e-5 just
# outside it; FP32 rounding of the trial stress (~1e-7) cannot move any of them across
BAND = np.array([-1e-3, -1e-5, -4e-6, -2e-6, 2e-6, 4e-6, 1e-5, 1e-3])


def _band_state():
    """Trial states placed at a relative distance delta from the yield surface, delta cycling
    through BAND over the Gauss points: the mixed path's FP32 elastic test leaves
    |phi_tr^2 - phi_y^2| < 1e-5 phi_y^2 to FP64 (reading R10), and most of these points lie
    inside that band.  alpha_n is set per Gauss point so that sqrt(2/3) sigma_y(alpha_n) =
    phi_tr / (1 + delta), with phi_tr the oracle's trial value (it does not depend on alpha_n)
    and Swift sigma_y inverted in closed form."""
    mesh = inputs.distorted_box_mesh(3, seed=8, amp=0.15)
    rng = np.random.default_rng(5)
    G = 0.001 * rng.uniform(-1, 1, (3, 3)) + np.diag([0.004, -0.002, -0.002])
    u = (mesh.X @ G.T + 0.0004 * rng.uniform(-1, 1, mesh.X.shape)).ravel()
    ep, _ = inputs.random_history(8 * mesh.n_el, 6, 0.0008, 0.0)
    hist = np.concatenate([ep, np.zeros((ep.shape[0], 1))], axis=1).reshape(mesh.n_el, 8, 7)
    mat = inputs.config0_material()
    th = mat.theta_vector()
    es = element.element_sweep(mesh.X, mesh.conn.astype(np.int64), u, hist, th, "swift", jacobians=None)
    K, e0, n = th[8], th[9], th[10]
    phi_tr = es["gp"]["ftr"] + np.sqrt(2.0 / 3.0) * K * e0 ** n
    delta = BAND[np.arange(phi_tr.size) % BAND.size]
    sy = phi_tr / (np.sqrt(2.0 / 3.0) * (1.0 + delta))
    assert np.all(sy > 1.05 * K * e0 ** n)          # every target lies above the initial yield
    hist[..., 6] = ((sy / K) ** (1.0 / n) - e0).reshape(mesh.n_el, 8)
    return mesh, u, hist, th, delta


def test_sweep_trial_states_in_the_fp64_decision_band():
    """R, K and the trial history of both precisions against the oracle where the
    elastic/plastic decision is a near tie: both precisions must take the oracle's decision at
    every point (the tangent jumps between the elastic and the plastic form there, so a wrong
    decision would show in K), the mixed path by its FP64 test inside the band."""
    mesh, u, hist, th, delta = _band_state()
    Ro, Ko, es = _oracle(mesh, u, hist, th, "swift", None)
    pl_o = es["gp"]["plastic"]
    assert np.array_equal(pl_o, delta > 0.0)           # the oracle sees the intended side
    ho = hist_oracle_to_soa(es["h_new"])
    for prec in ("fp64", "mixed"):
        R, K, Ht, st = _gpu(mesh, u, hist, th, "swift", None, prec)
        tol = TOL[prec]
        assert st["local_fail"] == 0
        assert int(st["plastic_gps"]) == int(pl_o.sum()), (prec, st["plastic_gps"], int(pl_o.sum()))
        assert rel_inf(R, Ro) < tol["R"], (prec, rel_inf(R, Ro))
        dK = (K - Ko).tocsr()
        kerr = np.abs(dK.data).max() / np.abs(Ko.data).max() if dK.nnz else 0.0
        assert kerr < tol["K"], (prec, kerr)
        # eps_p and alpha each against their own scale (alpha_n reaches ~1.8 here, eps_p ~3e-3)
        herr = np.abs(Ht[:6] - ho[:6]).max() / np.abs(ho[:6]).max()
        aerr = np.abs(Ht[6] - ho[6]).max() / np.abs(ho[6]).max()
        assert herr < tol["h"] and aerr < tol["h"], (prec, herr, aerr)
