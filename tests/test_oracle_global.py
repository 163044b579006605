"""Pins of the oracle's element, global Newton and adjoint (CPU only).

* P2: homogeneous uniaxial closed form of the whole forward solve (config-0 cube, roller
  symmetry BCs, 10 steps to 5 % engineering strain), with Swift hardening and with Voce
  hardening (config 1's sigma0, Q, b).
* P3: elastic and plastic patch tests on a distorted mesh (affine boundary data).
* P5: K^e equals central FD of R^e (consistent tangent, Eq. Stiffness_mat); K symmetric.
* R12: symmetric elimination and identity-row elimination (Algorithm
  gpu_chunked_assembly) give the same Newton update.
* P7: adjoint (Eq. dR_u, Eq. main_grad) = direct sensitivity to 1e-10, and = central FD
  (Algorithm finite_difference), for uniform and per-element parameters.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import element, solver
from paper_2606_17390_b300 import inputs


def _uniaxial_closed_form(t, mesh, law="swift", strain=0.05):
    """eps11 = ln(1 + strain t) = sigma_y(alpha)/E + alpha (G + H = 1, r11 = 1), T22 = T33 = 0,
    eps_p = alpha diag(1, -H, -G).  law "swift": sigma_y = K (eps0 + alpha)^n with the
    config-0 values; "voce": sigma_y = sigma0 + Q (1 - exp(-b alpha)) with the config-1 values
    (Eq. Hard with the sqrt(2/3) moved into the yield function, reading R1).  The hardening
    law is written out here, independently of the oracle, and alpha solved by 1-D Newton."""
    E, nu, G_, H_ = 70000.0, 0.33, 0.30, 0.70
    if law == "swift":
        K, e0, n = 500.0, 0.01, 0.2
        sy = lambda a: K * (e0 + a) ** n
        dsy = lambda a: K * n * (e0 + a) ** (n - 1)
    else:
        s0, Q, b = 150.0, 120.0, 12.0
        sy = lambda a: s0 + Q * (1.0 - np.exp(-b * a))
        dsy = lambda a: Q * b * np.exp(-b * a)
    e11 = np.log1p(strain * t)
    a = 0.0
    if sy(0.0) / E < e11:
        for _ in range(60):
            r = sy(a) / E + a - e11
            a -= r / (dsy(a) / E + 1.0)
    T11 = sy(a) if a > 0 else E * e11
    e22 = -nu * T11 / E - H_ * a
    e33 = -nu * T11 / E - G_ * a
    X = mesh.X
    u = np.stack([X[:, 0] * np.expm1(e11), X[:, 1] * np.expm1(e22), X[:, 2] * np.expm1(e33)], 1)
    return u.ravel(), a, T11, e11


def config0_voce_problem():
    """The config-0 cube and roller BCs with config 1's Voce material (same Hill constants)."""
    mesh, bc, _, ts = inputs.config0_problem()
    return mesh, bc, inputs.config1_material(), ts


@pytest.mark.parametrize("law", ["swift", "voce"])
def test_homogeneous_uniaxial_closed_form(law):
    if law == "swift":
        mesh, bc, mat, ts = inputs.config0_problem()
    else:
        mesh, bc, mat, ts = config0_voce_problem()
    prob = solver.from_inputs(mesh, bc, mat)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    alphas = []
    for n, t in enumerate(ts):
        uex, a, T11, e11 = _uniaxial_closed_form(t, mesh, law)
        assert a > 0                                   # every step is plastic
        alphas.append(a)
        assert np.abs(us[n] - uex).max() < 1e-12 * np.abs(uex).max()
        assert np.abs(hs[n + 1][..., 6] - a).max() < 1e-13
        ep = hs[n + 1][..., :6]
        assert np.abs(ep - a * np.array([1.0, -0.7, -0.3, 0, 0, 0])).max() < 1e-13
        # reaction on the driven face: A0 * P11 with P11 = T11 / F11
        R, _, _ = solver.residual(prob, us[n], hs[n], t, jacobians=None)
        face = bc.dof[(bc.value != 0.0)]
        assert abs(R[face].sum() - T11 / np.exp(e11)) < 1e-9 * T11
    if law == "voce":
        # the steps span b alpha from ~0.04 to ~0.6: the exponential's curvature is exercised,
        # so a misplaced factor on Q or b, or a sign in the exponent, moves u beyond 1e-12
        assert 12.0 * alphas[0] < 0.1 and 12.0 * alphas[-1] > 0.5


@pytest.mark.parametrize("plastic", [False, True])
def test_patch_test_distorted_mesh(plastic):
    mesh = inputs.distorted_box_mesh(3, seed=5, amp=0.25)
    Gm = np.array([[0.004, 0.001, -0.0005], [0.0, -0.0015, 0.001], [0.0005, 0.0, -0.0012]])
    Gm = Gm * (12.0 if plastic else 0.25)
    bnd = np.nonzero(np.any(np.isclose(mesh.X, 0.0) | np.isclose(mesh.X, 1.0), axis=1))[0]
    dof = (3 * bnd[:, None] + np.arange(3)).ravel()
    val = (mesh.X[bnd] @ Gm.T).ravel()
    mat = inputs.config1_material()
    prob = solver.Problem(X=mesh.X, conn=mesh.conn.astype(np.int64), fixed_dof=dof,
                          fixed_val=val, theta=mat.theta_vector(), hardening="voce")
    us, hs, infos = solver.forward(prob, [0.5, 1.0], rtol=1e-12)
    uex = (mesh.X @ Gm.T).ravel()
    assert np.abs(us[-1] - uex).max() < 1e-11 * np.abs(uex).max()
    n_pl = infos[-1]["plastic"]
    assert (n_pl == 8 * mesh.n_el) if plastic else (n_pl == 0)
    # homogeneous history
    assert np.ptp(hs[-1][..., 6]) < 1e-12


def _one_element_state(seed, scale):
    mesh = inputs.distorted_box_mesh(1, seed=seed, amp=0.0)
    X = mesh.X + np.random.default_rng(seed).uniform(-0.15, 0.15, mesh.X.shape)
    u = scale * np.random.default_rng(seed + 1).uniform(-1, 1, X.shape).ravel()
    return X, mesh.conn.astype(np.int64), u


@pytest.mark.parametrize("case", ["elastic", "plastic", "near_repeated"])
def test_element_tangent_vs_fd(case):
    X, conn, u = _one_element_state(7, {"elastic": 1e-4, "plastic": 0.04, "near_repeated": 0.0}[case])
    if case == "near_repeated":
        u = (0.03 * X @ np.diag([1.0, 1e-9, 0.0]).T).ravel()
    mat = inputs.config0_material()
    hist = np.zeros((1, 8, 7))
    if case != "elastic":
        ep, al = inputs.random_history(8, 3, 0.005, 0.02)
        hist[0, :, :6], hist[0, :, 6] = ep, al
    es = element.element_sweep(X, conn, u, hist, mat.theta_vector(), "swift")
    n_pl = int(es["gp"]["plastic"].sum())
    assert (n_pl == 0) if case == "elastic" else (n_pl > 0 or case == "near_repeated")
    Ke = es["Ke"][0]
    assert np.abs(Ke - Ke.T).max() < 1e-10 * np.abs(Ke).max()
    h = 1e-7
    fd = np.empty((24, 24))
    for j in range(24):
        up, um = u.copy(), u.copy()
        up[j] += h
        um[j] -= h
        fd[:, j] = (element.element_sweep(X, conn, up, hist, mat.theta_vector(), "swift", None, None)["Re"][0] -
                    element.element_sweep(X, conn, um, hist, mat.theta_vector(), "swift", None, None)["Re"][0]) / (2 * h)
    ed = solver.element_dofs(conn)[0]          # columns of fd are global dofs
    assert np.abs(fd[:, ed] - Ke).max() < 1e-6 * np.abs(Ke).max()


def test_symmetric_vs_row_elimination():
    mesh, bc, mat, ts = inputs.config0_problem(n=3)
    prob = solver.from_inputs(mesh, bc, mat)
    u = np.zeros(prob.n_dof)
    u[bc.dof] = 0.3 * bc.value
    R, K, _ = solver.residual(prob, u, np.zeros((prob.n_el, 8, 7)), 0.3)
    free = solver.free_mask(prob)
    du_sym = np.zeros(prob.n_dof)
    du_sym[free] = spla.spsolve(K[free][:, free].tocsc(), -R[free])
    Kr = K.tolil()
    rhs = -R.copy()
    for d in bc.dof:                     # identity rows, as in the paper's batched kernel
        Kr.rows[d] = [d]
        Kr.data[d] = [1.0]
        rhs[d] = 0.0
    du_row = spla.spsolve(Kr.tocsc(), rhs)
    assert np.abs(du_row - du_sym).max() < 1e-10 * np.abs(du_sym).max()


def _tiny_inverse_problem(per_element=False):
    mesh = inputs.box_mesh(3, 2, 1, 3.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.06, 0.02, 0.0))
    mat = inputs.config1_material()
    a = np.deg2rad(30.0)
    mat.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    th_true = mat.theta_vector()
    ts = inputs.load_factors(3)
    p_true = solver.from_inputs(mesh, bc, mat, th_true)
    u_gt, _, _ = solver.forward(p_true, ts, rtol=1e-13)
    rng = np.random.default_rng(4)
    u_gt = u_gt + 1e-3 * np.abs(u_gt).max() * rng.standard_normal(u_gt.shape)
    th_eval = th_true * (1 + 0.1 * rng.uniform(-1, 1, th_true.shape))
    if per_element:
        th_eval = th_eval[None, :] * (1 + 0.05 * rng.uniform(-1, 1, (mesh.n_el, 11)))
    prob = solver.from_inputs(mesh, bc, mat, th_eval)
    return prob, ts, u_gt


def test_adjoint_equals_direct_and_fd_uniform():
    prob, ts, u_gt = _tiny_inverse_problem()
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    assert sum(i["plastic"] for i in infos) > 0
    g = solver.adjoint(prob, ts, us, hs, u_gt)
    v = np.random.default_rng(9).standard_normal(11) * np.abs(prob.theta)
    d_dir = solver.direct_sensitivity(prob, ts, us, hs, u_gt, v)
    assert abs(d_dir - g @ v) < 1e-10 * np.abs(g * v).sum()
    fd = solver.fd_gradient(prob, ts, u_gt, h_rel=1e-6)
    gmax = np.abs(g).max()
    for i, gi in fd.items():
        if abs(g[i]) > 1e-3 * gmax:
            assert abs(gi - g[i]) < 1e-5 * abs(g[i]), (i, gi, g[i])


def test_adjoint_per_element_directional():
    prob, ts, u_gt = _tiny_inverse_problem(per_element=True)
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    g = solver.adjoint(prob, ts, us, hs, u_gt, per_element=True)
    assert g.shape == (prob.n_el, 11)
    v = np.zeros_like(prob.theta)
    rng = np.random.default_rng(11)
    v[:, [2, 3, 4, 8]] = rng.standard_normal((prob.n_el, 4)) * np.abs(prob.theta[:, [2, 3, 4, 8]])
    d_dir = solver.direct_sensitivity(prob, ts, us, hs, u_gt, v)
    assert abs(d_dir - np.sum(g * v)) < 1e-10 * np.abs(g * v).sum()
    fd = solver.fd_directional(prob, ts, u_gt, v, h=1e-6)
    assert abs(fd - np.sum(g * v)) < 1e-5 * abs(np.sum(g * v))


@pytest.mark.parametrize("case", ["elastic", "plastic"])
def test_fbar_element_tangent_vs_fd(case):
    """F-bar element (Eq. Fbar): K^e = dR^e/dd^e against central differences of R^e on a
    distorted element (the chain rule through J at the point and the element's Jbar; K^e is
    not symmetric)."""
    X, conn, u = _one_element_state(9, {"elastic": 1e-4, "plastic": 0.04}[case])
    mat = inputs.config0_material()
    hist = np.zeros((1, 8, 7))
    if case != "elastic":
        ep, al = inputs.random_history(8, 5, 0.005, 0.02)
        hist[0, :, :6], hist[0, :, 6] = ep, al
    es = element.element_sweep(X, conn, u, hist, mat.theta_vector(), "swift", fbar=True)
    Ke = es["Ke"][0]
    assert np.abs(Ke - Ke.T).max() > 1e-8 * np.abs(Ke).max()   # not symmetric
    h = 1e-7
    fd = np.empty((24, 24))
    for j in range(24):
        up, um = u.copy(), u.copy()
        up[j] += h
        um[j] -= h
        fd[:, j] = (element.element_sweep(X, conn, up, hist, mat.theta_vector(), "swift", None, None, fbar=True)["Re"][0] -
                    element.element_sweep(X, conn, um, hist, mat.theta_vector(), "swift", None, None, fbar=True)["Re"][0]) / (2 * h)
    ed = solver.element_dofs(conn)[0]
    assert np.abs(fd[:, ed] - Ke).max() < 1e-6 * np.abs(Ke).max()


def test_fbar_equals_standard_for_affine_motion_and_closed_form():
    """For an affine displacement J is uniform in the element, so Jbar = J, Fbar = F and the
    F-bar residual and history equal the standard ones; the homogeneous uniaxial forward
    (config 0) therefore keeps its closed form with the F-bar element."""
    X, conn, _ = _one_element_state(11, 0.0)
    G = 0.03 * np.random.default_rng(12).uniform(-1, 1, (3, 3))
    u = (X @ G.T).ravel()
    mat = inputs.config0_material()
    ep, al = inputs.random_history(8, 13, 0.005, 0.02)
    hist = np.zeros((1, 8, 7))
    hist[0, :, :6], hist[0, :, 6] = ep, al
    a = element.element_sweep(X, conn, u, hist, mat.theta_vector(), "swift")
    b = element.element_sweep(X, conn, u, hist, mat.theta_vector(), "swift", fbar=True)
    assert np.abs(a["Re"] - b["Re"]).max() < 1e-12 * np.abs(a["Re"]).max()
    assert np.abs(a["h_new"] - b["h_new"]).max() < 1e-14
    mesh, bc, mat, ts = inputs.config0_problem(n=3, n_steps=3)
    prob = solver.from_inputs(mesh, bc, mat, fbar=True)
    us, hs, _ = solver.forward(prob, ts, rtol=1e-13)
    for n, t in enumerate(ts):
        uex = _uniaxial_closed_form(t, mesh)[0]
        assert np.abs(us[n] - uex).max() < 1e-11 * np.abs(uex).max()
