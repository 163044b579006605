"""Pins of the oracle's Barlat Yld2004-18p material point (CPU only) against what the paper
and the mathematics fix: the printed step lengths of App. B's single-point line-search
analysis (golden fixture), the eigenvalue definition of Eq. Phi_barlat, central differences
of that definition, the isotropic reductions of App. A.2 (von Mises for m = 2 and 4, the
uniaxial and pure-shear closed forms for any even m), homogeneity, pressure insensitivity and
frame objectivity, the von Mises radial return in closed form, the closest-point projection
as the minimiser of the complementary energy over the yield set (perfect plasticity), central
differences of the projection for the implicit-differentiation tangent (App. D), and App. B's
robustness statement on a small sample of the pi-plane map."""
import os

import numpy as np
import pytest
from scipy.optimize import brentq, minimize

from oracle import barlat as BA
from oracle.material import complex_step_jacobian
from paper_2606_17390_b300 import inputs

ONES = (1.0,) * 9


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "barlat_linesearch_single_point.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {r[0]: (float(r[1]), int(r[2])) for r in rows}


def _model(mat, Theta=None):
    return BA.Barlat(mat.c1, mat.c2, mat.m, Theta)


def _cpp(model, mat, Ttr, alpn, **kw):
    return BA.cpp(model, mat.E, mat.nu, mat.hardening, mat.h, Ttr, alpn, **kw)


def _trial_states(model, mat, angle, scale, alpn):
    d = inputs.principal_plane_directions(angle)
    sy = BA.sigma_y(mat.hardening, mat.h, alpn)
    return (scale * sy / model.phi_poly(d))[:, None] * d


def test_golden_single_point_line_search():
    """App. B: third iteration: full step raises psi, the quadratic model gives 0.363, the
    minimiser along the direction is 0.46; plain Newton still unconverged after 10 steps."""
    g = _golden()
    mat = inputs.barlat_verification_material()
    model = _model(mat)
    T = np.array([[g["trial_11"][0], g["trial_22"][0], g["trial_33"][0], 0.0, 0.0, 0.0]])
    a0 = np.zeros(1)
    trace = []
    y, it, conv = _cpp(model, mat, T, a0, line_search=True, kmax=40, trace=trace)
    assert conv[0] and it[0] < 20
    t3 = trace[2]
    assert t3["psi1"][0] > t3["psi0"][0]                       # the full step raises the merit
    z, dec = g["third_iteration_zeta"]
    assert abs(t3["zeta"][0] - z) <= 0.5 * 10.0 ** -dec          # 0.363 as printed
    assert t3["zeta"][0] == pytest.approx(t3["psi0"][0] / (t3["psi0"][0] + t3["psi1"][0]), rel=1e-14)
    assert trace[0]["zeta"][0] == 1.0 and trace[1]["zeta"][0] == 1.0
    # the minimiser of psi along the third Newton direction
    G = lambda yy: BA.residual(model, mat.E, mat.nu, mat.hardening, mat.h, yy, T, a0)
    yk = np.concatenate([T, [[0.0, 0.0]]], axis=1)
    for k in range(3):
        dy = np.linalg.solve(complex_step_jacobian(G, yk, 8), -G(yk)[..., None])[..., 0]
        if k < 2:
            yk = yk + dy
    zz = np.linspace(0.0, 1.0, 2001)
    psi = [0.5 * np.sum(G(yk + z * dy) ** 2) for z in zz]
    zmin, dec = g["third_iteration_argmin"]
    assert abs(zz[int(np.argmin(psi))] - zmin) <= 0.5 * 10.0 ** -dec
    # standard Newton
    n_plain = int(g["plain_newton_unconverged_after"][0])
    _, it_p, conv_p = _cpp(model, mat, T, a0, line_search=False, kmax=n_plain)
    assert not conv_p[0] and it_p[0] == n_plain
    _, _, conv_p40 = _cpp(model, mat, T, a0, line_search=False, kmax=40)
    assert not conv_p40[0]
    # the converged point lies on the yield surface
    assert abs(model.phi_eig(y[:, :6])[0] - 1.0) < 1e-12


def _random_models():
    rng = np.random.default_rng(5)
    mat = inputs.barlat_verification_material()
    out = [(mat.c1, mat.c2, 8, None), (mat.c1, mat.c2, 8, inputs.random_rotation(1))]
    for m in (2, 4, 6, 12):
        out.append((tuple(rng.uniform(-0.2, 1.6, 9)), tuple(rng.uniform(-0.2, 1.6, 9)), m,
                    inputs.random_rotation(m)))
    return out


@pytest.mark.parametrize("k", range(6))
def test_power_trace_form_equals_eigenvalue_definition(k):
    c1, c2, m, Th = _random_models()[k]
    model = BA.Barlat(c1, c2, m, Th)
    T = inputs.random_stresses(64, seed=10 + k, scale=3.0)
    ref = model.phi_eig(T)
    assert np.abs(model.phi_poly(T) - ref).max() <= 1e-12 * ref.max()
    _, phi = model.flow(T)
    assert np.abs(phi - ref).max() <= 1e-12 * ref.max()


@pytest.mark.parametrize("k", range(6))
def test_flow_against_central_differences_of_the_definition(k):
    """dphi/dT_b (component b moving both symmetric entries) = w_b N_b."""
    c1, c2, m, Th = _random_models()[k]
    model = BA.Barlat(c1, c2, m, Th)
    T = inputs.random_stresses(16, seed=20 + k, scale=2.0)
    N, _ = model.flow(T)
    h = 1e-5
    for b in range(6):
        e = np.zeros(6)
        e[b] = h
        fd = (model.phi_eig(T + e) - model.phi_eig(T - e)) / (2 * h)
        assert np.abs(fd - BA.W_SHEAR[b] * N[:, b]).max() <= 1e-7 * np.abs(N).max()


def _von_mises(T):
    s = T.copy()
    s[:, :3] -= T[:, :3].mean(axis=1, keepdims=True)
    return np.sqrt(1.5 * np.sum(BA.W_SHEAR * s * s, axis=1))


@pytest.mark.parametrize("m", [2, 4])
def test_isotropic_coefficients_give_von_mises(m):
    """All 18 coefficients 1 and m = 2 or 4: phi = sqrt(3/2 s:s) (App. A.2)."""
    model = BA.Barlat(ONES, ONES, m, inputs.random_rotation(3))
    T = inputs.random_stresses(64, seed=30, scale=5.0)
    assert np.abs(model.phi_eig(T) - _von_mises(T)).max() <= 1e-12 * _von_mises(T).max()
    assert np.abs(model.phi_poly(T) - _von_mises(T)).max() <= 1e-12 * _von_mises(T).max()


@pytest.mark.parametrize("m", [6, 8, 12])
def test_isotropic_uniaxial_and_shear_closed_forms(m):
    """s' = s'' = s: uniaxial sigma n (x) n gives |sigma|; pure shear tau (e1 e2 + e2 e1) has
    principal values (tau, -tau, 0), so phi = tau (2^(m-1) + 1)^(1/m)."""
    model = BA.Barlat(ONES, ONES, m)
    Q = inputs.random_rotation(7)
    n = Q[:, 0]
    U = BA.voigt(np.outer(n, n))[None, :]
    for sig in (1.0, -2.5):
        assert model.phi_poly(sig * U)[0] == pytest.approx(abs(sig), rel=1e-13)
    Sh = BA.voigt(np.outer(Q[:, 0], Q[:, 1]) + np.outer(Q[:, 1], Q[:, 0]))[None, :]
    tau = 0.7
    assert model.phi_poly(tau * Sh)[0] == pytest.approx(tau * (2.0 ** (m - 1) + 1) ** (1.0 / m), rel=1e-12)


def test_homogeneity_pressure_and_frame():
    mat = inputs.barlat_verification_material()
    Th = inputs.random_rotation(11)
    model = _model(mat, Th)
    T = inputs.random_stresses(32, seed=40, scale=4.0)
    phi = model.phi_poly(T)
    for lam in (3.0, -2.5):
        assert np.abs(model.phi_poly(lam * T) - abs(lam) * phi).max() <= 1e-12 * phi.max() * 3
    Tp = T.copy()
    Tp[:, :3] += 7.0
    assert np.abs(model.phi_poly(Tp) - phi).max() <= 1e-12 * phi.max()
    # rotating the stress and the material frame together leaves phi unchanged
    Q = inputs.random_rotation(12)
    rotated = _model(mat, Q @ Th)
    TQ = BA.voigt(Q @ BA.tensor(T) @ Q.T)
    assert np.abs(rotated.phi_poly(TQ) - phi).max() <= 1e-12 * phi.max()


@pytest.mark.parametrize("hardening,h", [("voce", (1.0, 0.0, 0.0)), ("swift", (500.0, 0.01, 0.2))])
@pytest.mark.parametrize("m", [2, 4])
def test_von_mises_radial_return_closed_form(hardening, h, m):
    """Isotropic coefficients: T = T_tr - 2 mu dgamma (3/2) s_tr / sigma_tr with dgamma from
    sigma_tr - 3 mu dgamma = sigma_y(alpha_n + dgamma) (W = 1)."""
    E, nu = 1000.0, 0.3
    if hardening == "swift":
        E = 70000.0
    model = BA.Barlat(ONES, ONES, m)
    lam, mu = BA.lame(E, nu)
    rng = np.random.default_rng(50 + m)
    alpn = rng.uniform(0.0, 0.05, size=8)
    T = inputs.random_stresses(8, seed=51 + m, scale=1.0)
    sy = BA.sigma_y(hardening, h, alpn)
    vm = _von_mises(T)
    Ttr = T * (sy * rng.uniform(1.2, 6.0, size=8) / vm)[:, None]
    y, it, conv = BA.cpp(model, E, nu, hardening, h, Ttr, alpn)
    assert conv.all()
    s_tr = Ttr.copy()
    s_tr[:, :3] -= Ttr[:, :3].mean(axis=1, keepdims=True)
    str_ = _von_mises(Ttr)
    for p in range(8):
        dg = brentq(lambda g: str_[p] - 3 * mu * g - BA.sigma_y(hardening, h, alpn[p] + g), 0.0, str_[p] / (3 * mu))
        Tex = Ttr[p] - 2 * mu * dg * 1.5 * s_tr[p] / str_[p]
        assert y[p, 7] == pytest.approx(dg, rel=1e-10)
        assert y[p, 6] == pytest.approx(alpn[p] + dg, rel=1e-12)
        assert np.abs(y[p, :6] - Tex).max() <= 1e-11 * np.abs(Ttr[p]).max()


def test_projection_minimises_complementary_energy():
    """Perfect plasticity: the converged stress is the point of the convex set phi <= sigma0
    closest to T_tr in the complementary-energy norm (T_tr - T) : E^-1 : (T_tr - T); found here
    by a direct constrained minimisation over the eigenvalue definition of phi."""
    mat = inputs.barlat_verification_material()
    Th = inputs.random_rotation(21)
    model = _model(mat, Th)
    angle, scale = inputs.pi_plane_sample(6, seed=8)
    Ttr = _trial_states(model, mat, angle, scale, np.zeros(6))
    Ttr[:3, 3:] += inputs.random_stresses(3, seed=9, scale=0.5)[:, 3:]   # shear components too
    y, it, conv = _cpp(model, mat, Ttr, np.zeros(6))
    assert conv.all() and (y[:, 7] > 0).all()
    lam, mu = BA.lame(mat.E, mat.nu)

    def energy(T, p):
        d = Ttr[p] - T
        e = d / (2 * mu)
        e[:3] -= lam / (2 * mu * (3 * lam + 2 * mu)) * d[:3].sum()
        return 0.5 * np.sum(BA.W_SHEAR * d * e) * mat.E

    for p in range(6):
        T0 = Ttr[p] / model.phi_eig(Ttr[p:p + 1])[0]
        res = minimize(lambda x: energy(x, p), T0, method="SLSQP",
                       constraints=[dict(type="ineq", fun=lambda x: 1.0 - model.phi_eig(x[None, :])[0])],
                       options=dict(ftol=1e-16, maxiter=1000))
        assert np.abs(res.x - y[p, :6]).max() <= 2e-5 * np.abs(Ttr[p]).max(), (p, res.x, y[p, :6])
        assert energy(y[p, :6], p) <= res.fun * (1 + 1e-9)
        assert abs(model.phi_eig(y[p:p + 1, :6])[0] - 1.0) < 1e-12


def test_tangent_against_differences_of_the_projection():
    mat = inputs.barlat_verification_material()
    mat.h = (1.0, 0.5, 20.0)                                      # Voce hardening: alpha matters
    model = _model(mat, inputs.random_rotation(31))
    angle, scale = inputs.pi_plane_sample(4, seed=32, scale_max=5.0)
    alpn = np.array([0.0, 0.01, 0.02, 0.03])
    Ttr = _trial_states(model, mat, angle, scale, alpn)
    Ttr[:, 3:] += inputs.random_stresses(4, seed=33, scale=0.3)[:, 3:]
    y, _, conv = _cpp(model, mat, Ttr, alpn, kmax=60)
    assert conv.all()
    D = BA.cpp_tangent(model, mat.E, mat.nu, mat.hardening, mat.h, y, Ttr, alpn)
    h = 1e-6
    for b in range(6):
        e = np.zeros(6)
        e[b] = h
        yp, _, cp = _cpp(model, mat, Ttr + e, alpn, kmax=60)
        ym, _, cm = _cpp(model, mat, Ttr - e, alpn, kmax=60)
        assert cp.all() and cm.all()
        fd = (yp[:, :6] - ym[:, :6]) / (2 * h)
        assert np.abs(fd - D[:, :, b]).max() <= 1e-6 * np.abs(D).max()


def test_pi_plane_map_sample_line_search_converges_plain_newton_does_not():
    """App. B on a small sample of the map: the line search converges everywhere within 40
    iterations; standard Newton leaves a large part unconverged."""
    mat = inputs.barlat_verification_material()
    model = _model(mat)
    angle, scale = inputs.pi_plane_sample(200)
    Ttr = _trial_states(model, mat, angle, scale, np.zeros(200))
    _, it_ls, conv_ls = _cpp(model, mat, Ttr, np.zeros(200), line_search=True, kmax=40)
    _, it_nw, conv_nw = _cpp(model, mat, Ttr, np.zeros(200), line_search=False, kmax=40)
    assert conv_ls.all() and it_ls.max() <= 40
    assert (~conv_nw).sum() >= 40


def test_orthotropic_elasticity_reductions_and_symmetries():
    """Isotropic coefficients (lambda + 2 mu, lambda, mu) give lambda tr(e) I + 2 mu e in any
    frame; the tensor has the minor and major symmetries; rotating the frame and the strain
    together leaves the energy e : E : e unchanged; in the material frame a diagonal strain
    gives the stiffness matrix times the strain (closed form)."""
    E, nu = 70000.0, 0.33
    lam, mu = BA.lame(E, nu)
    e = inputs.random_stresses(16, seed=80, scale=1e-3)
    iso = BA.orthotropic_tensor((lam + 2 * mu,) * 3 + (lam,) * 3 + (mu,) * 3, inputs.random_rotation(81))
    assert np.abs(BA.elastic(iso, None, e) - BA.elastic(E, nu, e)).max() <= 1e-12 * E * 1e-3
    d = (210e3, 150e3, 120e3, 60e3, 50e3, 40e3, 30e3, 25e3, 20e3)
    Th = inputs.random_rotation(82)
    Eg = BA.orthotropic_tensor(d, Th)
    for perm in ("jikl", "ijlk", "klij"):
        assert np.abs(np.einsum("ijkl->" + perm, Eg) - Eg).max() <= 1e-9 * 210e3
    Q = inputs.random_rotation(83)
    Eq = BA.orthotropic_tensor(d, Q @ Th)
    eg = BA.tensor(e)
    eq = Q @ eg @ Q.T
    w1 = np.einsum("nij,ijkl,nkl->n", eg, Eg, eg)
    w2 = np.einsum("nij,ijkl,nkl->n", eq, Eq, eq)
    assert np.abs(w1 - w2).max() <= 1e-12 * np.abs(w1).max()
    El = BA.orthotropic_tensor(d)
    diag = np.array([1e-3, -2e-3, 0.5e-3, 0, 0, 0])
    C = np.array([[d[0], d[3], d[4]], [d[3], d[1], d[5]], [d[4], d[5], d[2]]])
    assert np.allclose(BA.elastic(El, None, diag[None])[0, :3], C @ diag[:3], rtol=1e-14, atol=0)
    shear = np.array([0, 0, 0, 1e-3, 2e-3, 3e-3])   # tensor components e12, e23, e13
    assert np.allclose(BA.elastic(El, None, shear[None])[0, 3:], 2 * np.array([d[6], d[7], d[8]]) * shear[3:],
                       rtol=1e-14, atol=0)


def test_orthotropic_projection_is_the_energy_minimiser():
    """With an orthotropic, rotated E the converged stress still minimises the complementary
    energy (T_tr - T) : E^-1 : (T_tr - T) over phi <= sigma0 (perfect plasticity)."""
    mat = inputs.barlat_verification_material()
    model = _model(mat, inputs.random_rotation(91))
    d = (2.0e3, 1.4e3, 1.1e3, 0.5e3, 0.45e3, 0.4e3, 0.35e3, 0.3e3, 0.25e3)
    Eg = BA.orthotropic_tensor(d, inputs.random_rotation(92))
    angle, scale = inputs.pi_plane_sample(4, seed=93, scale_max=8.0)
    Ttr = _trial_states(model, mat, angle, scale, np.zeros(4))
    y, it, conv = BA.cpp(model, Eg, None, mat.hardening, mat.h, Ttr, np.zeros(4))
    assert conv.all()
    S6 = np.linalg.inv(np.array([[Eg[i, j, k, l] * (1 if k == l else 2) for (k, l) in BA.VOIGT]
                                 for (i, j) in BA.VOIGT]))   # component compliance

    def energy(T, p):
        dT = Ttr[p] - T
        return 0.5 * np.sum(BA.W_SHEAR * dT * (S6 @ dT)) * 1e3

    for p in range(4):
        T0 = Ttr[p] / model.phi_eig(Ttr[p:p + 1])[0]
        res = minimize(lambda x: energy(x, p), T0, method="SLSQP",
                       constraints=[dict(type="ineq", fun=lambda x: 1.0 - model.phi_eig(x[None, :])[0])],
                       options=dict(ftol=1e-16, maxiter=1000))
        assert np.abs(res.x - y[p, :6]).max() <= 2e-5 * np.abs(Ttr[p]).max()
        assert energy(y[p, :6], p) <= res.fun * (1 + 1e-9)


# ------------------------------------------------------------ finite strain, element, forward
def _hill_isotropic_swift():
    """Hill-48 with F = G = H = 1/2, L = M = N = 3/2 (all r-ratios 1: von Mises), Swift."""
    th = inputs.config0_material().theta_vector().copy()
    th[2:8] = [0.5, 0.5, 0.5, 1.5, 1.5, 1.5]
    return th


def test_isotropic_barlat_gauss_point_equals_isotropic_hill():
    """All 18 coefficients 1 with m = 2 and isotropic Hill-48 are both J2 plasticity with alpha
    the equivalent plastic strain (W = 1 against sqrt(2/3) in both f and the alpha-rate), so
    the finite-strain Gauss points (P, dP/dF, history) agree although the two local solvers,
    their unknowns and their tangents are different code."""
    from oracle import material as M
    th = _hill_isotropic_swift()
    E, nu, K, e0, n = th[0], th[1], th[8], th[9], th[10]
    model = BA.Barlat(ONES, ONES, 2)
    loc = BA.local(model, E, nu, "swift", (K, e0, n))
    F = inputs.random_deformation_gradients(48, seed=201, scale=0.003)
    ep, al = inputs.random_history(48, seed=202, eps_scale=0.0015, alpha_max=0.02)
    gh = M.gauss_point(F, ep, al, th, "swift")
    gb = M.gauss_point(F, ep, al, th, "swift", local=loc)
    assert gh["plastic"].any() and (~gh["plastic"]).any()
    assert np.array_equal(gh["plastic"], gb["plastic"])
    sP = np.abs(gh["P"]).max()
    assert np.abs(gb["P"] - gh["P"]).max() <= 1e-10 * sP
    assert np.abs(gb["h_new"] - gh["h_new"]).max() <= 1e-11
    assert np.abs(gb["A"] - gh["A"]).max() <= 1e-8 * np.abs(gh["A"]).max()


def test_barlat_element_tangent_against_differences():
    """The element stiffness with the Barlat update (paper parameters, rotated frame, plastic
    state) against central differences of the element residual."""
    from oracle import element
    mat = inputs.barlat_verification_material()
    mat.E, mat.h = 70000.0, (1.0, 0.0, 0.0)
    model = BA.Barlat(mat.c1, mat.c2, mat.m, inputs.random_rotation(203))
    loc = BA.local(model, mat.E, mat.nu, "voce", (1.0, 0.0, 0.0))
    mesh = inputs.distorted_box_mesh(1, seed=204, amp=0.15)
    rng = np.random.default_rng(205)
    u = (mesh.X @ (4e-5 * rng.uniform(-1, 1, (3, 3))).T + 1e-5 * rng.uniform(-1, 1, mesh.X.shape)).ravel()
    hist = np.zeros((1, 8, 7))
    es = element.element_sweep(mesh.X, mesh.conn.astype(np.int64), u, hist, np.zeros(11), "voce", local=loc)
    assert es["gp"]["plastic"].any()
    Ke = es["Ke"][0]                               # element-local order (node a of conn, component)
    gdof = (3 * mesh.conn[0][:, None] + np.arange(3)).ravel()
    h = 1e-9
    fd = np.empty((24, 24))
    for j in range(24):
        e = np.zeros(mesh.n_dof)
        e[gdof[j]] = h
        rp = element.element_sweep(mesh.X, mesh.conn.astype(np.int64), u + e, hist, np.zeros(11), "voce",
                                   jacobians=None, local=loc)["Re"][0]
        rm = element.element_sweep(mesh.X, mesh.conn.astype(np.int64), u - e, hist, np.zeros(11), "voce",
                                   jacobians=None, local=loc)["Re"][0]
        fd[:, j] = (rp - rm) / (2 * h)
    assert np.abs(fd - Ke).max() <= 1e-6 * np.abs(Ke).max()


def test_isotropic_barlat_forward_equals_isotropic_hill():
    """The whole forward solve (config 0's cube, 4^3... here 2^3, 4 load steps) with the
    isotropic Barlat update equals the isotropic Hill-48 solve."""
    from oracle import solver
    mesh, bc, mat, ts = inputs.config0_problem(n=2, n_steps=4)
    th = _hill_isotropic_swift()
    E, nu, K, e0, n = th[0], th[1], th[8], th[9], th[10]
    ph = solver.from_inputs(mesh, bc, mat, th)
    pb = solver.from_inputs(mesh, bc, mat, th)
    pb.local = BA.local(BA.Barlat(ONES, ONES, 2), E, nu, "swift", (K, e0, n))
    uh, hh, ih = solver.forward(ph, ts, rtol=1e-12)
    ub, hb, ib = solver.forward(pb, ts, rtol=1e-12)
    assert sum(i["plastic"] for i in ih) > 0
    assert np.abs(ub - uh).max() <= 1e-10 * np.abs(uh).max()
    assert np.abs(np.asarray(hb) - np.asarray(hh)).max() <= 1e-10
