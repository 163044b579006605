"""Pins of the oracle's material point (CPU only) against what the paper and the mathematics
fix: Hill-48 closed forms (App. A.1), the von Mises radial return (App. A.1 isotropic case),
Kuhn-Tucker conditions and plastic incompressibility (Eq. KT, Eq. Ep_update), objectivity,
an independent route through the Frechet derivative of the matrix exponential for the spectral
derivatives (Sec. 2.2.5), and finite differences of the implicit-function tangent (App. D)."""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import material as M
from paper_2606_17390_b300 import inputs

SQ23 = np.sqrt(2.0 / 3.0)


def _golden_hill():
    path = os.path.join(os.path.dirname(__file__), "golden", "hill48_uniaxial_config0.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=float)


def _uniaxial(a_deg):
    a = np.deg2rad(a_deg)
    d = np.array([np.cos(a), np.sin(a), 0.0])
    return np.outer(d, d), np.array([-np.sin(a), np.cos(a), 0.0])


@pytest.mark.parametrize("row", range(3))
def test_hill_uniaxial_closed_forms(row):
    """sigma_a / sigma_y and r_a from App. A.1's p1..p9 tensor match the golden closed forms."""
    ang, sig_ratio, r_val = _golden_hill()[row]
    th = inputs.config0_material().theta_vector()
    Hg = M.hill_tensor(th, np.eye(3))
    U, w = _uniaxial(ang)
    phi_unit, HT = M.hill_phi(Hg, U)
    # yield: phi(sigma U) = sqrt(2/3) sigma_y  ->  sigma / sigma_y = sqrt(2/3) / phi(U)
    assert abs(SQ23 / phi_unit - sig_ratio) < 5e-7
    N = HT / phi_unit
    r = (w @ N @ w) / N[2, 2]
    assert abs(r - r_val) < 5e-7
    # the same closed forms to 1e-12 (the golden file rounds to 6 decimals)
    F_, G_, H_, N_ = 0.25, 0.30, 0.70, 1.5
    c, s = np.cos(np.deg2rad(ang)), np.sin(np.deg2rad(ang))
    sr = (F_ * s ** 4 + G_ * c ** 4 + H_ * (c * c - s * s) ** 2 + 2 * N_ * s * s * c * c) ** -0.5
    rr = (H_ + (2 * N_ - F_ - G_ - 4 * H_) * s * s * c * c) / (F_ * s * s + G_ * c * c)
    assert abs(SQ23 / phi_unit - sr) < 1e-12 and abs(r - rr) < 1e-12


def test_hill_shear_yield_and_rotation():
    """tau^y_12 = r12 sigma_0 / sqrt(3) (App. A.1 definition of r12); rotating the material
    axes by 45 deg about z turns uniaxial x-loading into the 45 deg closed form (reading R4)."""
    th = inputs.config0_material().theta_vector()
    Hg = M.hill_tensor(th, np.eye(3))
    T = np.zeros((3, 3))
    T[0, 1] = T[1, 0] = 1.0
    phi, _ = M.hill_phi(Hg, T)
    r12 = np.sqrt(3.0 / (2.0 * 1.5))
    assert abs(SQ23 / phi - r12 / np.sqrt(3.0)) < 1e-13
    a = np.deg2rad(45.0)
    Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    Hr = M.hill_tensor(th, Theta)
    U, _ = _uniaxial(0.0)
    phi_r, _ = M.hill_phi(Hr, U)
    assert abs(SQ23 / phi_r - _golden_hill()[1, 1]) < 5e-7


def test_hill_isotropic_is_von_mises():
    """All r = 1 (F=G=H=1/2, L=M=N=3/2): phi = sqrt(2/3) sigma_vm (App. A.1 isotropic case)."""
    th = inputs.config0_material().theta_vector()
    th[2:8] = [0.5, 0.5, 0.5, 1.5, 1.5, 1.5]
    rng = np.random.default_rng(0)
    for _ in range(5):
        T = M.sym(rng.normal(size=6) * 100)
        phi, _ = M.hill_phi(M.hill_tensor(th, np.eye(3)), T)
        assert abs(phi - SQ23 * M.von_mises(T)) < 1e-10 * phi


def test_radial_return_reduction():
    """Von Mises + linear hardening (Swift with n = 1: sigma_y = K eps0 + K alpha) is the
    textbook radial return: alpha_{n+1} = alpha_n + (q_tr - sigma_y(alpha_n)) / (3 mu + K)."""
    th = inputs.config0_material().theta_vector()
    th[2:8] = [0.5, 0.5, 0.5, 1.5, 1.5, 1.5]
    th[8:11] = [800.0, 0.25, 1.0]                 # sigma_y = 200 + 800 alpha
    rng = np.random.default_rng(1)
    B = 16
    eps = rng.normal(size=(B, 6)) * 0.01
    epn, alpn = inputs.random_history(B, 2, 0.002, 0.02)
    th_b = np.broadcast_to(th, (B, 11)).copy()
    out = M.local_update(eps, epn, alpn, th_b, "swift", np.broadcast_to(np.eye(3), (B, 3, 3)),
                         derivatives=False)
    lam, mu = M.lame(th)
    Ttr = M.elastic_stress(th_b, M.sym(eps) - M.sym(epn))
    s = Ttr - np.trace(Ttr, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3
    q = np.sqrt(1.5 * np.einsum("bij,bij->b", s, s))
    sy = 800.0 * (0.25 + alpn)
    pl = q > sy
    assert pl.sum() >= 8
    dal = np.where(pl, (q - sy) / (3 * mu + 800.0), 0.0)
    assert np.allclose(out["z"][:, 12], alpn + dal, rtol=0, atol=1e-15)
    fac = np.where(pl, 1.0 - 3 * mu * dal / q, 1.0)
    T_exp = Ttr - (1 - fac)[:, None, None] * s
    assert np.abs(M.sym(out["z"][:, :6]) - T_exp).max() < 1e-9


def _random_plastic_state(B, seed, hardening="swift"):
    mat = inputs.config0_material() if hardening == "swift" else inputs.config1_material()
    F = inputs.random_deformation_gradients(B, seed, 0.06)
    ep, al = inputs.random_history(B, seed + 1, 0.01, 0.05)
    return F, ep, al, mat.theta_vector(), hardening


@pytest.mark.parametrize("hardening", ["swift", "voce"])
def test_kuhn_tucker_incompressibility_work(hardening):
    """Eq. KT, Eq. Ep_update: dgamma >= 0, f(T, alpha) = 0 when plastic and <= 0 otherwise,
    tr(eps_p) unchanged (det G_p = 1), plastic work T : d eps_p = sigma_y d alpha."""
    F, ep, al, th, hd = _random_plastic_state(64, 10, hardening)
    o = M.gauss_point(F, ep, al, th, hd, None, jacobians=None)
    assert o["converged"].all()
    assert o["plastic"].sum() >= 32
    assert (o["dgamma"] >= 0).all()
    thb = np.broadcast_to(th, (64, 11))
    phi, _ = M.hill_phi(M.hill_tensor(thb, np.broadcast_to(np.eye(3), (64, 3, 3))), o["T"])
    sy = M.sigma_y(thb, o["h_new"][:, 6], hd)
    f = phi - SQ23 * sy
    assert np.abs(f[o["plastic"]]).max() < 1e-10 * sy.max()
    assert (f[~o["plastic"]] <= 1e-12 * sy.max()).all()
    tr_new = o["h_new"][:, :3].sum(axis=1)
    assert np.abs(tr_new - ep[:, :3].sum(axis=1)).max() < 1e-13 * np.abs(o["h_new"][:, :6]).max()
    dep = M.sym(o["h_new"][:, :6] - ep)
    work = np.einsum("bij,bij->b", o["T"], dep)
    dal = o["h_new"][:, 6] - al
    assert np.abs(work - sy * dal).max() < 1e-9 * np.abs(work).max()


def test_objectivity():
    """F -> R F leaves S, eps_p, alpha unchanged and maps P -> R P."""
    F, ep, al, th, hd = _random_plastic_state(16, 20)
    o = M.gauss_point(F, ep, al, th, hd, None, jacobians=None)
    R = scipy.linalg.expm(np.array([[0, -0.7, 0.2], [0.7, 0, -0.4], [-0.2, 0.4, 0.0]]))
    o2 = M.gauss_point(R[None] @ F, ep, al, th, hd, None, jacobians=None)
    assert np.abs(o2["S"] - o["S"]).max() < 1e-9 * np.abs(o["S"]).max()
    assert np.abs(o2["h_new"] - o["h_new"]).max() < 1e-13
    assert np.abs(o2["P"] - R[None] @ o["P"]).max() < 1e-9 * np.abs(o["P"]).max()


def _logm_sym(C):
    return 0.5 * scipy.linalg.logm(C)


def _dlog_via_expm_frechet(C, X):
    """D(1/2 log)(C)[X] without any eigen-decomposition: invert the Frechet derivative of
    the matrix exponential at L = logm(C) (scipy's Al-Mohy-Higham expm_frechet)."""
    L = np.real(scipy.linalg.logm(C))
    Mx = np.empty((9, 9))
    for q in range(9):
        E = np.zeros(9)
        E[q] = 1.0
        Mx[:, q] = scipy.linalg.expm_frechet(L, E.reshape(3, 3), compute_expm=False).ravel()
    return 0.5 * np.linalg.solve(Mx, X.ravel()).reshape(3, 3)


def _d2_half_log_block(C, X, Y):
    """Second Frechet derivative of 1/2 log at C in the directions X, Y, without an
    eigen-decomposition: the top-right block of log of the block upper-triangular matrix
    [[C, X, Y, 0], [0, C, 0, Y], [0, 0, C, X], [0, 0, 0, C]] (Higham and Relton, SIAM J.
    Matrix Anal. Appl. 35 (2014), Thm. 3.5), by scipy's inverse scaling-and-squaring logm."""
    Z = np.zeros((3, 3))
    B = np.block([[C, X, Y, Z], [Z, C, Z, Y], [Z, Z, C, X], [Z, Z, Z, C]])
    return 0.5 * np.real(scipy.linalg.logm(B)[0:3, 9:12])


@pytest.mark.parametrize("kind", ["random", "identity", "repeated", "near_repeated"])
def test_spectral_derivatives_vs_expm_frechet(kind):
    """Daleckii-Krein first derivative (P_L) equals the inverse of the Frechet derivative of
    the matrix exponential at log C (a route with no eigen-decomposition); the second
    derivative equals the block-matrix second Frechet derivative of 1/2 log (no
    eigen-decomposition either) and a central difference of the first; eps equals
    1/2 logm(C)."""
    rng = np.random.default_rng(3)
    if kind == "random":
        Fm = np.eye(3) + 0.2 * rng.uniform(-1, 1, (3, 3))
        C = Fm.T @ Fm
    elif kind == "identity":
        C = np.eye(3)
    elif kind == "repeated":
        Qr = scipy.linalg.expm(np.array([[0, .3, -.2], [-.3, 0, .5], [.2, -.5, 0.]]))
        C = Qr @ np.diag([1.1, 1.1, 0.9]) @ Qr.T
    else:
        Qr = scipy.linalg.expm(np.array([[0, .3, -.2], [-.3, 0, .5], [.2, -.5, 0.]]))
        C = Qr @ np.diag([1.1, 1.1 + 1e-9, 0.9]) @ Qr.T
    w, Q = M.eig_C(C[None])
    eps = M.log_strain(w, Q)[0]
    assert np.abs(eps - np.real(_logm_sym(C))).max() < 1e-13
    X = M.sym(rng.normal(size=6))
    Y = M.sym(rng.normal(size=6))
    d1 = M.dk1(w, Q, X[None])[0]
    d1_ref = _dlog_via_expm_frechet(C, X)
    assert np.abs(d1 - d1_ref).max() < 1e-12
    # second derivative D^2 eps[X, Y] vs central difference of D eps[X] along Y
    hd = 1e-5
    wp, Qp = M.eig_C((C + hd * Y)[None])
    wm, Qm = M.eig_C((C - hd * Y)[None])
    d2_fd = (M.dk1(wp, Qp, X[None])[0] - M.dk1(wm, Qm, X[None])[0]) / (2 * hd)
    d2 = M.dk2(w, Q, X[None], Y[None])[0]
    assert np.abs(d2 - d2_fd).max() < 1e-7 * max(1.0, np.abs(d2).max())
    assert np.abs(d2 - _d2_half_log_block(C, X, Y)).max() < 1e-12 * max(1.0, np.abs(d2).max())


@pytest.mark.parametrize("hardening", ["swift", "voce"])
def test_local_tangent_vs_fd(hardening):
    """dz/dp of App. D (implicit function theorem) equals central FD of the converged
    local update for all 24 inputs (eps, eps_p,n, alpha_n, theta)."""
    F, ep, al, th, hd = _random_plastic_state(8, 30, hardening)
    C = np.einsum("bki,bkj->bij", F, F)
    w, Q = M.eig_C(C)
    eps = M.vec6(M.log_strain(w, Q))
    B = 8
    thb = np.broadcast_to(th, (B, 11)).copy()
    Th = np.broadcast_to(np.eye(3), (B, 3, 3)).copy()
    o = M.local_update(eps, ep, al, thb, hd, Th)
    p = np.concatenate([eps, ep, al[:, None], thb], axis=1)
    for j in range(24):
        h = 1e-5 * max(abs(p[:, j]).max(), 1e-2)
        zz = []
        for s in (1, -1):
            q = p.copy()
            q[:, j] += s * h
            zz.append(M.local_update(q[:, :6], q[:, 6:12], q[:, 12], q[:, 13:], hd, Th,
                                     derivatives=False)["z"])
        fd = (zz[0] - zz[1]) / (2 * h)
        scale = np.abs(o["dz"][:, :, j]).max() + 1e-12
        assert np.abs(fd - o["dz"][:, :, j]).max() < 2e-5 * scale, j


def test_first_pk_tangent_vs_fd():
    """A = dP/dF (chain through P_L, L_L and App. D) equals central FD of P, including a
    point with two coincident principal stretches (C = I + 1e-9 perturbation)."""
    F, ep, al, th, hd = _random_plastic_state(6, 40)
    F[0] = np.diag([1.04, 0.99, 0.99])
    F[1] = np.diag([1.04, 0.99, 0.99 + 1e-9])
    o = M.gauss_point(F, ep, al, th, hd, None, jacobians="tangent")
    h = 1e-7
    for k in range(3):
        for l in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[:, k, l] += h
            Fm[:, k, l] -= h
            fd = (M.gauss_point(Fp, ep, al, th, hd, None, None)["P"] -
                  M.gauss_point(Fm, ep, al, th, hd, None, None)["P"]) / (2 * h)
            assert np.abs(fd - o["A"][..., k, l]).max() < 1e-6 * np.abs(o["A"]).max()


def test_hydrostatic_trial_stress_is_elastic_and_finite():
    """A purely volumetric strain gives a hydrostatic trial stress, which lies in the null
    space of the Hill tensor (App. A.1: p4..p6 make H deviatoric), so phi = 0 and the point is
    elastic (Eq. KT) at any pressure.  In rotated frames T : H : T rounds to small negative
    values in about half the cases; phi must still come out finite (0), never NaN."""
    th = inputs.config0_material().theta_vector()
    B = 200
    rng = np.random.default_rng(0)
    Th = np.stack([inputs.random_rotation(s) for s in range(B)])
    mag = 10.0 ** rng.uniform(-4.0, -1.0, B) * rng.choice([-1.0, 1.0], B)
    eps = np.zeros((B, 6))
    eps[:, :3] = mag[:, None]
    thb = np.tile(th, (B, 1))
    Hg = M.hill_tensor(thb, Th)
    T = M.elastic_stress(thb, M.sym(eps))
    phi, _ = M.hill_phi(Hg, T)
    assert np.all(np.isfinite(phi))
    assert np.all(phi <= 1e-6 * np.abs(T).max(axis=(1, 2)))   # sqrt of the rounding of T:H:T
    o = M.local_update(eps, np.zeros((B, 6)), np.zeros(B), thb, "swift", Th, derivatives=False)
    assert np.all(np.isfinite(o["ftr"])) and not o["plastic"].any()
    lam, mu = M.lame(th)
    assert np.allclose(o["z"][:, 0], (3.0 * lam + 2.0 * mu) * mag, rtol=1e-13, atol=0.0)
