"""Oracle, one Gauss point: finite-strain Hill-48 plasticity in logarithmic strain space.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain FP64 numpy, vectorised over a
leading batch of independent Gauss points and nothing else.

Formulation followed (paper Sec. 2.2.2-2.2.3, App. A-D):
* geometric pre-processor: C = F^T F, eps = 1/2 ln C by the spectral decomposition of C
  (Eq. c_decomp);
* log-space linear elasticity T = E : (eps - eps_p) with isotropic E (Eq. T);
* Hill-48 effective stress phi = sqrt(T : H : T) with the local H from p1..p9 and the
  rotation H_g = Theta Theta : H_l : Theta^T Theta^T (Eq. Phi_hill, App. A.1);
* yield function f = phi(T) - sqrt(2/3) sigma_y(alpha) and alpha-rate sqrt(2/3) gamma-rate
  (reading R1: this places the sqrt(2/3) so that r11 = sigma^y_11 / sigma_0 holds, App. A.1),
  hardening Swift sigma_y = K (eps0 + alpha)^n or Voce sigma_y = sigma0 + Q (1 - exp(-b alpha));
* elastic predictor (Eq. Tr_stress) and closest-point projection on y = [T, alpha, dgamma]
  (Eq. local_cpp) by Newton (Eq. local_solver) with the Scherzinger line search (App. B,
  Algorithm local_cpp of App. C); J^G is the complex-step Jacobian of G, exact to rounding,
  standing in for the paper's automatic differentiation;
* recovery eps_p,n+1 = eps_p,n + dgamma N, T = E : (eps - eps_p,n+1) (App. C);
* implicit differentiation of the converged local solve (App. D): ydot = -J_y^{-1} G_p pdot,
  zdot = dz/dy ydot + dz/dp pdot, with the partials by complex step;
* geometric post-processor S = P_L : T, P = F S (Eq. proj_lagrange, Eq. pk_stress), with
  P_L = 2 d eps/dC and L_L = 4 d^2 eps / dC^2 applied through the first and second
  Daleckii-Krein divided-difference formulas in the eigenbasis of C (Sec. 2.2.5).

Symmetric tensors are stored as 6 independent components in the order (11,22,33,12,23,13);
a derivative "with respect to component 12" moves T_12 and T_21 together.  The material
parameter vector is theta = (E, nu, F, G, H, L, M, N, h1, h2, h3) where (h1,h2,h3) =
(K, eps0, n) for Swift and (sigma0, Q, b) for Voce.
"""
from __future__ import annotations

import numpy as np

SQ23 = np.sqrt(2.0 / 3.0)
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]
N_THETA = 11

# local return-mapping controls (reading R8, App. B constants)
LOCAL_TOL = 1e-13
LOCAL_KMAX = 50
LS_JMAX = 10
LS_BETA = 1e-4
LS_ETA = 0.1
CS_H = 1e-30      # complex-step size


# ----------------------------------------------------------------------------- tensors
def sym(v):
    """(..., 6) components -> (..., 3, 3) symmetric tensor."""
    v = np.asarray(v)
    m = np.zeros(v.shape[:-1] + (3, 3), dtype=v.dtype)
    for q, (i, j) in enumerate(PAIRS):
        m[..., i, j] = v[..., q]
        m[..., j, i] = v[..., q]
    return m


def vec6(m):
    """(..., 3, 3) -> (..., 6) components (upper triangle, order 11,22,33,12,23,13)."""
    return np.stack([m[..., i, j] for (i, j) in PAIRS], axis=-1)


def ddot(a, b):
    return np.einsum("...ij,...ij->...", a, b)


# ----------------------------------------------------------------------- constitutive
def hill_tensor(theta, Theta):
    """Global Hill tensor H_g (..., 3,3,3,3) from (F,G,H,L,M,N) = theta[..., 2:8].

    App. A.1: r11 = 1/sqrt(G+H), r22 = 1/sqrt(F+H), r33 = 1/sqrt(F+G), r12 = sqrt(3/(2N)),
    r23 = sqrt(3/(2L)), r13 = sqrt(3/(2M)) (reading R2); p1..p3 = 2/(3 r_ii^2),
    p7 = 1/r12^2, p8 = 1/r23^2, p9 = 1/r13^2, p4 = (p3-p1-p2)/2, p5 = (p1-p2-p3)/2,
    p6 = (p2-p1-p3)/2.  The shear entries 1/2 p7 etc. are tensor components
    H_1212 = H_1221 = H_2112 = H_2121 = p7/2 (reading R3).  Rotation (reading R4):
    H_g,ijkl = Theta_ia Theta_jb Theta_kc Theta_ld H_l,abcd.
    """
    Fh, Gh, Hh, Lh, Mh, Nh = (theta[..., k] for k in range(2, 8))
    r11 = 1.0 / np.sqrt(Gh + Hh)
    r22 = 1.0 / np.sqrt(Fh + Hh)
    r33 = 1.0 / np.sqrt(Fh + Gh)
    r12 = np.sqrt(3.0 / (2.0 * Nh))
    r23 = np.sqrt(3.0 / (2.0 * Lh))
    r13 = np.sqrt(3.0 / (2.0 * Mh))
    p1 = 2.0 / (3.0 * r11 ** 2)
    p2 = 2.0 / (3.0 * r22 ** 2)
    p3 = 2.0 / (3.0 * r33 ** 2)
    p7 = 1.0 / r12 ** 2
    p8 = 1.0 / r23 ** 2
    p9 = 1.0 / r13 ** 2
    p4 = 0.5 * (p3 - p1 - p2)
    p5 = 0.5 * (p1 - p2 - p3)
    p6 = 0.5 * (p2 - p1 - p3)
    shape = np.shape(p1)
    Hl = np.zeros(shape + (3, 3, 3, 3), dtype=np.result_type(p1, float))
    Hl[..., 0, 0, 0, 0] = p1
    Hl[..., 1, 1, 1, 1] = p2
    Hl[..., 2, 2, 2, 2] = p3
    Hl[..., 0, 0, 1, 1] = p4
    Hl[..., 1, 1, 0, 0] = p4
    Hl[..., 1, 1, 2, 2] = p5
    Hl[..., 2, 2, 1, 1] = p5
    Hl[..., 0, 0, 2, 2] = p6
    Hl[..., 2, 2, 0, 0] = p6
    for (i, j), p in (((0, 1), p7), ((1, 2), p8), ((0, 2), p9)):
        for (a, b) in ((i, j), (j, i)):
            for (c, d) in ((i, j), (j, i)):
                Hl[..., a, b, c, d] = 0.5 * p
    Th = np.asarray(Theta, dtype=np.float64)
    if np.array_equal(Th, np.broadcast_to(np.eye(3), Th.shape)):
        return Hl
    # one index at a time (the same contraction as the four-fold product)
    Hg = np.einsum("...ia,...abcd->...ibcd", Th, Hl)
    Hg = np.einsum("...jb,...ibcd->...ijcd", Th, Hg)
    Hg = np.einsum("...kc,...ijcd->...ijkd", Th, Hg)
    return np.einsum("...ld,...ijkd->...ijkl", Th, Hg)


def lame(theta):
    E, nu = theta[..., 0], theta[..., 1]
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elastic_stress(theta, ee):
    """Eq. T with isotropic E (reading R5): T = lambda tr(ee) I + 2 mu ee, ee (...,3,3)."""
    lam, mu = lame(theta)
    tr = np.trace(ee, axis1=-2, axis2=-1)
    return lam[..., None, None] * tr[..., None, None] * np.eye(3) + 2.0 * mu[..., None, None] * ee


def sigma_y(theta, alpha, hardening):
    """Swift K (eps0 + alpha)^n or Voce sigma0 + Q (1 - exp(-b alpha)) (Eq. Hard, reading R1)."""
    h1, h2, h3 = theta[..., 8], theta[..., 9], theta[..., 10]
    if hardening == "swift":
        return h1 * (h2 + alpha) ** h3
    if hardening == "voce":
        return h1 + h2 * (1.0 - np.exp(-h3 * alpha))
    raise ValueError(hardening)


def hill_phi(Hg, T):
    """phi = sqrt(T : H : T) (Eq. Phi_hill) and H : T.  H is positive semi-definite with the
    hydrostatic direction in its null space, so T : H : T >= 0; near a hydrostatic T the sum
    can round slightly below zero, and is then taken as 0 (real part compared, so that a
    complex-step argument keeps its imaginary part elsewhere)."""
    HT = np.einsum("...ijkl,...kl->...ij", Hg, T)
    q = ddot(T, HT)
    q = np.where(np.real(q) > 0.0, q, 0.0 * q)
    return np.sqrt(q), HT


def local_residual(y, eps, epn, alpn, theta, hardening, Theta):
    """G(y) of Eq. local_cpp for y = [T (6), alpha, dgamma]; every argument batched (B, ...).

    G_T = T - E : (eps - eps_p,n - dgamma N(T)),  N = H:T / phi  (Eq. ep_evol)
    G_a = alpha - alpha_n - W dgamma,  W = sqrt(2/3)  (Eq. alpha_update)
    G_f = phi(T) - sqrt(2/3) sigma_y(alpha)          (Eq. yield_final, reading R1)
    """
    T = sym(y[..., :6])
    alpha = y[..., 6]
    dgam = y[..., 7]
    Hg = hill_tensor(theta, Theta)
    phi, HT = hill_phi(Hg, T)
    N = HT / phi[..., None, None]
    ee = sym(eps) - sym(epn) - dgam[..., None, None] * N
    GT = vec6(T - elastic_stress(theta, ee))
    Ga = alpha - alpn - SQ23 * dgam
    Gf = phi - SQ23 * sigma_y(theta, alpha, hardening)
    return np.concatenate([GT, Ga[..., None], Gf[..., None]], axis=-1)


def recover(y, eps, epn, alpn, theta, hardening, Theta):
    """z = (T_{n+1} (6), eps_p,{n+1} (6), alpha_{n+1}) from the converged y (App. C)."""
    T = sym(y[..., :6])
    Hg = hill_tensor(theta, Theta)
    phi, HT = hill_phi(Hg, T)
    N = HT / phi[..., None, None]
    epnew = sym(epn) + y[..., 7][..., None, None] * N
    Tn = elastic_stress(theta, sym(eps) - epnew)
    return np.concatenate([vec6(Tn), vec6(epnew), y[..., 6][..., None]], axis=-1)


def recover_elastic(eps, epn, alpn, theta):
    """z for an accepted elastic predictor: (E : (eps - eps_p,n), eps_p,n, alpha_n)."""
    T = elastic_stress(theta, sym(eps) - sym(epn))
    return np.concatenate([vec6(T), epn, alpn[..., None]], axis=-1)


def complex_step_jacobian(fun, x, nout):
    """d fun / d x (B, nout, nx) by complex step: Im fun(x + i h e_j) / h."""
    B, nx = x.shape
    J = np.empty((B, nout, nx))
    for j in range(nx):
        xc = x.astype(np.complex128)
        xc[:, j] += 1j * CS_H
        J[:, :, j] = np.imag(fun(xc)) / CS_H
    return J


def _scaled_norm(G, sref):
    s = np.concatenate([G[..., :6] / sref[..., None], G[..., 6:7],
                        G[..., 7:8] / sref[..., None]], axis=-1)
    return np.sqrt(np.sum(s * s, axis=-1))


def closest_point_projection(eps, epn, alpn, theta, hardening, Theta):
    """Plastic corrector (App. C, Algorithm local_cpp) for a batch of plastic points.

    Newton on G(y) = 0 from y0 = [T_tr, alpha_n, 0] (reading R7), line search of App. B
    (reading R9: the first quadratic-model step is tested before it is updated; on
    exhaustion the last step length is taken).  Returns (y, iterations, converged).
    """
    B = eps.shape[0]

    def G_of(yy, idx):
        return local_residual(yy, eps[idx], epn[idx], alpn[idx], theta[idx], hardening,
                              Theta[idx])

    Ttr = vec6(elastic_stress(theta, sym(eps) - sym(epn)))
    y = np.concatenate([Ttr, alpn[:, None], np.zeros((B, 1))], axis=1)
    # stress scale of the convergence test (reading R8): the rounding floor of G_T grows
    # with the trial stress, so the larger of sigma_y(alpha_n) and |T_tr| is used
    sref = np.maximum(sigma_y(theta, alpn, hardening), np.sqrt(np.sum(Ttr * Ttr, axis=-1)))
    iters = np.zeros(B, dtype=np.int64)
    conv = np.zeros(B, dtype=bool)
    active = np.arange(B)
    for k in range(LOCAL_KMAX + 1):
        G = G_of(y[active], active)
        done = _scaled_norm(G, sref[active]) <= LOCAL_TOL
        conv[active[done]] = True
        active = active[~done]
        G = G[~done]
        if active.size == 0 or k == LOCAL_KMAX:
            break
        iters[active] += 1
        idx = active
        J = complex_step_jacobian(lambda yy: G_of(yy, idx), y[active], 8)
        dy = np.linalg.solve(J, -G[..., None])[..., 0]
        psi0 = 0.5 * np.sum(G * G, axis=1)
        G1 = G_of(y[active] + dy, active)
        psi1 = 0.5 * np.sum(G1 * G1, axis=1)
        zeta = np.ones(active.size)
        need = np.nonzero(~(psi1 < (1.0 - 2.0 * LS_BETA) * psi0))[0]   # Eq. goldstein_full
        if need.size:
            z = psi0[need] / (psi0[need] + psi1[need])                    # Eq. alpha_init
            open_ = np.ones(need.size, dtype=bool)
            for _ in range(LS_JMAX + 1):
                m = need[open_]
                Gz = G_of(y[active[m]] + z[open_, None] * dy[m], active[m])
                psiz = 0.5 * np.sum(Gz * Gz, axis=1)
                ok = psiz < (1.0 - 2.0 * LS_BETA * z[open_]) * psi0[m]    # Eq. goldstein_full
                znew = psi0[m] / (psi0[m] + psiz)                           # Eq. alpha_update_ls
                zo = z[open_]
                z[open_] = np.where(ok, zo, np.maximum(LS_ETA * zo, znew))  # Eq. alpha_safeguard
                open_[np.nonzero(open_)[0][ok]] = False
                if not open_.any():
                    break
            zeta[need] = z
        y[active] = y[active] + zeta[:, None] * dy
    return y, iters, conv


def local_update(eps, epn, alpn, theta, hardening, Theta, derivatives=True):
    """Stress update of Algorithm global_stress_update (App. C), steps 2-6.

    Inputs (batched, B): eps (B,6), epn (B,6), alpn (B,), theta (B,11), Theta (B,3,3).
    Returns a dict with z = (T, eps_p,n+1, alpha_n+1) (B,13), dgamma, plastic flags,
    local iteration counts, and (if derivatives) dz/dp (B,13,24) for p = (eps, eps_p,n,
    alpha_n, theta) by implicit differentiation (App. D).
    """
    B = eps.shape[0]
    Ttr = elastic_stress(theta, sym(eps) - sym(epn))
    Hg = hill_tensor(theta, Theta)
    phi_tr, _ = hill_phi(Hg, Ttr)
    ftr = phi_tr - SQ23 * sigma_y(theta, alpn, hardening)
    plastic = ftr > 0.0                      # reading R10: f_tr <= 0 is elastic
    z = recover_elastic(eps, epn, alpn, theta)
    dgam = np.zeros(B)
    iters = np.zeros(B, dtype=np.int64)
    conv = np.ones(B, dtype=bool)
    P = np.nonzero(plastic)[0]
    if P.size:
        y, it, cv = closest_point_projection(eps[P], epn[P], alpn[P], theta[P], hardening,
                                             Theta[P])
        z[P] = recover(y, eps[P], epn[P], alpn[P], theta[P], hardening, Theta[P])
        dgam[P] = y[:, 7]
        iters[P] = it
        conv[P] = cv
    out = dict(z=z, dgamma=dgam, plastic=plastic, iters=iters, converged=conv, ftr=ftr)
    if not derivatives:
        return out
    p_all = np.concatenate([eps, epn, alpn[:, None], theta], axis=1)   # (B, 24)
    dz = np.empty((B, 13, 24))
    E_ = np.nonzero(~plastic)[0]
    if E_.size:
        def zel(pc):
            return recover_elastic(pc[:, 0:6], pc[:, 6:12], pc[:, 12], pc[:, 13:24])
        dz[E_] = complex_step_jacobian(zel, p_all[E_], 13)
    if P.size:
        pP = p_all[P]
        ThP = Theta[P]

        def G_y(yy):
            return local_residual(yy, pP[:, 0:6], pP[:, 6:12], pP[:, 12], pP[:, 13:24],
                                  hardening, ThP)

        def G_p(pc):
            return local_residual(y.astype(pc.dtype), pc[:, 0:6], pc[:, 6:12], pc[:, 12],
                                  pc[:, 13:24], hardening, ThP)

        def z_y(yy):
            return recover(yy, pP[:, 0:6], pP[:, 6:12], pP[:, 12], pP[:, 13:24], hardening, ThP)

        def z_p(pc):
            return recover(y.astype(pc.dtype), pc[:, 0:6], pc[:, 6:12], pc[:, 12],
                           pc[:, 13:24], hardening, ThP)

        Jy = complex_step_jacobian(G_y, y, 8)           # J_y (App. D)
        Gp = complex_step_jacobian(G_p, pP, 8)          # dG/dp
        ydot = -np.linalg.solve(Jy, Gp)                 # (B, 8, 24)
        dz[P] = complex_step_jacobian(z_y, y, 13) @ ydot + complex_step_jacobian(z_p, pP, 13)
        out["Jy"] = Jy
    out["dz"] = dz
    return out


# ------------------------------------------------------------------ spectral functions
def f_log(lam):
    return 0.5 * np.log(lam)


def f1(a, b):
    """First divided difference of f(l) = 1/2 ln l: (f(a) - f(b)) / (a - b), limit f'(a).
    Written as 1/2 log1p(d/b)/d, the same quantity without cancellation."""
    d = a - b
    x = d / b
    small = np.abs(x) < 1e-12
    xs = np.where(small, 1.0, x)
    val = np.where(small, (0.5 / b) * (1.0 - 0.5 * x), 0.5 * np.log1p(xs) / np.where(small, 1.0, d))
    return val


def f2(a, b, c):
    """Second divided difference f[a,b,c] of f(l) = 1/2 ln l (symmetric in its arguments).

    Sorted s1 <= s2 <= s3: (f[s3,s2] - f[s2,s1]) / (s3 - s1); when all three coincide to
    1e-5 relative, the limit f''(m)/2 at the mean m (first-order term vanishes at the mean).
    """
    a, b, c = np.broadcast_arrays(a, b, c)
    s = np.sort(np.stack([a, b, c], axis=-1), axis=-1)
    s1, s2, s3 = s[..., 0], s[..., 1], s[..., 2]
    m = (s1 + s2 + s3) / 3.0
    spread = s3 - s1
    close = spread <= 1e-5 * m
    den = np.where(close, 1.0, spread)
    gen = (f1(s3, s2) - f1(s2, s1)) / den
    lim = -0.25 / (m * m)                      # f''(m)/2 with f'' = -1/(2 l^2)
    return np.where(close, lim, gen)


def eig_C(C):
    w, Q = np.linalg.eigh(C)
    return w, Q


def log_strain(w, Q):
    """eps = sum_a 1/2 ln(lambda_a) n_a (x) n_a (Eq. c_decomp)."""
    return np.einsum("...ia,...a,...ja->...ij", Q, f_log(w), Q)


def dk1(w, Q, X):
    """D eps(C)[X]: first-order Daleckii-Krein formula Q (f[l_a,l_b] * (Q^T X Q)_ab) Q^T."""
    Xh = np.einsum("...ia,...ij,...jb->...ab", Q, X, Q)
    F1 = f1(w[..., :, None], w[..., None, :])
    return np.einsum("...ia,...ab,...jb->...ij", Q, F1 * Xh, Q)


def dk2(w, Q, X, Y):
    """D^2 eps(C)[X, Y]: second-order Daleckii-Krein formula
    Q ( sum_c f[l_a,l_c,l_b] (Xh_ac Yh_cb + Yh_ac Xh_cb) ) Q^T."""
    Xh = np.einsum("...ia,...ij,...jb->...ab", Q, X, Q)
    Yh = np.einsum("...ia,...ij,...jb->...ab", Q, Y, Q)
    F2 = f2(w[..., :, None, None], w[..., None, :, None], w[..., None, None, :])  # [a,c,b]
    M = np.einsum("...acb,...ac,...cb->...ab", F2, Xh, Yh) + \
        np.einsum("...acb,...ac,...cb->...ab", F2, Yh, Xh)
    return np.einsum("...ia,...ab,...jb->...ij", Q, M, Q)


# ------------------------------------------------------------------ full Gauss point
def gauss_point(F, epn, alpn, theta, hardening, Theta=None, jacobians="tangent", local=None):
    """Algorithm global_stress_update (App. C) plus the first Piola-Kirchhoff tangent.

    F (B,3,3); epn (B,6); alpn (B,); theta (11,) or (B,11); Theta None, (3,3) or (B,3,3).
    jacobians: None (P and history only), "tangent" (also A = dP/dF), or "all" (also
    dP/dh_old, dP/dtheta, dh/dF, dh/dh_old, dh/dtheta for the adjoint).
    History h = (eps_p (6), alpha).  local: None for the Hill-48 update, or another model's
    strain-driven update (eps, epn, alpn, derivatives) -> dict(z, dz, ...) with dz over
    (eps, eps_p,n, alpha_n) (e.g. barlat.local); theta, hardening and Theta are then unused,
    and jacobians "all" needs a model that declares `n_params` and returns the parameter
    columns of dz (dP/dtheta and dh/dtheta then run over that model's parameters).
    """
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    theta = np.broadcast_to(np.asarray(theta, dtype=np.float64), (B, N_THETA)).copy()
    if Theta is None:
        Theta = np.eye(3)
    Theta = np.broadcast_to(np.asarray(Theta, dtype=np.float64), (B, 3, 3)).copy()
    C = np.einsum("bki,bkj->bij", F, F)
    w, Q = eig_C(C)
    eps = vec6(log_strain(w, Q))
    if local is None:
        lu = local_update(eps, np.asarray(epn, float), np.asarray(alpn, float), theta, hardening,
                          Theta, derivatives=jacobians is not None)
    else:
        if jacobians == "all" and not hasattr(local, "n_params"):
            raise NotImplementedError("this local model provides no parameter derivatives")
        extra = {"param_derivatives": True} if jacobians == "all" else {}
        lu = local(eps, np.asarray(epn, float), np.asarray(alpn, float), derivatives=jacobians is not None, **extra)
    z = lu["z"]
    T = sym(z[:, :6])
    S = 2.0 * dk1(w, Q, T)                       # S = P_L : T   (Eq. proj_lagrange)
    P = F @ S                                    # P = F S       (Eq. pk_stress)
    h_new = z[:, 6:13]
    J = np.linalg.det(F)
    sigma = P @ np.swapaxes(F, 1, 2) / J[:, None, None]
    out = dict(P=P, S=S, T=T, h_new=h_new, eps=eps, sigma=sigma, dgamma=lu["dgamma"],
               plastic=lu["plastic"], iters=lu["iters"], converged=lu["converged"],
               ftr=lu["ftr"])
    if jacobians is None:
        return out
    dz = lu["dz"]
    # A = dP/dF, direction by direction (chain rule through C, eps, the local update, S)
    A = np.empty((B, 3, 3, 3, 3))
    dh_dF = np.empty((B, 7, 3, 3))
    for k in range(3):
        for l in range(3):
            dF = np.zeros((B, 3, 3))
            dF[:, k, l] = 1.0
            dC = np.swapaxes(dF, 1, 2) @ F + np.swapaxes(F, 1, 2) @ dF
            deps = vec6(dk1(w, Q, dC))
            dzk = np.einsum("bij,bj->bi", dz[:, :, 0:6], deps)
            dT = sym(dzk[:, :6])
            dS = 2.0 * dk1(w, Q, dT) + 2.0 * dk2(w, Q, T, dC)
            A[:, :, :, k, l] = dF @ S + F @ dS
            dh_dF[:, :, k, l] = dzk[:, 6:13]
    out["A"] = A
    out["dh_dF"] = dh_dF
    if jacobians == "tangent":
        return out

    def through_T(dzcols):          # dP for an input that enters only through z
        n = dzcols.shape[-1]
        dP = np.empty((B, 3, 3, n))
        for j in range(n):
            dT = sym(dzcols[:, :6, j])
            dP[..., j] = F @ (2.0 * dk1(w, Q, dT))
        return dP

    out["dP_dh"] = through_T(dz[:, :, 6:13])
    out["dh_dh"] = dz[:, 6:13, 6:13]
    out["dP_dtheta"] = through_T(dz[:, :, 13:])
    out["dh_dtheta"] = dz[:, 6:13, 13:]
    return out


def von_mises(sigma):
    s = sigma - np.trace(sigma, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
    return np.sqrt(1.5 * ddot(s, s))
