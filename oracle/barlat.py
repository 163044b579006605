"""Oracle, Barlat Yld2004-18p yield function and the closest-point projection driven by a
trial stress (Eq. Phi_barlat, App. A.2, Eq. local_cpp, App. B, App. C).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain FP64 numpy, vectorised over a
leading batch of independent material points and nothing else.

* phi(T) = [1/4 sum_ij |s'_i - s''_j|^m]^(1/m), s'_i and s''_j the eigenvalues of
  s' = C' : P : T_l and s'' = C'' : P : T_l (Eq. Phi_barlat), with P the deviatoric projector
  and C', C'' the 6x6 matrices of App. A.2 acting on tensor components in the order
  (11, 22, 33, 12, 23, 13): c44, c55, c66 scale the 12, 23, 13 shear components (reading R17).
  T_l = Theta^T T Theta is the stress in the material frame (the columns of Theta are the
  material axes); eigenvalues do not depend on the frame, so this is the paper's rotation of
  C', C'' into the global frame.  `phi_eig` evaluates this definition with eigenvalues.
* For an even integer m the double sum is a polynomial in power traces,
  sum_ij (a_i - b_j)^m = sum_k binom(m, k) (-1)^(m-k) tr(A^k) tr(B^(m-k)),
  evaluated after shifting A and B by the same multiple of I (the sum only sees
  differences a_i - b_j), which keeps the alternating sum well conditioned.  `phi_poly` and
  its gradient `flow` (N = dphi/dT, Eq. ep_evol) need no eigenvalues and take complex
  arguments, so the Jacobian of G follows by complex step.
* `cpp` solves G(y) = 0 for y = [T (6), alpha, dgamma] (Eq. local_cpp) with
  G_T = T - T_tr + dgamma E : N(T), G_alpha = alpha - alpha_n - W dgamma with W = 1 for this
  model (Eq. alpha_update), G_f = phi(T) - sigma_y(alpha) (Eq. yield_final); E isotropic
  (E, nu) or orthotropic from nine coefficients in the material frame (`orthotropic_tensor`).
  Newton (Eq. local_solver) from y0 = [T_tr, alpha_n, 0] (reading R7), optionally with the
  line search of App. B (Goldstein test Eq. goldstein_full, quadratic model Eq. alpha_init and
  Eq. alpha_update_ls, safeguard Eq. alpha_safeguard; reading R9 on the order), converged
  when the scaled residual norm of reading R8 is <= tol.
* `cpp_tangent` gives dT/dT_tr at the converged point by implicit differentiation (App. D):
  J_G dy = [dT_tr; 0; 0].

Parity pins (tests/test_oracle_barlat.py): phi_poly against phi_eig; flow against central
differences of phi_eig; the isotropic reductions (all 18 coefficients 1: von Mises for
m = 2 and m = 4, uniaxial and pure-shear closed forms for any even m); homogeneity and
pressure insensitivity; the von Mises radial return in closed form; the projection against
a direct minimisation of the complementary energy over the yield set; the paper's printed
step length of the third line-search iteration (App. B).
"""
from __future__ import annotations

from math import comb

import numpy as np

from .material import LS_BETA, LS_ETA, LS_JMAX, LOCAL_TOL, _scaled_norm, complex_step_jacobian

VOIGT = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))
W_SHEAR = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])    # X : Y = sum_a w_a X_a Y_a

# deviatoric projector on tensor components (App. A.2)
P_DEV = np.array([[2, -1, -1, 0, 0, 0], [-1, 2, -1, 0, 0, 0], [-1, -1, 2, 0, 0, 0],
                  [0, 0, 0, 3, 0, 0], [0, 0, 0, 0, 3, 0], [0, 0, 0, 0, 0, 3]], dtype=np.float64) / 3.0


def transform_matrix(c):
    """The 6x6 matrix of App. A.2 from (c12, c13, c21, c23, c31, c32, c44, c55, c66)."""
    c12, c13, c21, c23, c31, c32, c44, c55, c66 = c
    C = np.zeros((6, 6), dtype=np.result_type(*c, np.float64))   # complex coefficients allowed
    C[0, 1], C[0, 2] = -c12, -c13
    C[1, 0], C[1, 2] = -c21, -c23
    C[2, 0], C[2, 1] = -c31, -c32
    C[3, 3], C[4, 4], C[5, 5] = c44, c55, c66
    return C


def voigt(T):
    """(..., 3, 3) -> (..., 6) components in the order (11, 22, 33, 12, 23, 13)."""
    return np.stack([T[..., i, j] for i, j in VOIGT], axis=-1)


def tensor(v):
    """(..., 6) components -> symmetric (..., 3, 3)."""
    T = np.zeros(v.shape[:-1] + (3, 3), dtype=v.dtype)
    for a, (i, j) in enumerate(VOIGT):
        T[..., i, j] = v[..., a]
        T[..., j, i] = v[..., a]
    return T


class Barlat:
    """Yld2004-18p with coefficients c1 = C' and c2 = C'' (9 each), even integer m, optional
    material frame Theta (3x3, columns = material axes)."""

    def __init__(self, c1, c2, m, Theta=None):
        self.c1 = np.asarray(c1)
        self.c2 = np.asarray(c2)
        self.C1 = transform_matrix(c1)
        self.C2 = transform_matrix(c2)
        self.m = int(m)
        if self.m != m or self.m < 2 or self.m % 2:
            raise ValueError("the power-trace form needs an even integer exponent m >= 2")
        self.Theta = np.eye(3) if Theta is None else np.asarray(Theta, dtype=np.float64)

    def transformed(self, T):
        """s' and s'' (..., 3, 3) for stress components T (..., 6) in the global frame."""
        Tg = tensor(T)
        Tl = np.swapaxes(self.Theta, -1, -2) @ Tg @ self.Theta
        s = voigt(Tl) @ P_DEV.T
        return tensor(s @ self.C1.T), tensor(s @ self.C2.T)

    # -- the definition -------------------------------------------------------------------
    def phi_eig(self, T):
        A, B = self.transformed(np.asarray(T, dtype=np.float64))
        a = np.linalg.eigvalsh(A)
        b = np.linalg.eigvalsh(B)
        S = np.sum(np.abs(a[..., :, None] - b[..., None, :]) ** self.m, axis=(-2, -1))
        return (0.25 * S) ** (1.0 / self.m)

    # -- the polynomial form (complex arguments allowed) --------------------------------
    def _shifted_powers(self, T):
        A, B = self.transformed(T)
        c = (np.trace(A, axis1=-2, axis2=-1) + np.trace(B, axis1=-2, axis2=-1)) / 6.0
        I = np.eye(3)
        A = A - c[..., None, None] * I
        B = B - c[..., None, None] * I
        PA = [np.broadcast_to(I, A.shape).astype(A.dtype)]
        PB = [np.broadcast_to(I, B.shape).astype(B.dtype)]
        for _ in range(self.m):
            PA.append(PA[-1] @ A)
            PB.append(PB[-1] @ B)
        tA = [np.trace(X, axis1=-2, axis2=-1) for X in PA]
        tB = [np.trace(X, axis1=-2, axis2=-1) for X in PB]
        return PA, PB, tA, tB

    def _S(self, tA, tB):
        m = self.m
        return sum(comb(m, k) * (-1) ** (m - k) * tA[k] * tB[m - k] for k in range(m + 1))

    def phi_poly(self, T):
        _, _, tA, tB = self._shifted_powers(T)
        return (0.25 * self._S(tA, tB)) ** (1.0 / self.m)

    def flow(self, T):
        """(N, phi): N = dphi/dT as tensor components (..., 6), dphi = N : dT.

        dS = sum_k binom(m,k)(-1)^(m-k) [k tr(B^(m-k)) A^(k-1) : dA + (m-k) tr(A^k) B^(m-k-1) : dB]
        with dA = C' P dT_l and dB = C'' P dT_l (the shift is a fixed multiple of I here: S does
        not change with it), dT_l = Theta^T dT Theta; phi = (S/4)^(1/m)."""
        m = self.m
        PA, PB, tA, tB = self._shifted_powers(T)
        S = self._S(tA, tB)
        GA = sum(comb(m, k) * (-1) ** (m - k) * k * tB[m - k][..., None, None] * PA[k - 1]
                 for k in range(1, m + 1))
        GB = sum(comb(m, k) * (-1) ** (m - k) * (m - k) * tA[k][..., None, None] * PB[m - k - 1]
                 for k in range(0, m))
        # X : tensor(C v) = (w X_voigt) . (C v) with v = P voigt(dT_l)
        gl = (voigt(GA) * W_SHEAR) @ self.C1 @ P_DEV + (voigt(GB) * W_SHEAR) @ self.C2 @ P_DEV
        Nl = tensor(gl / W_SHEAR)                                   # dS/dT_l as a tensor
        Ng = self.Theta @ Nl @ np.swapaxes(self.Theta, -1, -2)       # back to the global frame
        phi = (0.25 * S) ** (1.0 / m)
        return voigt(Ng) * (0.25 / m) * phi[..., None] ** (1 - m), phi


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def orthotropic_tensor(d, Theta=None):
    """The fourth-order elasticity tensor (3, 3, 3, 3) from nine stiffness coefficients in the
    material frame (Eq. T; reading R22): d = (E1111, E2222, E3333, E1122, E1133, E2233, E1212,
    E2323, E1313) with the minor and major symmetries, rotated into the global frame as
    E_g,ijkl = Theta_ia Theta_jb Theta_kc Theta_ld E_l,abcd (columns of Theta = material axes)."""
    d1, d2, d3, d4, d5, d6, d7, d8, d9 = d
    El = np.zeros((3, 3, 3, 3))
    El[0, 0, 0, 0], El[1, 1, 1, 1], El[2, 2, 2, 2] = d1, d2, d3
    for (a, b), v in (((0, 1), d4), ((0, 2), d5), ((1, 2), d6)):
        El[a, a, b, b] = El[b, b, a, a] = v
    for (a, b), v in (((0, 1), d7), ((1, 2), d8), ((0, 2), d9)):
        El[a, b, a, b] = El[a, b, b, a] = El[b, a, a, b] = El[b, a, b, a] = v
    Q = np.eye(3) if Theta is None else np.asarray(Theta, dtype=np.float64)
    return np.einsum("ia,jb,kc,ld,abcd->ijkl", Q, Q, Q, Q, El)


def elastic(E, nu, e):
    """E : e on tensor components: isotropic lambda tr(e) I + 2 mu e for a number E (with nu),
    or the contraction with a fourth-order tensor E (3, 3, 3, 3) (nu unused)."""
    if np.ndim(E) == 4:
        return voigt(np.einsum("ijkl,...kl->...ij", E, tensor(e)))
    lam, mu = lame(E, nu)
    out = 2 * mu * e
    out[..., :3] += lam * np.sum(e[..., :3], axis=-1, keepdims=True)
    return out


def sigma_y(hardening, h, alpha):
    """Swift K (eps0 + alpha)^n, or Voce as Eq. Hard prints it, sigma0 + sqrt(2/3) Q
    (1 - exp(-b alpha)) (W = 1 and f = phi - sigma_y for this model; reading R19); perfect
    plasticity is Voce with Q = 0."""
    if hardening == "swift":
        K, e0, n = h
        return K * (e0 + alpha) ** n
    s0, Q, b = h
    return s0 + np.sqrt(2.0 / 3.0) * Q * (1.0 - np.exp(-b * alpha))


def residual(model, E, nu, hardening, h, y, Ttr, alpn):
    """G(y) of Eq. local_cpp for y = [T (6), alpha, dgamma] (..., 8)."""
    N, phi = model.flow(y[..., :6])
    GT = y[..., :6] - Ttr + y[..., 7:8] * elastic(E, nu, N)
    Ga = y[..., 6] - alpn - y[..., 7]
    Gf = phi - sigma_y(hardening, h, y[..., 6])
    return np.concatenate([GT, Ga[..., None], Gf[..., None]], axis=-1)


def cpp(model, E, nu, hardening, h, Ttr, alpn, line_search=True, kmax=40, tol=LOCAL_TOL,
        beta=LS_BETA, eta=LS_ETA, jmax=LS_JMAX, trace=None):
    """Plastic corrector for a batch of trial stresses Ttr (B, 6) with alpha_n (B,).

    Returns (y (B, 8), iterations (B,), converged (B,)).  Every point is treated as plastic
    (the caller tests f_tr).  `trace`, a list, receives per Newton iteration a dict with the
    active indices, psi(0), psi(1) and the step length taken."""
    Ttr = np.asarray(Ttr, dtype=np.float64)
    alpn = np.asarray(alpn, dtype=np.float64)
    Bn = Ttr.shape[0]

    def G_of(yy, idx):
        return residual(model, E, nu, hardening, h, yy, Ttr[idx], alpn[idx])

    y = np.concatenate([Ttr, alpn[:, None], np.zeros((Bn, 1))], axis=1)
    sref = np.maximum(sigma_y(hardening, h, alpn), np.sqrt(np.sum(Ttr * Ttr, axis=-1)))
    iters = np.zeros(Bn, dtype=np.int64)
    conv = np.zeros(Bn, dtype=bool)
    active = np.arange(Bn)
    for k in range(kmax + 1):
        G = G_of(y[active], active)
        bad = ~np.all(np.isfinite(G), axis=1)
        done = (_scaled_norm(G, sref[active]) <= tol) & ~bad
        conv[active[done]] = True
        keep = ~(done | bad)
        active, G = active[keep], G[keep]
        if active.size == 0 or k == kmax:
            break
        iters[active] += 1
        idx = active
        J = complex_step_jacobian(lambda yy: G_of(yy, idx), y[active], 8)
        dy = np.linalg.solve(J, -G[..., None])[..., 0]
        zeta = np.ones(active.size)
        psi0 = 0.5 * np.sum(G * G, axis=1)
        psi1 = np.full(active.size, np.nan)
        if line_search:
            G1 = G_of(y[active] + dy, active)
            psi1 = 0.5 * np.sum(G1 * G1, axis=1)
            need = np.nonzero(~(psi1 < (1.0 - 2.0 * beta) * psi0))[0]        # Eq. goldstein_full
            if need.size:
                z = psi0[need] / (psi0[need] + psi1[need])                     # Eq. alpha_init
                open_ = np.ones(need.size, dtype=bool)
                for _ in range(jmax + 1):
                    sel = need[open_]
                    Gz = G_of(y[active[sel]] + z[open_, None] * dy[sel], active[sel])
                    psiz = 0.5 * np.sum(Gz * Gz, axis=1)
                    ok = psiz < (1.0 - 2.0 * beta * z[open_]) * psi0[sel]      # Eq. goldstein_full
                    znew = psi0[sel] / (psi0[sel] + psiz)                        # Eq. alpha_update_ls
                    zo = z[open_]
                    z[open_] = np.where(ok, zo, np.maximum(eta * zo, znew))      # Eq. alpha_safeguard
                    open_[np.nonzero(open_)[0][ok]] = False
                    if not open_.any():
                        break
                zeta[need] = z
        if trace is not None:
            trace.append(dict(active=active.copy(), psi0=psi0, psi1=psi1, zeta=zeta.copy()))
        y[active] = y[active] + zeta[:, None] * dy
    return y, iters, conv


def cpp_tangent(model, E, nu, hardening, h, y, Ttr, alpn):
    """dT/dT_tr (B, 6, 6) at converged points by implicit differentiation (App. D): with
    dG/dT_tr = [-I; 0; 0], J_G dy/dT_tr = [I; 0; 0].  Column b is the response to a change of
    component b of T_tr (for a shear component both symmetric entries move)."""
    Ttr = np.asarray(Ttr, dtype=np.float64)
    J = complex_step_jacobian(lambda yy: residual(model, E, nu, hardening, h, yy, Ttr, alpn), y, 8)
    rhs = np.zeros((y.shape[0], 8, 6))
    rhs[:, :6, :] = np.eye(6)
    return np.linalg.solve(J, rhs)[:, :6, :]


# ------------------------------------------------------------------ parameters
N_PARAMS = 23   # c' (9), c'' (9), E, nu, the three hardening parameters


def params(model, E, nu, h):
    """The parameter vector p = (c' (9), c'' (9), E, nu, h (3)) of an isotropic-elastic model."""
    return np.concatenate([model.c1, model.c2, [E, nu], np.asarray(h, dtype=np.float64)]).astype(np.float64)


def unpack(p, m, Theta=None):
    """(model, E, nu, h) from a parameter vector (complex entries allowed)."""
    return Barlat(p[0:9], p[9:18], m, Theta), p[18], p[19], p[20:23]


def _cs_params(fun, p, nout, B):
    """d fun / d p (B, nout, n_p) by complex step for parameters shared by all B points:
    fun(p) (B, nout) with the complex parameter vector p."""
    from .material import CS_H
    J = np.empty((B, nout, p.size))
    for j in range(p.size):
        pc = p.astype(np.complex128)
        pc[j] += 1j * CS_H
        J[:, :, j] = np.imag(fun(pc)) / CS_H
    return J


# ------------------------------------------------------------------ strain-driven update
def local_update(model, E, nu, hardening, h, eps, epn, alpn, derivatives=True, kmax=None, param_derivatives=False):
    """Stress update of Algorithm global_stress_update (App. C), steps 2-6, for this model,
    from the total log strain: T_tr = E : (eps - eps_p,n), the elastic test (reading R10),
    the projection `cpp`, and the recovery eps_p,n+1 = eps_p,n + dgamma N(T), T = E : (eps -
    eps_p,n+1), alpha_n+1 (components, order 11,22,33,12,23,13).

    Returns dict(z (B, 13) = (T, eps_p,n+1, alpha_n+1), dgamma, plastic, iters, converged, ftr)
    and, if derivatives, dz (B, 13, 13) = dz/dp for p = (eps, eps_p,n, alpha_n) by implicit
    differentiation of the converged local system (App. D); with param_derivatives (isotropic
    elasticity only) dz is (B, 13, 13 + N_PARAMS), the last columns dz/dq for the material
    parameters q = params(model, E, nu, h), by the same implicit differentiation with the
    parameter derivatives of G and z taken by complex step."""
    from .material import LOCAL_KMAX
    kmax = LOCAL_KMAX if kmax is None else kmax
    eps = np.asarray(eps, dtype=np.float64)
    epn = np.asarray(epn, dtype=np.float64)
    alpn = np.asarray(alpn, dtype=np.float64)
    B = eps.shape[0]
    p_all = np.concatenate([eps, epn, alpn[:, None]], axis=1)        # (B, 13)

    def ttr(pc):
        return elastic(E, nu, pc[:, 0:6] - pc[:, 6:12])

    def z_el(pc):
        return np.concatenate([ttr(pc), pc[:, 6:12], pc[:, 12:13]], axis=1)

    def z_of(yy, pc):
        N, _ = model.flow(yy[:, :6])
        epnew = pc[:, 6:12] + yy[:, 7:8] * N
        return np.concatenate([elastic(E, nu, pc[:, 0:6] - epnew), epnew, yy[:, 6:7]], axis=1)

    Ttr = ttr(p_all)
    ftr = model.phi_poly(Ttr) - sigma_y(hardening, h, alpn)
    plastic = ftr > 0.0
    z = z_el(p_all)
    dgam = np.zeros(B)
    iters = np.zeros(B, dtype=np.int64)
    conv = np.ones(B, dtype=bool)
    P = np.nonzero(plastic)[0]
    y = None
    if P.size:
        y, it, cv = cpp(model, E, nu, hardening, h, Ttr[P], alpn[P], kmax=kmax)
        z[P] = z_of(y, p_all[P])
        dgam[P] = y[:, 7]
        iters[P] = it
        conv[P] = cv
    out = dict(z=z, dgamma=dgam, plastic=plastic, iters=iters, converged=conv, ftr=ftr)
    if not derivatives:
        return out
    dz = np.empty((B, 13, 13))
    Eidx = np.nonzero(~plastic)[0]
    if Eidx.size:
        dz[Eidx] = complex_step_jacobian(z_el, p_all[Eidx], 13)
    if P.size:
        pP = p_all[P]
        Jy = complex_step_jacobian(
            lambda yy: residual(model, E, nu, hardening, h, yy, ttr(pP), pP[:, 12]), y, 8)
        Gp = complex_step_jacobian(
            lambda pc: residual(model, E, nu, hardening, h, y.astype(pc.dtype), ttr(pc), pc[:, 12]), pP, 8)
        ydot = -np.linalg.solve(Jy, Gp)                                 # (B, 8, 13)
        zy = complex_step_jacobian(lambda yy: z_of(yy, pP), y, 13)
        zp = complex_step_jacobian(lambda pc: z_of(y.astype(pc.dtype), pc), pP, 13)
        dz[P] = zy @ ydot + zp
    if param_derivatives:
        if np.ndim(E) == 4:
            raise NotImplementedError("parameter derivatives are written for isotropic elasticity")
        q = params(model, E, nu, h)
        m, Th = model.m, model.Theta
        dq = np.empty((B, 13, N_PARAMS))
        if Eidx.size:
            pE = p_all[Eidx]

            def z_el_q(qc):
                _, Ec, nuc, _ = unpack(qc, m, Th)
                return np.concatenate([elastic(Ec, nuc, pE[:, 0:6] - pE[:, 6:12]), pE[:, 6:12], pE[:, 12:13]], axis=1)
            dq[Eidx] = _cs_params(z_el_q, q, 13, Eidx.size)
        if P.size:
            def G_q(qc):
                mc, Ec, nuc, hc = unpack(qc, m, Th)
                return residual(mc, Ec, nuc, hardening, hc, y, elastic(Ec, nuc, pP[:, 0:6] - pP[:, 6:12]), pP[:, 12])

            def z_q(qc):
                mc, Ec, nuc, _ = unpack(qc, m, Th)
                N, _ = mc.flow(y[:, :6])
                epnew = pP[:, 6:12] + y[:, 7:8] * N
                return np.concatenate([elastic(Ec, nuc, pP[:, 0:6] - epnew), epnew, y[:, 6:7]], axis=1)
            ydot_q = -np.linalg.solve(Jy, _cs_params(G_q, q, 8, P.size))
            dq[P] = zy @ ydot_q + _cs_params(z_q, q, 13, P.size)
        dz = np.concatenate([dz, dq], axis=2)
    out["dz"] = dz
    return out


def local(model, E, nu, hardening, h, kmax=None):
    """The update above as the callable (eps, epn, alpn, derivatives) that
    material.gauss_point takes in place of the Hill-48 update."""
    def f(eps, epn, alpn, derivatives=True, param_derivatives=False):
        return local_update(model, E, nu, hardening, h, eps, epn, alpn, derivatives, kmax, param_derivatives)
    f.n_params = N_PARAMS
    return f
