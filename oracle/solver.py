"""Oracle, global level: assembly, Dirichlet elimination, Newton, load steps, objective,
discrete adjoint, direct sensitivity and central finite differences.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Assembly K = A_e K^e, R = A_e R^e (Sec. 2.2.4); COO -> CSR summation is the library
  step (scipy.sparse), standing in for the triplet assembly of App. E.
* Dirichlet data: u[dof] = t * value is imposed on u before the first Newton iteration of a
  step and the linear solves run on the free block of K (reading R12: the same converged u as
  identity-row elimination, with a symmetric matrix).
* Newton (Eq. Stiffness_mat): K(d^k) dd = -R(d^k) until ||R_free|| <= rtol * max(ref, 1)
  (reading R11) with ref the norm of the predictor's right-hand side; the linear solve is
  scipy's sparse direct solver.  Each step starts from the linearised Dirichlet increment on
  the converged start-of-step state (reading R14; a step that starts from u_{n-1} with only
  the new boundary values can land on an indefinite tangent and diverge on perforated plates).
* Objective J = w sum_n ||u^n - u_gt^n||^2 over all dofs and steps (Sec. 2.3, reading R16).
* Adjoint (Eq. dR_u, Eq. main_grad, Algorithm adjoint_ad) with the history written out:
  states (u^n, h^n), R^n(u^n, h^{n-1}, theta) = 0, h^n = H(u^n, h^{n-1}, theta).  With
  mu^N = 0, for n = N..1:  ubar = dJ^n/du^n + (dH/du^n)^T mu^n;  K^T lambda = -ubar (free
  dofs);  mu^{n-1} = (dR^n/dh^{n-1})^T lambda + (dH/dh^{n-1})^T mu^n;
  g += (dR^n/dtheta)^T lambda + (dH/dtheta)^T mu^n.
* Direct sensitivity (forward mode of the same chain) and central FD (Algorithm
  finite_difference) are the independent checks of the adjoint.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import element


@dataclasses.dataclass
class Problem:
    X: np.ndarray
    conn: np.ndarray
    fixed_dof: np.ndarray
    fixed_val: np.ndarray
    theta: np.ndarray            # (11,) uniform or (n_el, 11) per element
    hardening: str
    Theta: np.ndarray | None = None
    f_ext: np.ndarray | None = None   # nodal dead load at t = 1 (n_dof,), optional
    fbar: bool = False                # F-bar element (Eq. Fbar); K is then non-symmetric
    local: object = None              # another model's stress update (barlat.local); theta unused

    @property
    def n_dof(self):
        return 3 * self.X.shape[0]

    @property
    def n_el(self):
        return self.conn.shape[0]


def from_inputs(mesh, bc, mat, theta=None, fbar=False):
    th = mat.theta_vector() if theta is None else np.asarray(theta, dtype=np.float64)
    return Problem(X=mesh.X, conn=mesh.conn.astype(np.int64), fixed_dof=bc.dof,
                   fixed_val=bc.value, theta=th, hardening=mat.hardening,
                   Theta=None if np.allclose(mat.Theta, np.eye(3)) else mat.Theta, fbar=fbar)


def element_dofs(conn):
    return (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(conn.shape[0], 24)


def assemble_R(prob, Re):
    R = np.zeros(prob.n_dof)
    np.add.at(R, element_dofs(prob.conn), Re)
    return R


def assemble_K(prob, Ke):
    ed = element_dofs(prob.conn)
    rows = np.repeat(ed, 24, axis=1).ravel()
    cols = np.tile(ed, (1, 24)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(prob.n_dof, prob.n_dof)).tocsr()


def free_mask(prob):
    m = np.ones(prob.n_dof, dtype=bool)
    m[prob.fixed_dof] = False
    return m


def residual(prob, u, hist, t=1.0, jacobians="tangent"):
    """R(u) = f_int(u; h_n) - t f_ext and, with jacobians, K = dR/du."""
    es = element.element_sweep(prob.X, prob.conn, u, hist, prob.theta, prob.hardening,
                               prob.Theta, jacobians=jacobians, fbar=prob.fbar, local=prob.local)
    R = assemble_R(prob, es["Re"])
    if prob.f_ext is not None:
        R = R - t * prob.f_ext
    K = assemble_K(prob, es["Ke"]) if jacobians is not None else None
    return R, K, es


def newton_step(prob, u0, hist, t, rtol=1e-10, maxit=30, atol_floor=1.0, t_prev=None, prev=None):
    """Equilibrium at load factor t from the converged start-of-step state u0 (at t_prev).

    Predictor (reading R14): the Dirichlet increment du_D is linearised at the start-of-step
    state, u = u0 + du_D + K_ff^{-1} (-(R(u0) + K du_D - dt f_ext))_f.  K and R are those of
    the previous step's last Newton iteration (`prev`, its consistent algorithmic tangent at
    u0), or, without `prev` (first step), the sweep at (u0, h_{n-1}).  The Newton iterations
    that follow are Eq. Stiffness_mat; the predictor changes the iteration count only.
    Without t_prev: u = u0 with the new Dirichlet values.  info["last"] = (R, K) of the last
    iteration, the `prev` of the next step.
    """
    free = free_mask(prob)
    u = u0.copy()
    ref = None
    if t_prev is not None:
        if prev is not None:
            R0, K0 = prev
        else:
            R0, K0, _ = residual(prob, u, hist, t_prev)
        duD = np.zeros(prob.n_dof)
        duD[prob.fixed_dof] = (t - t_prev) * prob.fixed_val
        b = -(R0 + K0 @ duD)
        if prob.f_ext is not None:
            b = b + (t - t_prev) * prob.f_ext
        ref = max(float(np.linalg.norm(b[free])), atol_floor)
        u = u + duD
        if np.any(b[free] != 0.0):
            u[free] += spla.spsolve(K0[free][:, free].tocsc(), b[free])
    u[prob.fixed_dof] = t * prob.fixed_val
    history = []
    for it in range(maxit + 1):
        R, K, es = residual(prob, u, hist, t)
        rn = float(np.linalg.norm(R[free]))
        history.append(rn)
        if ref is None:
            ref = max(rn, atol_floor)
        if rn <= rtol * ref:
            return u, es, dict(iters=it, res=history, converged=True, last=(R, K))
        if it == maxit:
            break
        Kff = K[free][:, free]
        du = spla.spsolve(Kff.tocsc(), -R[free])
        u[free] += du
    return u, es, dict(iters=maxit, res=history, converged=False)


class NewtonDivergence(RuntimeError):
    pass


def forward(prob, t_steps, rtol=1e-10, maxit=30, hist0=None, predictor=True):
    """Load-step loop; returns u^n (N, n_dof), h^n (N+1, n_el, 8, 7), per-step info.
    Raises NewtonDivergence if a step does not converge."""
    hist = np.zeros((prob.n_el, 8, 7)) if hist0 is None else hist0.copy()
    u = np.zeros(prob.n_dof)
    us, hs, infos = [], [hist.copy()], []
    t_prev = 0.0
    prev = None
    for t in t_steps:
        u, es, info = newton_step(prob, u, hist, t, rtol=rtol, maxit=maxit,
                                  t_prev=t_prev if predictor else None, prev=prev)
        if not info["converged"]:
            raise NewtonDivergence(f"step t={t}: residual history {info['res'][-3:]}")
        prev = info.pop("last")
        t_prev = t
        hist = es["h_new"].copy()                  # commit h_n = H(u_n, h_{n-1}, theta)
        us.append(u.copy())
        hs.append(hist.copy())
        info["plastic"] = int(es["gp"]["plastic"].sum())
        info["sigma"] = es["gp"]["sigma"].reshape(prob.n_el, 8, 3, 3)
        infos.append(info)
    return np.array(us), np.array(hs), infos


def objective(us, u_gt, w=1.0):
    return float(w * np.sum((us - u_gt) ** 2))


def _gp_cotangent_from_dofs(prob, es, lam):
    """P-bar per Gauss point: w detJ0 sum_a lambda_a (x) g_a (shape (n_el, 8, 3, 3))."""
    le = lam.reshape(-1, 3)[prob.conn]                 # (n_el, 8, 3)
    return np.einsum("eg,eai,egaJ->egiJ", es["wdet"], le, es["g"])


def _dofs_from_F_cotangent(prob, es, Fbar):
    """u-bar = sum_gp sum_l Fbar_kl g_al, scattered to the dofs."""
    ue = np.einsum("egkl,egal->eak", Fbar, es["g"]).reshape(prob.n_el, 24)
    return assemble_R(prob, ue)


def n_params(prob):
    """Length of the parameter vector the adjoint differentiates: Hill-48's 11, or the local
    model's own (e.g. Barlat's 23; uniform parameters only)."""
    if prob.local is None:
        return 11
    if not hasattr(prob.local, "n_params"):
        raise NotImplementedError("this local model provides no parameter derivatives")
    return prob.local.n_params


def adjoint(prob, t_steps, us, hs, u_gt, w=1.0, per_element=False):
    """dJ/dtheta by the discrete adjoint; (n_p,) for uniform parameters, (n_el, n_p) if
    per_element, with n_p = n_params(prob) (Hill-48's theta, or the local model's vector)."""
    if prob.fbar:
        raise NotImplementedError("the adjoint of the F-bar element is not part of the oracle")
    npar = n_params(prob)
    free = free_mask(prob)
    n_el = prob.n_el
    N = len(t_steps)
    mu = np.zeros((n_el, 8, 7))
    gth = np.zeros((n_el, npar))
    for n in range(N - 1, -1, -1):
        R, K, es = residual(prob, us[n], hs[n], t_steps[n], jacobians="all")
        gp = es["gp"]
        mu_f = mu.reshape(-1, 7)
        Fbar = np.einsum("bj,bjkl->bkl", mu_f, gp["dh_dF"]).reshape(n_el, 8, 3, 3)
        ubar = 2.0 * w * (us[n] - u_gt[n]) + _dofs_from_F_cotangent(prob, es, Fbar)
        lam = np.zeros(prob.n_dof)
        Kff = K[free][:, free]
        lam[free] = spla.spsolve(Kff.T.tocsc(), -ubar[free])
        Pbar = _gp_cotangent_from_dofs(prob, es, lam).reshape(-1, 3, 3)
        hbar = np.einsum("biJ,biJj->bj", Pbar, gp["dP_dh"]) + \
            np.einsum("bj,bjk->bk", mu_f, gp["dh_dh"])
        tbar = np.einsum("biJ,biJj->bj", Pbar, gp["dP_dtheta"]) + \
            np.einsum("bj,bjk->bk", mu_f, gp["dh_dtheta"])
        gth += tbar.reshape(n_el, 8, npar).sum(axis=1)
        mu = hbar.reshape(n_el, 8, 7)
    return gth if per_element else gth.sum(axis=0)


def direct_sensitivity(prob, t_steps, us, hs, u_gt, dtheta, w=1.0):
    """dJ/dtheta . dtheta by forward (tangent) propagation; dtheta (n_p,) or (n_el, n_p) with
    n_p = n_params(prob)."""
    if prob.fbar:
        raise NotImplementedError("the sensitivity of the F-bar element is not part of the oracle")
    npar = n_params(prob)
    free = free_mask(prob)
    n_el = prob.n_el
    dth = np.broadcast_to(np.asarray(dtheta, dtype=np.float64), (n_el, npar))
    dth_gp = np.repeat(dth[:, None, :], 8, axis=1).reshape(-1, npar)
    hdot = np.zeros((n_el * 8, 7))
    dJ = 0.0
    for n in range(len(t_steps)):
        R, K, es = residual(prob, us[n], hs[n], t_steps[n], jacobians="all")
        gp = es["gp"]
        Pdot = np.einsum("biJj,bj->biJ", gp["dP_dtheta"], dth_gp) + \
            np.einsum("biJj,bj->biJ", gp["dP_dh"], hdot)
        Re_dot = np.einsum("eg,egiJ,egaJ->eai", es["wdet"], Pdot.reshape(n_el, 8, 3, 3),
                           es["g"]).reshape(n_el, 24)
        rhs = assemble_R(prob, Re_dot)
        udot = np.zeros(prob.n_dof)
        udot[free] = spla.spsolve(K[free][:, free].tocsc(), -rhs[free])
        Fdot = np.einsum("eai,egaj->egij", udot.reshape(-1, 3)[prob.conn], es["g"]).reshape(-1, 3, 3)
        hdot = np.einsum("bjkl,bkl->bj", gp["dh_dF"], Fdot) + \
            np.einsum("bjk,bk->bj", gp["dh_dh"], hdot) + \
            np.einsum("bjk,bk->bj", gp["dh_dtheta"], dth_gp)
        dJ += float(2.0 * w * np.dot(us[n] - u_gt[n], udot))
    return dJ


def fd_gradient(prob, t_steps, u_gt, h_rel=1e-6, w=1.0, index=None, rtol=1e-13):
    """Central differences (Algorithm finite_difference) with step h_rel * |theta_i|."""
    th0 = np.asarray(prob.theta, dtype=np.float64)
    idx = range(th0.shape[-1]) if index is None else index
    g = {}
    for i in idx:
        h = h_rel * abs(th0[..., i]).max()
        vals = []
        for s in (+1, -1):
            th = th0.copy()
            th[..., i] += s * h
            p = dataclasses.replace(prob, theta=th)
            us, _, _ = forward(p, t_steps, rtol=rtol)
            vals.append(objective(us, u_gt, w))
        g[i] = (vals[0] - vals[1]) / (2 * h)
    return g


def fd_directional(prob, t_steps, u_gt, direction, h=1e-6, w=1.0, rtol=1e-13):
    """Central difference of J along a parameter direction (same shape as theta)."""
    vals = []
    for s in (+1, -1):
        p = dataclasses.replace(prob, theta=np.asarray(prob.theta) + s * h * np.asarray(direction))
        us, _, _ = forward(p, t_steps, rtol=rtol)
        vals.append(objective(us, u_gt, w))
    return (vals[0] - vals[1]) / (2 * h)
