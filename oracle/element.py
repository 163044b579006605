"""Oracle, hex8 element (paper Sec. 2.2.4): trilinear shape functions, 2x2x2 Gauss
quadrature, element residual R^e_I = int P . grad0 N_I dV and stiffness K^e = dR^e/dd^e.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Node order C3D8 (bottom face 0-1-2-3 counter-clockwise seen from +z, top face 4-7);
Gauss points at +-1/sqrt(3) with unit weights, numbered g = i + 2 j + 4 k with xi
fastest.  History per Gauss point h = (eps_p (6), alpha).
"""
from __future__ import annotations

import numpy as np

from . import material

NODE_NAT = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
_G = 1.0 / np.sqrt(3.0)
GP_NAT = np.array([[(2 * i - 1) * _G, (2 * j - 1) * _G, (2 * k - 1) * _G]
                   for k in range(2) for j in range(2) for i in range(2)])
GP_W = np.ones(8)


def shape(xi):
    """N_a(xi) = 1/8 (1 + xi_a xi)(1 + eta_a eta)(1 + zeta_a zeta), shape (..., 8)."""
    return 0.125 * np.prod(1.0 + NODE_NAT * np.asarray(xi)[..., None, :], axis=-1)


def dshape(xi):
    """dN_a/dxi_j, shape (8, 3)."""
    xi = np.asarray(xi, dtype=np.float64)
    t = 1.0 + NODE_NAT * xi[None, :]
    d = np.empty((8, 3))
    for j in range(3):
        others = [k for k in range(3) if k != j]
        d[:, j] = 0.125 * NODE_NAT[:, j] * t[:, others[0]] * t[:, others[1]]
    return d


DN_GP = np.stack([dshape(x) for x in GP_NAT])        # (8 gp, 8 nodes, 3)


def gradients(Xe):
    """Reference shape-function gradients g[e, gp, a, :] = dN_a/dX and w*det(J0) per gp.
    Xe (n_el, 8, 3)."""
    J0 = np.einsum("eai,gaj->egij", Xe, DN_GP)        # dX_i/dxi_j
    det = np.linalg.det(J0)
    Jinv = np.linalg.inv(J0)                           # dxi_j/dX_i
    g = np.einsum("gaj,egji->egai", DN_GP, Jinv)
    return g, det * GP_W[None, :]


def element_sweep(X, conn, u, hist, theta, hardening, Theta=None, jacobians="tangent", fbar=False, local=None):
    """All elements at once.

    X (n_nodes,3), conn (n_el,8), u (n_dof,), hist (n_el,8,7) history at t_n,
    theta (11,) or (n_el,11), Theta None/(3,3)/(n_el,3,3).
    Returns Re (n_el,24), Ke (n_el,24,24) if jacobians, h_new (n_el,8,7), the Gauss-point
    dict of material.gauss_point (arrays flattened over (el, gp)), g and wdet.

    local: another model's strain-driven update for material.gauss_point (e.g. barlat.local);
    theta, hardening and Theta are then unused.

    fbar: the F-bar element of Sec. 2.2.4 (Eq. Fbar): the constitutive model receives
    Fbar = (Jbar / J)^(1/3) F with Jbar = (1/V_e) int_e J dV, the residual is
    R^e_I = int P(Fbar) . grad0 N_I dV, and K^e = dR^e/dd^e follows by the chain rule through
    Fbar (J at the point and Jbar of the element), which makes K non-symmetric.
    """
    conn = np.asarray(conn, dtype=np.int64)
    n_el = conn.shape[0]
    Xe = X[conn]                                       # (n_el, 8, 3)
    ue = u.reshape(-1, 3)[conn]                        # (n_el, 8, 3)
    g, wdet = gradients(Xe)
    F = np.eye(3) + np.einsum("eai,egaj->egij", ue, g)  # F = I + sum_a u_a (x) g_a
    if fbar:
        return _element_sweep_fbar(F, g, wdet, hist, theta, hardening, Theta, jacobians, n_el, local)
    theta = np.asarray(theta, dtype=np.float64)
    th = np.broadcast_to(theta if theta.ndim == 1 else theta[:, None, :], (n_el, 8, 11))
    if Theta is None:
        Th = np.broadcast_to(np.eye(3), (n_el, 8, 3, 3))
    else:
        Theta = np.asarray(Theta, dtype=np.float64)
        Th = np.broadcast_to(Theta if Theta.ndim == 2 else Theta[:, None], (n_el, 8, 3, 3))
    gp = material.gauss_point(F.reshape(-1, 3, 3), hist[..., :6].reshape(-1, 6),
                              hist[..., 6].reshape(-1), th.reshape(-1, 11), hardening,
                              Th.reshape(-1, 3, 3), jacobians=jacobians, local=local)
    P = gp["P"].reshape(n_el, 8, 3, 3)
    Re = np.einsum("eg,egiJ,egaJ->eai", wdet, P, g).reshape(n_el, 24)
    out = dict(Re=Re, h_new=gp["h_new"].reshape(n_el, 8, 7), gp=gp, g=g, wdet=wdet, F=F)
    if jacobians is not None:
        A = gp["A"].reshape(n_el, 8, 3, 3, 3, 3)
        Ke = np.einsum("eg,egaJ,egiJkL,egbL->eaibk", wdet, g, A, g).reshape(n_el, 24, 24)
        out["Ke"] = Ke
    return out


def _element_sweep_fbar(F, g, wdet, hist, theta, hardening, Theta, jacobians, n_el, local=None):
    J = np.linalg.det(F)                                          # (n_el, 8)
    Jbar = np.einsum("eg,eg->e", wdet, J) / wdet.sum(axis=1)      # volume average of J
    s = np.cbrt(Jbar[:, None] / J)                                # (Jbar / J)^(1/3)
    Fb = s[..., None, None] * F
    theta = np.asarray(theta, dtype=np.float64)
    th = np.broadcast_to(theta if theta.ndim == 1 else theta[:, None, :], (n_el, 8, 11))
    if Theta is None:
        Th = np.broadcast_to(np.eye(3), (n_el, 8, 3, 3))
    else:
        Theta = np.asarray(Theta, dtype=np.float64)
        Th = np.broadcast_to(Theta if Theta.ndim == 2 else Theta[:, None], (n_el, 8, 3, 3))
    gp = material.gauss_point(Fb.reshape(-1, 3, 3), hist[..., :6].reshape(-1, 6),
                              hist[..., 6].reshape(-1), th.reshape(-1, 11), hardening,
                              Th.reshape(-1, 3, 3), jacobians=jacobians, local=local)
    P = gp["P"].reshape(n_el, 8, 3, 3)                            # P(Fbar)
    Re = np.einsum("eg,egiJ,egaJ->eai", wdet, P, g).reshape(n_el, 24)
    out = dict(Re=Re, h_new=gp["h_new"].reshape(n_el, 8, 7), gp=gp, g=g, wdet=wdet, F=F, Fbar=Fb, Jbar=Jbar)
    if jacobians is not None:
        A = gp["A"].reshape(n_el, 8, 3, 3, 3, 3)                  # dP/dFbar
        Finv = np.linalg.inv(F)
        # spatial gradients F^-T g_b (the derivative of J is J F^-T)
        sg = np.einsum("egLk,egbL->egbk", Finv, g)
        # dJbar/du_bk = (1/V) sum_q w det J0 J_q (F_q^-T g_b)_k
        dJbar = np.einsum("eg,eg,egbk->ebk", wdet, J, sg) / wdet.sum(axis=1)[:, None, None]
        # dFbar_mn / du_bk = s (delta_mk g_b,n - 1/3 F_mn (F^-T g_b)_k) + Fbar_mn / (3 Jbar) dJbar/du_bk
        eye = np.eye(3)
        dFb = (s[..., None, None, None, None]
               * (np.einsum("mk,egbn->egmnbk", eye, g) - np.einsum("egmn,egbk->egmnbk", F, sg) / 3.0)
               + np.einsum("egmn,ebk->egmnbk", Fb, dJbar) / (3.0 * Jbar)[:, None, None, None, None, None])
        Ke = np.einsum("eg,egaJ,egiJmn,egmnbk->eaibk", wdet, g, A, dFb).reshape(n_el, 24, 24)
        out["Ke"] = Ke
    return out
