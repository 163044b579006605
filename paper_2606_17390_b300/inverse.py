"""Inverse identification of material parameters (paper Sec. 2.3 step (e) and Sec. 4): the
displacement misfit J(theta) and its gradient from hfe_adjoint, minimised by the
bound-constrained L-BFGS-B of scipy over normalised parameters

    rho_i = 2 (theta_i - theta_min_i) / theta_ref_i - 1,   rho_i in [-1, 1],
    theta_i = (rho_i + 1) theta_ref_i / 2 + theta_min_i,

with theta_ref = theta_max - theta_min, and the paper's stopping criteria (maxiter 45,
maxfun 90, ftol 1e-10, gtol 1e-10).  Host-side optimiser logic only: every forward solve and
gradient runs in libhfe.so.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

__all__ = ["normalize", "denormalize", "IdentifyResult", "identify"]

PAPER_CRITERIA = dict(maxiter=45, maxfun=90, ftol=1e-10, gtol=1e-10)


def normalize(theta, theta_min, theta_ref):
    """rho = 2 (theta - theta_min) / theta_ref - 1."""
    return 2.0 * (np.asarray(theta, dtype=np.float64) - theta_min) / theta_ref - 1.0


def denormalize(rho, theta_min, theta_ref):
    """theta = (rho + 1) theta_ref / 2 + theta_min."""
    return (np.asarray(rho, dtype=np.float64) + 1.0) * theta_ref / 2.0 + theta_min


@dataclasses.dataclass
class IdentifyResult:
    theta: np.ndarray            # full parameter array at the optimum (layout of theta0)
    J: float
    iterations: int
    evaluations: int
    success: bool
    message: str
    history: list                # (J, theta of the identified entries) per evaluation
    seconds: float


def identify(solver, t, u_target, theta0, index, theta_min, theta_ref, w=1.0, criteria=None):
    """Minimise J over the entries `index` of theta (an (11,) uniform array, or (n_el, 11) with
    `index` a tuple of numpy index arrays / a boolean mask selecting per-element entries),
    starting from theta0 and bounded by [theta_min, theta_min + theta_ref] (arrays of the
    selected entries' shape).  The other entries stay at theta0."""
    from scipy.optimize import minimize

    crit = dict(PAPER_CRITERIA)
    if criteria:
        crit.update(criteria)
    theta = np.array(theta0, dtype=np.float64)
    tmin = np.asarray(theta_min, dtype=np.float64)
    tref = np.asarray(theta_ref, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    history = []

    def fun(rho):
        th = theta.copy()
        th[index] = denormalize(rho.reshape(tmin.shape), tmin, tref)
        solver.set_material(th, getattr(solver, "Theta_axes", None))
        J, g, _ = solver.adjoint(t, u_target, w)
        g = g.reshape(th.shape) if th.ndim > 1 else g.reshape(-1)[: th.size]
        history.append((J, th[index].copy()))
        # d theta / d rho = theta_ref / 2
        return J, (g[index] * tref / 2.0).ravel()

    rho0 = normalize(theta[index], tmin, tref).ravel()
    t0 = time.perf_counter()
    res = minimize(fun, rho0, jac=True, method="L-BFGS-B", bounds=[(-1.0, 1.0)] * rho0.size,
                   options=dict(maxiter=crit["maxiter"], maxfun=crit["maxfun"], ftol=crit["ftol"],
                                gtol=crit["gtol"]))
    secs = time.perf_counter() - t0
    th = theta.copy()
    th[index] = denormalize(res.x.reshape(tmin.shape), tmin, tref)
    solver.set_material(th, getattr(solver, "Theta_axes", None))
    return IdentifyResult(theta=th, J=float(res.fun), iterations=int(res.nit), evaluations=int(res.nfev),
                          success=bool(res.success), message=str(res.message), history=history, seconds=secs)
