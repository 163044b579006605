"""Inverse identification of material parameters (paper Sec. 2.3 step (e) and Sec. 4): the
displacement misfit J(theta) and its gradient from hfe_adjoint, minimised by the
bound-constrained L-BFGS-B of scipy over normalised parameters

    rho_i = 2 (theta_i - theta_min_i) / theta_ref_i - 1,   rho_i in [-1, 1],
    theta_i = (rho_i + 1) theta_ref_i / 2 + theta_min_i,

with theta_ref = theta_max - theta_min, and the paper's stopping criteria (maxiter 45,
maxfun 90, ftol 1e-10, gtol 1e-10).  With warm_start (Sec. 3.6) each forward pass starts its
load steps from the previous pass's displacements (hfe_set_warm_start) whenever every
identified parameter moved by less than 10 % since that pass, and cold otherwise.  Host-side
optimiser logic only: every forward solve and gradient runs in libhfe.so.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

__all__ = ["normalize", "denormalize", "IdentifyResult", "identify", "warm_start_applies"]

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
    warm_passes: int = 0         # evaluations whose forward pass started from the previous one


WARM_START_TOL = 0.1   # relative change of every parameter below which the record is reused


def warm_start_applies(theta, theta_prev, tol=WARM_START_TOL):
    """True when every entry changed by less than tol relative to the recorded pass's value
    (an entry that was 0 there must still be 0)."""
    if theta_prev is None:
        return False
    theta, theta_prev = np.asarray(theta, dtype=np.float64), np.asarray(theta_prev, dtype=np.float64)
    d = np.abs(theta - theta_prev)
    return bool(np.all((d == 0.0) | (d < tol * np.abs(theta_prev))))


def identify(solver, t, u_target, theta0, index, theta_min, theta_ref, w=1.0, criteria=None,
             warm_start=False):
    """Minimise J over the entries `index` of theta (an (11,) uniform array, or (n_el, 11) with
    `index` a tuple of numpy index arrays / a boolean mask selecting per-element entries),
    starting from theta0 and bounded by [theta_min, theta_min + theta_ref] (arrays of the
    selected entries' shape).  The other entries stay at theta0.  warm_start: reuse the
    previous forward pass under the 10 % rule (the record is freed at the end)."""
    from scipy.optimize import minimize

    crit = dict(PAPER_CRITERIA)
    if criteria:
        crit.update(criteria)
    theta = np.array(theta0, dtype=np.float64)
    tmin = np.asarray(theta_min, dtype=np.float64)
    tref = np.asarray(theta_ref, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    history = []
    warm = dict(prev=None, passes=0)

    def fun(rho):
        th = theta.copy()
        th[index] = denormalize(rho.reshape(tmin.shape), tmin, tref)
        solver.set_material(th, getattr(solver, "Theta_axes", None))
        if warm_start:
            use = warm_start_applies(th[index], warm["prev"])
            solver.set_warm_start("use" if use else "record")
            warm["passes"] += int(use)
        J, g, _ = solver.adjoint(t, u_target, w)
        if warm_start:
            warm["prev"] = th[index].copy()
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
    if warm_start:
        solver.set_warm_start("off")
    th = theta.copy()
    th[index] = denormalize(res.x.reshape(tmin.shape), tmin, tref)
    solver.set_material(th, getattr(solver, "Theta_axes", None))
    return IdentifyResult(theta=th, J=float(res.fun), iterations=int(res.nit), evaluations=int(res.nfev),
                          success=bool(res.success), message=str(res.message), history=history, seconds=secs,
                          warm_passes=warm["passes"])
