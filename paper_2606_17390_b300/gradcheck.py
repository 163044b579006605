"""Finite-difference verification of adjoint gradients (Sec. 2.3, Alg. finite_difference, and
the error measure of Sec. 3.2).

The central difference of the misfit J along each parameter, as the paper states it:
[dJ/dtheta]_i ~ (J(theta + h e_i) - J(theta - h e_i)) / (2h), two forward solves per component.
The check compares the adjoint gradient with it along a direction D in parameter space,
E_FD,check(h) = |g_adjoint . D - g_FD(h) . D| (every D_i = 0.1 in the paper), over the step
sizes h = 1e-1, 1e-2, ..., 1e-11: truncation error dominates at large h, rounding error at
small h, and the smallest E shows how well the two gradients agree.

Host-side driver only: J is any callable (objective() builds one from a Solver, whose every
forward solve runs in libhfe.so).  An optional per-parameter scale turns h into the relative
step h * scale_i for parameters of very different magnitudes (E in MPa against n).
"""
from __future__ import annotations

import numpy as np

__all__ = ["PAPER_STEPS", "PAPER_DIRECTION", "objective", "fd_gradient", "fd_check"]

PAPER_STEPS = tuple(10.0 ** -k for k in range(1, 12))   # h = 1e-1 ... 1e-11
PAPER_DIRECTION = 0.1                                    # D_i


def objective(solver, t, u_target, w=1.0):
    """J(theta) = w sum_n ||u^n(theta) - u_target^n||^2 of a forward run from the zero state
    (the misfit hfe_adjoint differentiates), theta in the solver's parameter layout."""
    t = np.asarray(t, dtype=np.float64)
    u_target = np.asarray(u_target, dtype=np.float64)

    def J(theta):
        solver.set_material(np.asarray(theta, dtype=np.float64), getattr(solver, "Theta_axes", None))
        solver.set_state(None, None)
        u, _ = solver.forward(t)
        return float(w * np.sum((u - u_target) ** 2))

    return J


def fd_gradient(J, theta, h, index=None, scale=None):
    """Central differences of J at theta (Alg. finite_difference) for the entries `index` of
    the flattened theta (all by default), step h (times scale_i when a scale is given).
    Returns the differences in the order of `index`."""
    theta = np.asarray(theta, dtype=np.float64)
    flat = theta.ravel()
    idx = np.arange(flat.size) if index is None else np.asarray(index).ravel()
    sc = np.ones(idx.size) if scale is None else np.broadcast_to(np.asarray(scale, dtype=np.float64), idx.shape)
    g = np.empty(idx.size)
    for k, i in enumerate(idx):
        hi = h * sc[k]
        tp, tm = flat.copy(), flat.copy()
        tp[i] += hi
        tm[i] -= hi
        g[k] = (J(tp.reshape(theta.shape)) - J(tm.reshape(theta.shape))) / (2.0 * hi)
    return g


def fd_check(J, g_adjoint, theta, steps=PAPER_STEPS, direction=PAPER_DIRECTION, index=None, scale=None):
    """E_FD,check(h) = |g_adjoint . D - g_FD(h) . D| for each step h; g_adjoint holds the
    adjoint gradient of the same entries as `index` (all entries by default) and D is the
    direction (a scalar fills every component).  Returns a list of dicts (h, E, g_fd) and the
    reference directional derivative g_adjoint . D."""
    g_adjoint = np.asarray(g_adjoint, dtype=np.float64).ravel()
    D = np.broadcast_to(np.asarray(direction, dtype=np.float64), g_adjoint.shape)
    ref = float(g_adjoint @ D)
    out = []
    for h in steps:
        g_fd = fd_gradient(J, theta, h, index=index, scale=scale)
        out.append({"h": float(h), "E": abs(ref - float(g_fd @ D)), "g_fd": g_fd})
    return out, ref
