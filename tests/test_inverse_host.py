"""The inverse loop's host logic (inverse.identify) driven by the oracle through a
duck-typed solver: per-element parameters selected by a boolean mask (normalisation, the
chain d theta / d rho, the gradient layout), recovery of a per-element sigma0 field from a
noiseless target, and the 10 % warm-start rule switching the solver between recording and
reusing passes."""
import dataclasses

import numpy as np

from oracle import solver
from paper_2606_17390_b300 import inputs, inverse


class OracleSolver:
    """The calls identify makes (set_material, adjoint, set_warm_start) on the oracle."""

    def __init__(self, prob):
        self.prob = prob
        self.Theta_axes = None
        self.warm_modes = []

    def set_material(self, theta, Theta=None):
        self.prob = dataclasses.replace(self.prob, theta=np.array(theta, dtype=np.float64))

    def set_warm_start(self, mode):
        self.warm_modes.append(mode)

    def adjoint(self, t, u_target, w=1.0):
        us, hs, _ = solver.forward(self.prob, t, rtol=1e-13)
        per_el = np.ndim(self.prob.theta) > 1
        g = solver.adjoint(self.prob, t, us, hs, u_target, w=w, per_element=per_el)
        return solver.objective(us, u_target, w), np.atleast_2d(g), {}


def test_identify_per_element_sigma0_with_warm_start():
    mesh = inputs.box_mesh(3, 2, 1, 3.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.06, 0.02, 0.0))
    mat = inputs.config1_material()
    ts = inputs.load_factors(3)
    th_true = np.tile(mat.theta_vector(), (mesh.n_el, 1))
    th_true[:, 8] *= 1.0 + 0.1 * np.linspace(-1, 1, mesh.n_el)          # sigma0 field
    p_true = solver.from_inputs(mesh, bc, mat, th_true)
    u_gt, _, _ = solver.forward(p_true, ts, rtol=1e-13)
    mask = np.zeros_like(th_true, dtype=bool)
    mask[:, 8] = True
    tmin, tref = 0.8 * th_true[mask], 0.4 * th_true[mask]                # bounds 0.8 ... 1.2 x truth
    th0 = th_true.copy()
    th0[mask] = inverse.denormalize(np.full(mask.sum(), 0.3), tmin, tref)
    s = OracleSolver(solver.from_inputs(mesh, bc, mat, th0))
    res = inverse.identify(s, ts, u_gt, th0, mask, tmin, tref, w=1e6, warm_start=True,
                           criteria=dict(maxiter=30, maxfun=40))
    assert res.theta.shape == th_true.shape
    assert np.array_equal(res.theta[~mask], th0[~mask])                 # unselected entries kept
    assert np.allclose(res.theta[mask], th_true[mask], rtol=1e-3), (res.theta[mask], th_true[mask])
    assert res.J < 1e-6 * res.history[0][0]
    # the rule: the first pass records, later passes within 10 % reuse, the record is freed
    assert s.warm_modes[0] == "record" and s.warm_modes[-1] == "off"
    assert res.warm_passes == s.warm_modes.count("use") and res.warm_passes > 0
