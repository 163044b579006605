"""Parity at the full 100^3 size (1,000,000 elements, 3,090,903 dofs) in the launch
configuration the benchmark times, where the oracle cannot run the whole problem:

* the tangent sweep at the benchmark's clamped-platen compression state, checked on sampled
  nodes against the oracle's element routine on the elements around each node (residual
  rows, stiffness columns extracted with the SpMV, trial history of those elements);
* the homogeneous variant (roller symmetry, Hill with G + H = 1) through whole forward load
  steps against the uniaxial closed form, which holds at any mesh size and step size.
"""
import numpy as np
import pytest

from oracle import element
from paper_2606_17390_b300 import hfe, inputs
from tests._helpers import hist_soa_to_oracle

pytestmark = pytest.mark.gpu

N = 100
LOAD = 0.5
TOL = {"fp64": dict(R=1e-11, K=1e-9, h=1e-12), "mixed": dict(R=2e-5, K=1e-4, h=1e-5)}


@pytest.fixture(scope="module")
def cube_state():
    mesh, bc, mat, _ = inputs.config2_problem(N, 10)
    u, hist = inputs.compression_state(mesh, LOAD)
    return mesh, bc, mat, u, hist


def _sample_nodes(mesh, rng, k):
    """k interior nodes and k nodes next to the clamped faces (x = 0 and x = 1)."""
    X = mesh.X
    h = 1.0 / N
    interior = np.nonzero((X.min(axis=1) > 1.5 * h) & (X.max(axis=1) < 1 - 1.5 * h))[0]
    near = np.nonzero((np.abs(X[:, 0] - h) < 1e-9) | (np.abs(X[:, 0] - (1 - h)) < 1e-9))[0]
    return np.concatenate([rng.choice(interior, k, replace=False), rng.choice(near, k, replace=False)])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_config2_tangent_sweep_sampled(cube_state, precision):
    import torch
    mesh, bc, mat, u, hist = cube_state
    rng = np.random.default_rng(7)
    nodes = _sample_nodes(mesh, rng, 5)
    free = np.ones(mesh.n_dof, bool)
    free[bc.dof] = False
    with hfe.from_inputs(mesh, bc, mat, precision=precision) as s:
        s.set_state(None, hist)
        R = torch.empty(mesh.n_dof, dtype=torch.float64, device="cuda")
        H = np.empty((7, mesh.n_el * 8))
        _, _, st = s.sweep(torch.from_numpy(u).cuda(), LOAD, tangent=True, R_out=R, hist_out=H)
        R = R.cpu().numpy()
        cols = {}
        for n in nodes:
            j = 3 * int(n) + 1
            if not free[j]:
                continue
            e = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
            e[j] = 1.0
            cols[j] = s.spmv(e).cpu().numpy()
    assert st["plastic_gps"] > 0
    tol = TOL[precision]
    conn = mesh.conn.astype(np.int64)
    hist_o = hist_soa_to_oracle(hist, mesh.n_el)
    H_o = hist_soa_to_oracle(H, mesh.n_el)
    for n in nodes:
        els = np.nonzero((conn == n).any(axis=1))[0]
        es = element.element_sweep(mesh.X, conn[els], u, hist_o[els], mat.theta_vector(), mat.hardening)
        scale_R = np.abs(es["Re"]).max()
        # residual rows of node n: sum of its element contributions
        Rn = np.zeros(3)
        for k, el in enumerate(els):
            a = int(np.nonzero(conn[el] == n)[0][0])
            Rn += es["Re"][k, 3 * a:3 * a + 3]
        assert np.abs(R[3 * n:3 * n + 3] - Rn).max() <= tol["R"] * scale_R, (n, R[3 * n:3 * n + 3], Rn)
        # trial history of the elements around n
        assert np.abs(H_o[els] - es["h_new"]).max() <= tol["h"] * max(1.0, np.abs(es["h_new"]).max())
        # stiffness column of dof 3n+1 on the free rows of the elements around n
        j = 3 * int(n) + 1
        if j not in cols:
            continue
        col = np.zeros(mesh.n_dof)
        for k, el in enumerate(els):
            a = int(np.nonzero(conn[el] == n)[0][0])
            rows = (3 * conn[el][:, None] + np.arange(3)[None, :]).ravel()
            np.add.at(col, rows, es["Ke"][k][:, 3 * a + 1])
        rows = np.unique((3 * conn[els][:, :, None] + np.arange(3)).ravel())
        rows = rows[free[rows]]
        scale_K = np.abs(es["Ke"]).max()
        assert np.abs(cols[j][rows] - col[rows]).max() <= tol["K"] * scale_K
        # nothing outside the elements around n
        outside = np.setdiff1d(np.nonzero(free)[0], rows)
        assert np.abs(cols[j][outside]).max() == 0.0


def _compression_closed_form(t, X):
    """Homogeneous uniaxial compression along x (roller symmetry, Swift hardening, G + H = 1,
    r11 = 1): |eps11| = sigma_y(alpha)/E + alpha while plastic, T11 = -sigma_y(alpha),
    eps_p = alpha diag(-1, H, G), eps22 = -nu T11/E + H alpha, eps33 = -nu T11/E + G alpha."""
    E, nu, K, e0, n, G_, H_ = 70000.0, 0.33, 500.0, 0.01, 0.2, 0.30, 0.70
    e11 = np.log1p(-0.1 * t)
    m = -e11
    a = 0.0
    if K * e0 ** n / E < m:
        for _ in range(60):
            r = K * (e0 + a) ** n / E + a - m
            a -= r / (K * n * (e0 + a) ** (n - 1) / E + 1.0)
    T11 = -(K * (e0 + a) ** n) if a > 0 else E * e11
    e22 = -nu * T11 / E + H_ * a
    e33 = -nu * T11 / E + G_ * a
    u = np.stack([X[:, 0] * np.expm1(e11), X[:, 1] * np.expm1(e22), X[:, 2] * np.expm1(e33)], 1)
    return u.ravel(), a


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_config2h_fullsize_closed_form(precision):
    """The first load steps of ten (10 % compression in total; every step is plastic) on the
    full 100^3 cube: three with the mixed defaults, two in FP64 with the tight tolerances
    (newton_rtol 1e-12, pcg_rtol 1e-13) that 1e-10 needs at this size (1e-11 / 1e-12 leaves
    4e-10)."""
    mesh, bc, mat, ts = inputs.config2h_problem(N, 10)
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    ns = 2 if precision == "fp64" else 3
    with hfe.from_inputs(mesh, bc, mat, precision=precision, **opts) as s:
        hist = np.empty((7, mesh.n_el * 8))
        u, st = s.forward(ts[:ns], hist_out=hist)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for k in range(ns):
        uex, a = _compression_closed_form(ts[k], mesh.X)
        assert a > 0
        assert np.abs(u[k] - uex).max() <= tol * np.abs(uex).max(), (k, np.abs(u[k] - uex).max())
    _, a = _compression_closed_form(ts[ns - 1], mesh.X)
    assert np.abs(hist[6] - a).max() <= (1e-12 if precision == "fp64" else 1e-6) * max(a, 1.0)
