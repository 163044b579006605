"""The F-bar element (Sec. 2.2.4, Eq. Fbar) on the GPU against the oracle's F-bar element:
one tangent sweep on a distorted mesh with a mixed elastic/plastic state (residual, the
non-symmetric tangent through the exported block-CSR, trial history), whole forward runs
solved with BiCGSTAB (the homogeneous closed form, and a reduced perforated plate against the
oracle's forward), and the discrete adjoint (BiCGSTAB on the transposed tangent) against
central differences of the oracle's F-bar forward solve."""
import numpy as np
import pytest

from oracle import element, solver
from paper_2606_17390_b300 import hfe, inputs
from tests._helpers import bsr_to_csr, hist_oracle_to_soa, mixed_state, rel_inf

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(R=1e-11, K=1e-9, h=1e-12), "mixed": dict(R=2e-5, K=1e-4, h=1e-5)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fbar_sweep_vs_oracle(precision):
    mesh = inputs.distorted_box_mesh(4, seed=5, amp=0.2)
    keep = np.arange(mesh.n_el) != 7              # ragged tail
    mesh = inputs.Mesh(X=mesh.X, conn=mesh.conn[keep])
    mat = inputs.config0_material()
    u, hist = mixed_state(mesh, 31)
    conn = mesh.conn.astype(np.int64)
    es = element.element_sweep(mesh.X, conn, u, hist, mat.theta_vector(), "swift", fbar=True)
    assert 0.05 < es["gp"]["plastic"].mean() < 0.95
    prob = solver.Problem(X=mesh.X, conn=conn, fixed_dof=np.zeros(0, np.int64), fixed_val=np.zeros(0),
                          theta=mat.theta_vector(), hardening="swift", fbar=True)
    Ro, Ko = solver.assemble_R(prob, es["Re"]), solver.assemble_K(prob, es["Ke"])
    assert abs(Ko - Ko.T).max() > 1e-6 * abs(Ko).max()           # the F-bar tangent is not symmetric
    with hfe.Solver(mesh.X, mesh.conn, np.zeros(0, np.int64), np.zeros(0), mat.theta_vector(), "swift",
                    precision=precision, fbar=1) as s:
        s.set_state(np.zeros(mesh.n_dof), hist_oracle_to_soa(hist))
        Ht = np.empty((7, 8 * mesh.n_el))
        R, _, st = s.sweep(u, 1.0, tangent=True, hist_out=Ht)
        K = bsr_to_csr(*s.get_bsr(), mesh.n_nodes)
    tol = TOL[precision]
    assert rel_inf(R, Ro) < tol["R"], rel_inf(R, Ro)
    dK = (K - Ko).tocsr()
    assert np.abs(dK.data).max() / np.abs(Ko.data).max() < tol["K"]
    ho = hist_oracle_to_soa(es["h_new"])
    assert np.abs(Ht - ho).max() / np.abs(ho[:6]).max() < tol["h"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fbar_forward_closed_form_and_plate(precision):
    from tests.test_oracle_global import _uniaxial_closed_form
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    tol = 1e-10 if precision == "fp64" else 1e-5
    mesh, bc, mat, ts = inputs.config0_problem(n=3, n_steps=5)
    with hfe.from_inputs(mesh, bc, mat, precision=precision, fbar=1, **opts) as s:
        u, st = s.forward(ts)
    for n, t in enumerate(ts):
        uex = _uniaxial_closed_form(t, mesh)[0]
        assert np.abs(u[n] - uex).max() < tol * np.abs(uex).max()
    mesh, bc, mat, ts = inputs.config1_problem(nx=16, ny=8, nz=2, n_steps=20)
    ts = ts[:4]
    us, _, infos = solver.forward(solver.from_inputs(mesh, bc, mat, fbar=True), ts, rtol=1e-13)
    assert infos[-1]["plastic"] > 0
    with hfe.from_inputs(mesh, bc, mat, precision=precision, fbar=1, **opts) as s:
        u, st = s.forward(ts)
    for n in range(len(ts)):
        assert np.abs(u[n] - us[n]).max() < tol * np.abs(us[n]).max(), (n, np.abs(u[n] - us[n]).max())


@pytest.fixture(scope="module")
def fbar_fd_gradient():
    """The rotated Voce problem of the adjoint tests with the F-bar element: target = the
    oracle's F-bar forward at theta_true plus seeded noise; at theta = theta_true (1 + 0.1 U),
    dJ/dtheta_q by central differences of J over the oracle's FP64 forward (h = 1e-6 |theta_q|)."""
    mesh = inputs.box_mesh(4, 2, 1, 4.0, 2.0, 1.0)
    bc = inputs.clamp_displace_bcs(mesh, (0.08, 0.02, 0.0))
    mat = inputs.config1_material()
    a = np.deg2rad(30.0)
    mat.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    ts = inputs.load_factors(4)
    th_true = mat.theta_vector()
    u_gt, _, infos = solver.forward(solver.from_inputs(mesh, bc, mat, th_true, fbar=True), ts, rtol=1e-13)
    assert all(i["plastic"] > 0 for i in infos)
    rng = np.random.default_rng(4)
    u_gt = u_gt + 1e-3 * np.abs(u_gt).max() * rng.standard_normal(u_gt.shape)
    th = th_true * (1 + 0.1 * rng.uniform(-1, 1, 11))

    def J(t):
        us, _, _ = solver.forward(solver.from_inputs(mesh, bc, mat, t, fbar=True), ts, rtol=1e-13)
        return solver.objective(us, u_gt)

    fd = np.empty(11)
    for q in range(11):
        e = np.zeros(11)
        e[q] = 1e-6 * abs(th[q])
        fd[q] = (J(th + e) - J(th - e)) / (2 * e[q])
    return mesh, bc, mat, ts, u_gt, th, J(th), fd


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fbar_adjoint_vs_oracle_finite_differences(fbar_fd_gradient, precision):
    mesh, bc, mat, ts, u_gt, th, Jo, fd = fbar_fd_gradient
    opts = dict(newton_rtol=1e-12, pcg_rtol=1e-13) if precision == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=precision, theta=th, fbar=1, **opts) as s:
        J, g, st = s.adjoint(ts, u_gt)
    g = g[0]
    assert abs(J - Jo) < 1e-8 * Jo
    assert np.linalg.norm(g - fd) < 1e-6 * np.linalg.norm(fd), (g, fd)
    # per component: central differences carry the forward's convergence noise (about 1e-13 J)
    # divided by h, ~1e-12 absolute here, which is the floor for the smallest components
    big = np.abs(fd) > 1e-3 * np.abs(fd).max()
    assert np.all(np.abs(g[big] - fd[big]) < 1e-6 * np.abs(fd[big]) + 1e-7 * np.abs(fd).max()), (g, fd)
