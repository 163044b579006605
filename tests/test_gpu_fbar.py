"""The F-bar element (Sec. 2.2.4, Eq. Fbar) on the GPU against the oracle's F-bar element:
one tangent sweep on a distorted mesh with a mixed elastic/plastic state (residual, the
non-symmetric tangent through the exported block-CSR, trial history), whole forward runs
solved with BiCGSTAB (the homogeneous closed form, and a reduced perforated plate against the
oracle's forward), and the adjoint refused."""
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
        with pytest.raises(hfe.HfeError) as e:
            s.adjoint(ts, us)
        assert e.value.status == -1
    for n in range(len(ts)):
        assert np.abs(u[n] - us[n]).max() < tol * np.abs(us[n]).max(), (n, np.abs(u[n] - us[n]).max())
