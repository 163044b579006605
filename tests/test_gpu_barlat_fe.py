"""The Barlat Yld2004-18p material in the hex8 path (hfe_set_barlat, FP64 and mixed handles): the tangent sweep
on a distorted mesh with a mixed elastic/plastic state against the oracle's element with the
Barlat stress update (residual, tangent through the exported block-CSR, trial history);
forward runs against the oracle's forward; the isotropic model against the GPU's isotropic
Hill-48 forward; switching back to Hill-48; and the refusals (adjoint, invalid material)."""
import numpy as np
import pytest

from oracle import barlat as BA
from oracle import element, solver
from paper_2606_17390_b300 import hfe, inputs
from tests._helpers import bsr_to_csr, hist_oracle_to_soa, hist_soa_to_oracle, mixed_state, rel_inf

pytestmark = pytest.mark.gpu

ONES = (1.0,) * 9
OPTS = dict(newton_rtol=1e-12, pcg_rtol=1e-13)
TOL = {"fp64": dict(R=1e-11, K=1e-9, h=1e-12, u=1e-10), "mixed": dict(R=2e-5, K=1e-4, h=1e-5, u=1e-5)}
CASES = [("fp64", "fp64"), ("fp64", "mixed"), ("mixed", "mixed")]   # (handle, projection)


def _material(iso=False, rotated=True):
    """The paper's Yld2004-18p coefficients (m = 8) at config 0's elasticity and Swift
    hardening, in a frame rotated by 30 degrees about z; or all coefficients 1 with m = 2."""
    m = inputs.barlat_verification_material()
    th = inputs.config0_material().theta_vector()
    m.E, m.nu, m.hardening, m.h = th[0], th[1], "swift", (th[8], th[9], th[10])
    if iso:
        m.c1, m.c2, m.m = ONES, ONES, 2
    if rotated:
        a = np.deg2rad(30.0)
        m.Theta = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])
    return m


def _local(m):
    return BA.local(BA.Barlat(m.c1, m.c2, m.m, m.Theta), m.E, m.nu, m.hardening, m.h)


@pytest.mark.parametrize("handle,projection", CASES)
def test_barlat_sweep_vs_oracle(handle, projection):
    mesh = inputs.distorted_box_mesh(3, seed=7, amp=0.2)
    u, hist = mixed_state(mesh, 41)
    m = _material()
    conn = mesh.conn.astype(np.int64)
    es = element.element_sweep(mesh.X, conn, u, hist, np.zeros(11), "swift", local=_local(m))
    assert 0.05 < es["gp"]["plastic"].mean() < 0.95
    prob = solver.Problem(X=mesh.X, conn=conn, fixed_dof=np.zeros(0, np.int64), fixed_val=np.zeros(0),
                          theta=np.zeros(11), hardening="swift")
    Ro, Ko = solver.assemble_R(prob, es["Re"]), solver.assemble_K(prob, es["Ke"])
    th = inputs.config0_material().theta_vector()
    with hfe.Solver(mesh.X, mesh.conn, np.zeros(0, np.int64), np.zeros(0), th, "swift", precision=handle) as s:
        s.set_barlat(m, precision=projection)
        s.set_state(np.zeros(mesh.n_dof), hist_oracle_to_soa(hist))
        Ht = np.empty((7, 8 * mesh.n_el))
        R, _, st = s.sweep(u, 1.0, tangent=True, hist_out=Ht)
        K = bsr_to_csr(*s.get_bsr(), mesh.n_nodes)
    tol = TOL[handle]
    assert abs(st["plastic_gps"] - int(es["gp"]["plastic"].sum())) <= (0 if handle == "fp64" else 2)
    assert rel_inf(R, Ro) < tol["R"], rel_inf(R, Ro)
    assert abs(K - Ko).max() < tol["K"] * abs(Ko).max()
    Hn = hist_soa_to_oracle(Ht, mesh.n_el)
    assert np.abs(Hn - es["h_new"]).max() < tol["h"]


@pytest.mark.parametrize("handle,projection", CASES)
def test_barlat_forward_vs_oracle(handle, projection):
    """Config 0's cube (3^3, roller symmetry, stretch along x) in 4 steps, anisotropic and
    rotated: every step's displacement against the oracle's forward (the local projection in
    FP64, or its FP32 iteration with the FP64 finish)."""
    mesh, bc, mat, ts = inputs.config0_problem(n=3, n_steps=4)
    m = _material()
    prob = solver.from_inputs(mesh, bc, mat)
    prob.local = _local(m)
    us, hs, infos = solver.forward(prob, ts, rtol=1e-13)
    assert infos[-1]["plastic"] > 0
    opts = OPTS if handle == "fp64" else {}
    with hfe.from_inputs(mesh, bc, mat, precision=handle, **opts) as s:
        s.set_barlat(m, precision=projection)
        u, st = s.forward(ts)
    for n in range(len(ts)):
        assert np.abs(u[n] - us[n]).max() < TOL[handle]["u"] * np.abs(us[n]).max(), (n, np.abs(u[n] - us[n]).max())


def test_isotropic_barlat_equals_isotropic_hill_on_gpu_and_switch_back():
    """All coefficients 1 with m = 2 and isotropic Hill-48 are both J2 plasticity: the two GPU
    forward runs agree; hfe_set_barlat(NULL) returns the handle to Hill-48."""
    mesh, bc, mat, ts = inputs.config0_problem(n=3, n_steps=4)
    th = inputs.config0_material().theta_vector().copy()
    th[2:8] = [0.5, 0.5, 0.5, 1.5, 1.5, 1.5]
    m = _material(iso=True, rotated=False)
    with hfe.from_inputs(mesh, bc, mat, precision="fp64", theta=th, **OPTS) as s:
        uh, _ = s.forward(ts)
        s.set_barlat(m)
        s.set_state(None, None)
        ub, st = s.forward(ts)
        s.set_barlat(None)
        s.set_state(None, None)
        uh2, _ = s.forward(ts)
    assert st["plastic_gps"] > 0
    assert np.abs(ub - uh).max() <= 1e-10 * np.abs(uh).max()
    assert np.array_equal(uh, uh2)


def test_barlat_refusals():
    mesh, bc, mat, ts = inputs.config0_problem(n=2, n_steps=2)
    m = _material()
    with hfe.from_inputs(mesh, bc, mat, precision="fp64") as s:
        s.set_barlat(m)
        u, _ = s.forward(ts)
        with pytest.raises(hfe.HfeError) as e:
            s.adjoint(ts, u)
        assert e.value.status == -1
        bad = _material()
        bad.m = 7
        with pytest.raises(hfe.HfeError):
            s.set_barlat(bad)
