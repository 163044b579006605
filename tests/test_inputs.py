"""The seeded synthetic inputs (paper_2606_17390_b300/inputs.py) against the recipes they
implement: sizes of the benchmark meshes, positive C3D8 orientation, one face-connected
component with solid grips for the perforated plate, config 4's holes as config 1's at twice
the resolution, the stated material parameter vectors, and determinism."""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_2606_17390_b300 import inputs

# C3D8 faces (outward normal irrelevant here)
FACES = ((0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7))
SIGNS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                  [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)


def _det_centre(mesh):
    Xe = mesh.X[mesh.conn]                                # (n_el, 8, 3)
    J = np.einsum("eai,aj->eij", Xe, SIGNS / 8.0)          # dX/dxi at the element centre
    return np.linalg.det(J)


def _n_components(mesh):
    f = np.sort(mesh.conn[:, FACES].reshape(-1, 4), axis=1)
    _, key = np.unique(f, axis=0, return_inverse=True)
    key = key.ravel()
    el = np.repeat(np.arange(mesh.n_el), 6)
    order = np.argsort(key, kind="stable")
    k, e = key[order], el[order]
    same = k[1:] == k[:-1]
    a, b = e[:-1][same], e[1:][same]
    A = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(mesh.n_el, mesh.n_el))
    return connected_components(A, directed=False)[0]


def test_config_sizes_and_materials():
    m0, _, mat0, t0 = inputs.config0_problem()
    assert (m0.n_el, m0.n_nodes, m0.n_dof, len(t0)) == (64, 125, 375, 10)
    assert np.allclose(t0, np.arange(1, 11) / 10.0, rtol=0, atol=1e-15)
    assert np.array_equal(mat0.theta_vector(), [70000.0, 0.33, 0.25, 0.30, 0.70, 1.5, 1.5, 1.5, 500.0, 0.01, 0.2])
    m1, _, mat1, t1 = inputs.config1_problem()
    assert (m1.n_el, m1.n_nodes, m1.n_dof, len(t1)) == (55780, 74080, 222240, 20)
    assert np.array_equal(mat1.theta_vector()[8:], [150.0, 120.0, 12.0]) and mat1.hardening == "voce"
    m2, _, _, t2 = inputs.config2_problem()
    assert (m2.n_el, m2.n_nodes, m2.n_dof, len(t2)) == (1000000, 1030301, 3090903, 10)


def test_meshes_are_positively_oriented():
    for mesh in (inputs.box_mesh(5, 4, 3), inputs.distorted_box_mesh(4, seed=3, amp=0.2),
                 inputs.config1_problem(nx=48, ny=24, nz=2, n_steps=2)[0]):
        assert (_det_centre(mesh) > 0).all()


def test_plate_recipe():
    m1 = inputs.config1_problem()[0]
    assert _n_components(m1) == 1
    c = m1.X[m1.conn].mean(axis=1)
    ix = np.floor(c[:, 0] / 0.5).astype(int)
    iy = np.floor(c[:, 1] / 0.5).astype(int)
    assert ((ix < 4).sum(), (ix >= 196).sum()) == (1600, 1600)           # 4 solid grip columns per end
    cols = np.unique(ix * 100 + iy)
    assert 0.65 * 20000 < cols.size <= 0.70 * 20000 + 2 * 4 * 100        # columns above the 70th percentile removed
    assert m1.n_el == 4 * cols.size                                      # through-thickness columns


def test_config4_holes_follow_config1_at_twice_the_resolution():
    m1 = inputs.config1_problem()[0]
    m4 = inputs.config4_problem()[0]
    assert _n_components(m4) == 1
    c1 = m1.X[m1.conn].mean(axis=1)
    solid = np.zeros((200, 100), bool)
    solid[np.floor(c1[:, 0] / 0.5).astype(int), np.floor(c1[:, 1] / 0.5).astype(int)] = True
    c4 = m4.X[m4.conn].mean(axis=1)
    inside = solid[np.floor(c4[:, 0] / 0.5).astype(int), np.floor(c4[:, 1] / 0.5).astype(int)]
    assert inside.mean() > 0.95, inside.mean()
    assert abs(m4.n_el / (4 * m1.n_el) - 1.0) < 0.05


def test_generators_are_deterministic():
    a = inputs.config1_problem(nx=48, ny=24, nz=2, n_steps=2)[0]
    b = inputs.config1_problem(nx=48, ny=24, nz=2, n_steps=2)[0]
    assert np.array_equal(a.X, b.X) and np.array_equal(a.conn, b.conn)
    c = inputs.config1_problem(nx=48, ny=24, nz=2, n_steps=2, seed=2)[0]
    assert c.n_el != a.n_el or not np.array_equal(c.conn, a.conn)
    assert np.array_equal(inputs.pi_plane_sample(100)[1], inputs.pi_plane_sample(100)[1])
