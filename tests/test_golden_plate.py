"""The stored oracle forward of the 50 x 25 x 2 perforated plate (tests/golden/
plate_forward_50x25x2.npz, written by tests/golden/make_plate_forward_50x25x2.py) still matches
its inputs and the oracle: the mesh sizes and load factors of inputs.config1_problem, the
sample indices in range, and the first load step recomputed by the oracle (about 15 s on one
core) equal to the stored sample."""
import os

import numpy as np

from oracle import material, solver
from paper_2606_17390_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "plate_forward_50x25x2.npz")


def test_stored_plate_forward_matches_inputs_and_oracle():
    g = np.load(GOLDEN)
    mesh, bc, mat, ts = inputs.config1_problem(nx=50, ny=25, nz=2, n_steps=20)
    assert mesh.n_el == int(g["n_el"]) and mesh.n_dof == int(g["n_dof"])
    assert np.array_equal(np.asarray(ts), g["ts"])
    assert g["u_sample"].shape == (20, g["dofs"].size) and g["dofs"].max() < mesh.n_dof
    assert g["gps"].max() < 8 * mesh.n_el
    assert np.all(np.diff(g["plastic"]) >= 0) and 0 < g["plastic"][-1] < 8 * mesh.n_el
    us, _, infos = solver.forward(solver.from_inputs(mesh, bc, mat), ts[:1], rtol=1e-12)
    assert np.abs(us[0][g["dofs"]] - g["u_sample"][0]).max() <= 1e-12 * g["u_max"][0]
    assert abs(np.abs(us[0]).max() - g["u_max"][0]) <= 1e-12 * g["u_max"][0]
    assert infos[0]["plastic"] == g["plastic"][0]
    vm = material.von_mises(infos[0]["sigma"].reshape(-1, 3, 3))
    assert vm.max() < float(g["vm_max"])          # the plate hardens: step 1 below step 20
