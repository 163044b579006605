"""Writes plate_forward_50x25x2.npz: the FP64 oracle's forward solve of the perforated plate
(the config-1 problem at 50 x 25 x 2 elements, Voce hardening, all 20 load steps, Newton to
1e-12), kept as a sample so that the GPU test need not rerun the oracle (about six minutes of
one host core).

Stored: the load factors; per step max |u| and u at 600 seeded dof indices; after the last
step max von Mises over all Gauss points and the von Mises stress at 1,000 seeded Gauss
points; the plastic Gauss-point count per step.  Run from the repository root:

    python tests/golden/make_plate_forward_50x25x2.py

It calls only the oracle and the seeded input generators."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import material, solver  # noqa: E402
from paper_2606_17390_b300 import inputs  # noqa: E402

NX, NY, NZ, N_STEPS = 50, 25, 2, 20
N_DOF_SAMPLE, N_GP_SAMPLE = 600, 1000


def main():
    mesh, bc, mat, ts = inputs.config1_problem(nx=NX, ny=NY, nz=NZ, n_steps=N_STEPS)
    us, _, infos = solver.forward(solver.from_inputs(mesh, bc, mat), ts, rtol=1e-12)
    rng = np.random.default_rng(2024)
    dofs = np.sort(rng.choice(mesh.n_dof, N_DOF_SAMPLE, replace=False))
    vm = material.von_mises(infos[-1]["sigma"].reshape(-1, 3, 3))
    gps = np.sort(rng.choice(vm.size, N_GP_SAMPLE, replace=False))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plate_forward_50x25x2.npz")
    np.savez_compressed(out, ts=np.asarray(ts), n_el=mesh.n_el, n_dof=mesh.n_dof, dofs=dofs,
                        u_max=np.abs(us).max(axis=1), u_sample=us[:, dofs], gps=gps, vm_sample=vm[gps],
                        vm_max=vm.max(), plastic=np.array([i["plastic"] for i in infos]))
    print(out, mesh.n_el, mesh.n_dof, [i["plastic"] for i in infos])


if __name__ == "__main__":
    main()
