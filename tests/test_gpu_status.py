"""Determinism and error statuses of the Gauss-point sweep (hfe_gp_sweep): two sweeps of the
same state give bit-identical residuals and tangents (the element colouring leaves one
writer per block and launch, so no floating-point atomics reorder sums); an inverted element
and a displacement that is not a number return HFE_EDETJ, a local return mapping cut off
before it converges returns HFE_ELOCAL; after an error the handle sweeps as before."""
import numpy as np
import pytest

from paper_2606_17390_b300 import hfe, inputs
from tests._helpers import hist_oracle_to_soa, mixed_state

pytestmark = pytest.mark.gpu

HFE_EDETJ, HFE_ELOCAL = -4, 2


def _solver(mesh, precision, **options):
    th = inputs.config0_material().theta_vector()
    return hfe.Solver(mesh.X, mesh.conn, np.zeros(0, np.int64), np.zeros(0), th, "swift", precision=precision,
                      **options)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sweep_bit_identical_and_error_statuses(precision):
    mesh = inputs.distorted_box_mesh(3, seed=7, amp=0.2)
    u, hist = mixed_state(mesh, 41)
    with _solver(mesh, precision) as s:
        s.set_state(np.zeros(mesh.n_dof), hist_oracle_to_soa(hist))
        R1, _, st1 = s.sweep(u)
        K1 = s.get_bsr()[2]
        R2, _, _ = s.sweep(u)
        K2 = s.get_bsr()[2]
        assert 0 < st1["plastic_gps"] < 8 * mesh.n_el
        assert np.array_equal(R1, R2) and np.array_equal(K1, K2)
        inverted = -2.0 * mesh.X.ravel()                   # F = I + grad u = -I
        with pytest.raises(hfe.HfeError) as e:
            s.sweep(inverted)
        assert e.value.status == HFE_EDETJ
        bad = u.copy()
        bad[5] = np.nan
        with pytest.raises(hfe.HfeError) as e:
            s.sweep(bad)
        assert e.value.status == HFE_EDETJ
        R3, _, _ = s.sweep(u)
        K3 = s.get_bsr()[2]
        assert np.array_equal(R3, R1) and np.array_equal(K3, K1)


def test_local_return_mapping_cut_off_reports_elocal():
    mesh = inputs.distorted_box_mesh(3, seed=7, amp=0.2)
    u, hist = mixed_state(mesh, 41)
    with _solver(mesh, "fp64", local_maxit=1) as s:
        s.set_state(np.zeros(mesh.n_dof), hist_oracle_to_soa(hist))
        with pytest.raises(hfe.HfeError) as e:
            s.sweep(u)
        assert e.value.status == HFE_ELOCAL


HFE_EBARRIER = 5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_barrier_wait_that_runs_out(precision):
    """The one-launch Krylov solves wait at grid barriers with a bounded number of polls
    (options.barrier_spin_limit).  With the bound set to 0 every waiting CTA gives up at its
    first poll (no flag is left set for ever, no GPU fault): hfe_solve and hfe_forward return
    HFE_EBARRIER, the forward leaves the stored state at its last converged step, and the same
    handle, given the default bound again, solves bit for bit like a fresh handle."""
    mesh, bc, mat, ts = inputs.config2_problem(n=12, n_steps=4)
    b = np.random.default_rng(1).standard_normal(mesh.n_dof)
    b[bc.dof] = 0.0
    with hfe.from_inputs(mesh, bc, mat, precision=precision) as ref:
        ref.sweep(np.zeros(mesh.n_dof), 0.0)
        x_ref, st_ref = ref.solve(b)
        ref.set_state(None, None)
        u_ref, _ = ref.forward(ts)
    with hfe.from_inputs(mesh, bc, mat, precision=precision, barrier_spin_limit=0) as s:
        default = hfe.Options()
        hfe.lib().hfe_default_options(__import__("ctypes").byref(default), hfe.PRECISION[precision])
        s.sweep(np.zeros(mesh.n_dof), 0.0)
        with pytest.raises(hfe.HfeError, match="grid barrier") as e:
            s.solve(b)
        assert e.value.status == HFE_EBARRIER
        with pytest.raises(hfe.HfeError) as e:
            s.forward(ts[:1])
        assert e.value.status == HFE_EBARRIER
        u0, _ = s.get_state()
        assert s.get_load() == 0.0 and not np.any(u0)
        s.set_barrier_spin_limit(default.barrier_spin_limit)
        s.sweep(np.zeros(mesh.n_dof), 0.0)
        x, st = s.solve(b)
        assert np.array_equal(x, x_ref) and st["pcg_iters"] == st_ref["pcg_iters"]
        s.set_state(None, None)
        u, _ = s.forward(ts)
        assert np.array_equal(u, u_ref)
    with pytest.raises(hfe.HfeError) as e:
        hfe.from_inputs(mesh, bc, mat, precision=precision, barrier_spin_limit=-1)
    assert e.value.status == -1
