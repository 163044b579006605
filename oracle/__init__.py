"""Plain FP64 CPU oracle for the hex8 Gauss-point sweep, the global Newton solve and the
discrete adjoint of finite-strain Hill-48 plasticity in logarithmic strain space.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or executes this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, header, table or
constant generator with ``paper_2606_17390_b300`` (the CUDA path); both sides receive the
same arrays from ``paper_2606_17390_b300.inputs``, which holds no arithmetic of the method.

Modules
-------
material  : one Gauss point — geometric pre-processor (Sec. 2.2.2 (a), Eq. c_decomp),
            log-space elasticity (Eq. T), Hill-48 yield (Eq. Phi_hill, App. A.1),
            hardening (Eq. Hard), closest-point projection with the Scherzinger line
            search (Eq. local_cpp, Eq. local_solver, App. B, App. C), implicit
            differentiation of the local solve (App. D), geometric post-processor
            (Eq. proj_lagrange, Eq. pk_stress) and the first Piola-Kirchhoff tangent.
element   : hex8 trilinear element with 2x2x2 Gauss quadrature (Sec. 2.2.4).
solver    : assembly, Dirichlet elimination, global Newton (Eq. Stiffness_mat), load-step
            loop, objective (Sec. 2.3), discrete adjoint (Eq. dR_u, Eq. main_grad,
            Algorithm adjoint_ad), direct sensitivity, central finite differences
            (Algorithm finite_difference).

Pins (tests/test_oracle_*.py, marked "not gpu"): Hill-48 closed-form uniaxial yield
stresses and r-values, the homogeneous uniaxial closed form of the whole forward solve,
elastic and plastic patch tests, plastic incompressibility (tr eps_p = 0, i.e. det G_p = 1),
Kuhn-Tucker conditions and objectivity, the von Mises radial-return special case, finite
differences of the element residual (consistent tangent), an independent complex-step route
through a non-spectral matrix logarithm for the spectral derivatives, and adjoint =
direct sensitivity = central finite differences.
"""
