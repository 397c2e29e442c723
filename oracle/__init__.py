"""CPU FP64 oracle for the SC-4DVAR Gauss-Newton hot path (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The CUDA library never calls it, and it shares no code with the CUDA path:
the two sides meet only in ``sc4dvar_inputs`` (seeded draws, no arithmetic of
the method).

Everything here is plain numpy in float64, written for a reader who checks it
against the paper (Cheng, Rao, Sandu, Saibaba, "Randomized preconditioned
solvers for strong constraint 4D-Var data assimilation", arXiv 2401.15758):

* ``philox``    - Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
                  the Box-Muller map to standard normals used for Omega, Psi, v.
* ``rk4``       - classic RK4 step, its tangent-linear step and its discrete
                  adjoint step (Sandu's discrete RK adjoint, cited in Sec. 2.1).
* ``burgers``   - semi-discrete periodic Burgers right-hand side, its Jacobian and
                  the Jacobian transpose (Sec. 5.1 model, periodic reading).
* ``prior``     - circulant square root of the squared-exponential prior.
* ``fourdvar``  - the SC-4DVAR problem: cost (Eq. 4dvar_cf), gradient
                  (Eq. 4dvar_gradient), A and A^T of Eq. Rhalf, GN Hessian products.
* ``sketch``    - RandSVD (Alg. 1), Remark 1, Nystrom (Alg. 2), SingleView
                  (Alg. 3), adaptive RandSVD (Alg. 4), adaptive SingleView
                  (Alg. 5), adaptive Nystrom, the QR update of Alg. 6, the Woodbury
                  preconditioner (Eq. woodbury) and the kappa estimators
                  (Eqs. condtext, condtext2).
* ``solvers``   - PCG for Eq. pcgsystem, SketchSolv (Eq. dxsol) and the
                  Gauss-Newton loop with the reuse-or-recompute rule (Sec. 3.2).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, dense assembled matrices or published test vectors.
"""
