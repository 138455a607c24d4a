"""Independent FP64 CPU oracle for the step-off TEM forward model and its adjoint.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path
(``paper_2506_11657_gb300``) never imports, links or runs anything here, and
this package imports nothing from the product: the two share no code.  Inputs
come as plain arrays (the seeded workload generators build them).

Contents, each citing the passage it follows:

* ``yee``       -- assembled Yee edge discretisation: K, M, f, Q (Sec. 2.2).
* ``rational``  -- shared-pole rational family, RKFIT-style fit, uniform error,
                   conjugate-pair reduction (Sec. 3.2-3.3).
* ``solvers``   -- T0 dense eigendecomposition (Eq. (expm)), T1 sparse LU per
                   pole, T2 Jacobi-COCG per pole.
* ``tem``       -- forward d = sum_i Re(c_i Q (K - xi_i M)^{-1} f) (Eq. (rmj),
                   (rmjQ)) and the adjoint gradient w.r.t. log sigma (Sec. 4).
* ``halfspace`` -- closed-form central-loop halfspace response (Sec. 5 check).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
value fixed by the paper or by mathematics (see tests/test_oracle_*.py).  One
printed value is not reproduced: the closest pole pair of the degree-28 family
(Fig. 1 caption); the pole fit is pinned by the accuracy Table instead.
"""
