"""FP64 CPU oracle for the multiscale lookup-table stiffness assembly.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or execute
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline/reference leg use it.  It shares no code with the CUDA library.

It is written to be checked against the paper by eye, in the paper's notation:

* ``bspline``     -- B-spline bases by the Cox-de Boor recursion (eq. 1-4).
* ``quadrature``  -- Gauss-Legendre rules and the Lagrange interpolation basis.
* ``micro``       -- the reference tile T^r (eq. 3): patches, numbering, I_coo (eq. 56).
* ``tables``      -- the stiffness lookup table (eq. 49-52, 57) by element quadrature.
* ``pullback``    -- the macro field A_ij (eq. 37) through the curvilinear
                     formalism of appendix A (eq. 79-97), literally.
* ``macro``       -- tile maps M^(t) (eq. 7-8) and their Jacobians.
* ``assembly``    -- global numbering/CSR, the lookup ("pi") form (eq. 50, 58)
                     and the standard full-Gauss ("bullet") form of Sec. 3.3.
* ``invariants``  -- rigid-body modes, constant-strain energy, E_mat (eq. 62).
* ``adjoint``     -- u^T (dK/dP) u by complex-step differentiation (Sec. 4.1.2).
* ``mlp``         -- FP64 forward/backward of the width -> low-rank-table network.
"""
