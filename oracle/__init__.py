"""Plain, slow CPU oracle for the Whittle–Matérn surface sampler.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import, call or execute it.  It shares no code with the
CUDA library under ``paper_2605_24882_gb300/csrc``.

It computes, in float64 with numpy/scipy, exactly what the sampler defines:

* ``bspline``    -- Cox–de Boor B-spline bases (Definition 2.1, Sec. 2.1) and
                    the p-open dyadic knot vectors Xi_{j,p} (Sec. 2.3).
* ``geometry``   -- the six-patch cube-sphere and the periodic torus maps F_m,
                    first fundamental form K_m and surface measure a_m (Sec. 3.2).
* ``space``      -- the C0-glued spline space S^0_{j,p} (Eq. def::space2):
                    global DOF numbering and element connectivity.
* ``assembly``   -- mass and stiffness matrices by Gauss quadrature of the
                    pulled-back forms (Eqs. eq:mass, eq:stiffness), assembled CSR.
* ``philox``     -- Philox4x32-10 (Salmon et al., SC'11) and the normal transform.
* ``noise``      -- white-noise load vectors b = sum_q sqrt(w_q a_q) xi_q phi(x_q),
                    whose covariance is the quadrature mass matrix (Sec. 3.3).
* ``fractional`` -- the integer/fractional split of beta and the improved split
                    (Sec. 3.4), sinc nodes and weights (Eq. eq:beta-approx), and
                    the fields u_s by direct sparse solves and an explicit sum;
                    the field-loss gradient by the adjoint identity.
* ``nurbs``      -- NURBS patches as geometry maps (Sec. 2.2) with the Surface
                    interface, so the glued space and assembly apply to them.
* ``sqrt_mass``  -- loads f = sqrt(M) y by the Hale–Higham–Trefethen sum
                    (Sec. 3.3, Eq. eq:sqrt) and bounds of the mass spectrum.

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints (Figs. 1, 4, 5), closed forms (areas, spherical harmonics,
gnomonic area element), invariants (S 1 = 0, symmetry, B B^T = M) and brute
force (dense generalised eigen-decomposition, dense matrix square roots).
``tests/test_oracle_mutants.py`` plants mistakes in a copy of this package and
checks that the pins catch each one.  No function here is
"parity unpinned".
"""
