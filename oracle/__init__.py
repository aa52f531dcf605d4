"""Plain FP64 CPU oracle for the Sparse Gauss-Newton (SGN) step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, calls or links it,
and this package imports nothing from the product path: the two share only
the seeded input generators in ``sgn_inputs``.

What is here, each written from the definition it cites:

* ``elements``     -- compressible neo-Hookean element energy, force,
                      Hessian and parameter column (Sec. 5 "Inverse Elastic
                      Design"; derivatives of Eq. optProb's constraint).
* ``system``       -- sparse assembly of dc/dx, dc/dp, the objective blocks
                      A, B, C (Eq. reducedGN), the saddle-point matrix of
                      Eq. sparseSystemGN, the dense Gauss-Newton Hessian
                      (Eq. HGN / reducedGN), the sensitivity matrix
                      (Eq. dxdp), the total gradient (Eq. totalGradient), the
                      adjoint multipliers (Appendix A, Theorem 2) and the
                      a-posteriori error bound of a computed step.
* ``equilibrium``  -- forward simulation: Newton's method with a
                      backtracking line search that keeps the potential
                      monotone (Sec. 5, "Computing Equilibrium States").
* ``learned``      -- the learned warm start of that Newton solve: RBF design
                      map, snapshot basis (SVD of the centred snapshots), the
                      GELU MLP with its backpropagated gradients, AdamW.

Parity pins: every function above is checked in ``tests/test_oracle_*.py``
against something other than itself (complex-step derivatives, the
linear-elastic closed form at F = I, finite differences of the equilibrium
map, brute-force Gauss-Newton from finite-difference Jacobians, Theorem 1,
Theorem 2, the saddle-point inertia; for ``learned``: the GELU closed form and
its finite differences, finite-difference MLP gradients, AdamW's first step in
closed form, orthonormality and exact reconstruction of low-rank snapshots, the
RBF map at a centre).  No function here is "parity unpinned".
"""
