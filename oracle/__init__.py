"""FP64 CPU oracle for the frequency-domain CQM-BEM single-layer solve.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference against which the CUDA library is checked.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  The product path (the C-ABI library and its
Python binding) never imports, calls or links anything here, and nothing here
imports the product.

It follows the paper (Seibel, "Boundary Element Methods for the Wave Equation
based on Hierarchical Matrices and Adaptive Cross Approximation") step by step:

* ``cqm``        -- CQM frequencies (eq. cqm_freq) and the R-scaled transforms
                    (eq. omega_n), written as plain O(L^2) sums.
* ``quadrature`` -- the element rules: Radon's 7-point rule, a collapsed
                    Gauss-Legendre rule, and the Sauter-Schwab singular rules.
* ``galerkin``   -- P0 Galerkin entries of the Laplace-domain single layer
                    (Sec. 3.2, eq. fundsol) and dense matrices V_l.
* ``incident``   -- the Galerkin right-hand side of a plane-wave pulse.
* ``dense``      -- the decoupled frequency-domain solve (Remark in Sec. 6.2):
                    forward transform, one LU solve per frequency, inverse
                    transform.
* ``cluster``    -- cluster tree (Def. 2) and block partition (Defs. 3-4,
                    eq. qadm).
* ``h2``         -- Chebyshev interpolation bases (eqs. degexp, uniformlr; Def. 5)
                    and the H^2-expanded matrices V_l.
* ``maca``       -- multivariate adaptive cross approximation (Sec. 5.1, Alg. 2).
* ``mot``        -- marching on in time with the CQM weights (Sec. 3.2, eq. dft),
                    the paper's own time stepping.
* ``dlayer``     -- the P0 Galerkin double layer (Sec. 2.2), its H^2 column
                    basis, and the direct formulation of the Dirichlet problem
                    (Sec. 7.2, eq. cqmdir) decoupled in frequency.
* ``mixed``      -- P1 elements, the adjoint double layer and the hypersingular
                    operator (Maue's form), dense and in H^2 form, and the mixed
                    boundary-value problem (Sec. 2.3 eq. wavegalform, Sec. 3.2 eq.
                    cqmgalapx) decoupled in frequency and by marching on in time.

Parity pins: every module is checked in ``tests/test_oracle_*.py`` against
closed forms, invariants or brute force.  The conventions the paper leaves
open (quadrature orders, near-singular threshold, cluster splitting and
ordering tie-breaks) are fixed by reading; they are shared with the CUDA path
by specification only and are "parity unpinned" as choices: any reading gives
a valid method, and only oracle-vs-CUDA agreement is gated for them.
"""
