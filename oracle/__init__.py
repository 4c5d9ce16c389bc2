"""Plain, slow, FP64 CPU oracle for the semi matrix-free twogrid-preconditioned FGMRES.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA library.

What it computes (the exact discrete method, assembled, in complex128):
  * fem.py    -- Lagrange P1/P2 triangles and P1 Kuhn tetrahedra on the unit
                 square/cube; element matrices by exact integration of
                 barycentric monomials; assembled CSR K, M, B (Sec. 2,
                 eq. discreteproblem / sys_matrix); load vectors; canonical
                 interpolation P between the 2h and h spaces (Sec. 4);
                 heterogeneous wavenumbers k(x) = k_max mu(x) with one value
                 per simplex (Sec. 2 with k in L^inf, Sec. 6).
  * solver.py -- damped Jacobi, the twogrid V(nu,nu)-cycle of Algorithm 1 with
                 a direct coarse solve, and flexible GMRES(m) (Saad 1993) with
                 modified Gram-Schmidt and complex Givens rotations (Sec. 4);
                 problems with constant or heterogeneous k.
  * qfem.py   -- tensor-product Q_p elements (p = 1..3) on squares / cubes, the
                 paper's own discretisation (Sec. 2), with optional element-local k.
  * shiftmap.py -- the fitted shift-exponent map of eq. shiftexp with the
                 weights of Table tab:optweights (Sec. 5).
  * lfa.py    -- local Fourier analysis of the twogrid method (Sec. 3): stencil
                 symbols, the 4 x 4 harmonic matrix T_hat, rho_loc(sigma) and
                 sigma_c, for the paper's Q1 and the solver's P1 Kuhn triangles.

Pins: see tests/test_oracle_*.py. Every function is pinned by a closed form,
an invariant, a textbook special case or brute force; the iteration counts
of the paper's own experiments are not reproducible here (other elements,
heterogeneous k from unavailable velocity models): parity unpinned against
the paper's tables, pinned against the mathematics.
"""
