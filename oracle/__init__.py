"""Plain CPU FP64 oracle for the CEED bake-off problems (test infrastructure only).

This package is the independent definition against which the CUDA path is
checked.  It is slow on purpose and shares no code with the CUDA path: it
builds every element matrix by naive full quadrature (no sum factorization),
assembles the global sparse matrix, removes the Dirichlet rows and columns and
runs textbook Jacobi-preconditioned CG.  Only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import it; the
product path never does.

Modules and the passages of the paper they follow:

* ``quadrature`` -- GLL and GL points and weights (Sec. 4, after Eq. (18); Table 1).
* ``basis``      -- Lagrange interpolants h_i on the GLL points and their derivatives (Eq. (18)).
* ``mesh``       -- the deformed-box mesh, the global-to-local map Q and the Dirichlet set
                    (Sec. 3, Eqs. (18), (20), (21)).
* ``element``    -- element stiffness and mass matrices by full quadrature
                    (Eqs. (6)-(7), (14)-(15) with the quadrature of Table 1).
* ``assemble``   -- A = Q^T A_L Q and B = Q^T B_L Q (Eq. (21)), Dirichlet restriction.
* ``pcg``        -- diagonally preconditioned CG (Sec. 3).
* ``problems``   -- the bake-off problems BP1/BP3/BP5/BP6 built end to end.
* ``adjoint``    -- dJ/dkappa for -div(kappa grad u) = f (Eq. (4) with mu = kappa).

Equation numbers follow the order of the paper's numbered displays.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, library routines, invariants and brute force; none is "parity unpinned".
"""
