"""CPU FP64 oracle of the p-multigrid spectral element Laplace solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never links, imports or calls it, and the oracle
shares no code with the library: every piece here is a plain restatement of
the paper's definitions (assembled sparse stiffness matrix, Galerkin Laplace
problem, Algorithms 1-3) in NumPy/SciPy, slow and obviously correct.

Modules:
  refelem   nodes, quadrature and Lagrange bases on triangles / prisms (Section 3.1)
  mesh      global node numbering, Dirichlet node sets, node coordinates
  assemble  geometric factors and the assembled stiffness matrix (Eq. laplaceproblemdiscrete)
  solvers   Dirichlet lifting, direct solve, transfers (Section 4.1), Chebyshev
            smoothing, V-cycle (Algorithm 1), PDC (Algorithm 2), PCG (Algorithm 3), FGMRES
  mlp       the per-element correction network (forward / backward / Adam) in FP64
  learned   one learned correction sweep (network correction, minimal-residual step,
            residual verdict with the Chebyshev fallback)

Parity pins: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and library routines; functions
without such a pin are marked "parity unpinned" in their docstring.
"""
