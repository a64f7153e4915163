"""CPU oracle for the w-BFBT Stokes solver (Rudi, Stadler & Ghattas, arXiv 1607.03936).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
and the bench's CPU-baseline leg may import anything from this package.  It
shares no code, tables or constants with the CUDA path: every quantity
(GLL nodes, derivative matrices, pressure basis, operators, transfers,
smoother, Krylov method) is computed here from its definition, in float64,
with assembled SciPy sparse matrices and sparse-direct or dense solves.

Modules
-------
gll        1-D GLL nodes/weights, Lagrange derivatives, the P_{k-1} monomial basis
mesh       structured hexahedral brick: node and element numbering
sinker     multi-sinker viscosity and forcing (Sec. 2.1)
operators  assembled A, B, B^T, lumped weights C/D, K_w, Q_k Poisson L_c
multigrid  nested transfers, coefficient coarsening, Chebyshev-Jacobi, V-cycles
krylov     right-preconditioned flexible GMRES(m)
wbfbt      w-BFBT (Eq. wbfbt), block preconditioner (Eq. precond-stokes), solve
mapped     A, B and the load vector on mapped (isoparametric) hexahedra; the mapped solve

Parity status: every function is pinned by a CPU test against closed forms,
symbolic integrals, invariants or brute force, except the upper spectral bound
of the w-BFBT-preconditioned Schur complement (Theorem 3.1), whose constants
the paper leaves unknown: that quantity is "parity unpinned" and is only
reported.
"""
