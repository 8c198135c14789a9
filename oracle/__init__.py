"""FP64 CPU oracle for the WADG strong-weak right-hand side (test infrastructure).

This package is test infrastructure, not product code: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline and reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library: it uses
its own orthonormal (modal) basis, its own Golub-Welsch quadrature and its own
geometry, and it reaches the library only through nodal values at the
equispaced lattice (the interface format).

Modules and the passages of Chan, Hewett & Warburton (arXiv:1608.03836) they
follow:
  polynomials  Jacobi / Dubiner bases and Gauss-Jacobi rules (Sec. 2, Sec. 4:
               quadrature exact to degree 2N+1 for the update)
  discretization  reference operators, mesh connectivity and geometric
               factors of the isoparametric map (Sec. 4.1, polynomiality of
               J dx^/dx and n J^f)
  wadg         strong-weak formulation (Sec. 4.1), exact-inverse DG and the
               weight-adjusted inverse M^-1 M_{1/J} M^-1 (Sec. 4, Eq. (matfree)
               of Sec. 6.2, Sec. 7 for c^2/J), pseudo-projection (Theorem in
               Sec. 3), LSRK45 (Sec. 5.2), energy and error diagnostics.
  adjoint      discrete adjoint of the RHS and of the LSRK step.

Every function that has no independent pin says "parity unpinned" in its
docstring; at present every function is pinned by tests in tests/.
"""
