"""CPU oracle for the P3 Helmholtz system — TEST INFRASTRUCTURE, not the product.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg may
import this package. It shares no code with the CUDA path: its own P3 basis,
quadrature (Stroud conical-product Gauss-Jacobi rules), dof numbering,
assembly and a sparse direct solve (SciPy SuperLU) in complex128.

What it computes (Sec. "Tetrahedral finite element method", Eq. eqh / eq1):
the Galerkin P3 discretisation of -Lap u - k^2 u = s on a tet mesh with
k = omega / c, first-order absorbing (Robin) faces d_n u - i k u = g,
homogeneous Dirichlet on the free surface, and the discrete solution
u = A^{-1} F. The two-level ORAS preconditioner (Eq. 2lvl, Eq. oras) changes
only how fast GMRES reaches that u, so the converged GPU wavefield is
compared with this direct solution.

Pins (tests/test_oracle_*.py) tie each function to the mathematics:
Lagrange property and partition of unity of the basis, exact monomial
integrals of the quadrature, annihilation of constants and exact energy of
linear fields by the stiffness matrix, element and face volumes of the mass
matrices, exact reproduction of cubic manufactured solutions, h^4 decay of
the L2 error of a plane wave with impedance data, and dense brute force.
"""
