"""CPU oracle for the spline-collocation Faddeev-Merkuriev solve.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may import it.  The product path (the CUDA library and its Python binding)
never imports, calls or links anything here, and this package never imports
the product.

It is a plain, slow, obviously-correct restatement of the paper's method in
NumPy / SciPy, in float64:

* ``splines``  -- cubic Hermite basis, node maps, Gauss-point collocation
  (Section 3.1; Section 4 node maps and Gauss collocation);
* ``physics``  -- masses, Jacobi rotation, Coulomb potentials, Merkuriev
  cut-off, Wigner d-functions and the parity-adapted F basis (Section 2);
* ``system``   -- the collocation matrices H and S of Eq. FM-lin assembled
  entry by entry from Eqs. FM-pre / FM-fin and Eqs. r-form / s-rot;
* ``precond``  -- the tensor-trick preconditioner of Eq. prec-2, step by step
  as Section 3.2 builds it (1D decompositions by LAPACK);
* ``solvers``  -- sparse-LU linear solves and shift-invert Arnoldi
  (Eq. FM-lin) plus dense brute force for tiny grids.

Every function is pinned by tests under ``tests/`` against closed forms,
invariants, brute force and the energies printed in the paper.
"""
