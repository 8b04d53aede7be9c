"""FP64 CPU oracle for the beta-spread MAC elastic Helmholtz multigrid (arXiv 2307.03242).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this package. The product path (the
CUDA library and its Python binding) never imports or calls it.

The oracle is deliberately plain and slow: every operator is assembled as a
scipy.sparse matrix from the paper's one-dimensional factor matrices (standard
and beta-spread first derivatives, averaging, mass spreading), following the
paper's formulas literally. The smoother extracts each cell's (2d+1)x(2d+1)
submatrix from the assembled operator and solves it with a dense LU. Nothing is
blocked, fused or reordered. Complex FP64 throughout.

Modules
  discretization  -- Section 3.1 operator H^beta and its shifted version (Eq. 3.10, 3.11; 3D Section 5.3)
  transfer        -- Section 2.3 restriction / prolongation (Eq. pIntergrid, u2Intergrid)
  smoother        -- Section 2.3 / 3.2 Vanka box smoother, red-black, Jacobi within a colour
  multigrid       -- Algorithm 1 applied recursively (V-cycle), re-discretised coarse operators
  krylov          -- right-preconditioned restarted flexible GMRES (Saad 1993), modified Gram-Schmidt
  twogrid         -- Section 4.3 convergence factor in practice (Eq. convFactor) of the two-grid cycle
  lexvanka.c      -- the lexicographic (Gauss-Seidel over cells) Vanka sweep, compiled with gcc
  kaczmarz        -- Sections 3.2 / 5.3 coarsest solve: Schur complement eliminating p, FGMRES(5)
                     preconditioned by parallel hybrid (component-averaged) Kaczmarz steps
                     (the step itself in kaczmarz.c, compiled with gcc)
  adjoint         -- misfit gradient wrt lambda, mu, rho by the adjoint-state method (direct solves)

Parity status: every function is pinned by tests/test_oracle_*.py against the
paper's printed stencils, closed-form Fourier symbols, the two-grid symbol of
Eq. symbolTG, dense direct solves, plane-wave solutions and Table 1's two-grid
convergence factors (economic Vanka in lexicographic order); the adjoint
gradient by central finite differences of the misfit; the Kaczmarz coarsest solve by the full
system's direct solve, the row-projection property, the Bjorck-Elfving SOR identity, hand
averages, the solution as fixed point and monotone error decrease. The full Vanka smoother
has no printed symbol or factor in the paper; it is pinned by the single-cell
exactness property and by the converged solves only.
"""
from .discretization import Problem, assemble, apply, active_mask, coarsen, gamma_abl, dof_shape, window
from .transfer import restriction, prolongation
from .smoother import cell_dofs, cell_blocks, red_black_sweep, vanka_cell_update
from .multigrid import Hierarchy, vcycle
from .krylov import fgmres

__all__ = ["Problem", "assemble", "apply", "active_mask", "coarsen", "gamma_abl", "dof_shape", "window",
           "restriction", "prolongation", "cell_dofs", "cell_blocks", "red_black_sweep",
           "vanka_cell_update", "Hierarchy", "vcycle", "fgmres"]
