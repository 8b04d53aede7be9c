"""Multigrid V-cycle on the shifted operator (oracle; test infrastructure only).

Algorithm 1 (two-grid cycle) applied recursively (Section 2.2): one recursive call gives the
V-cycle, two recursive calls (the second starting from the first one's result) the W-cycle, and
the K-cycle uses the two recursive calls as preconditioners of two steps of a flexible Krylov
method for the coarse problem (Section 2.2, after Notay and Vassilevski; here generalised
conjugate residuals, GCR(2), since the operator is not Hermitian): nu_1 pre-relaxations, residual restriction
r_2h = R(q - A_h u), coarse problem, correction u += P e_2h, nu_2
post-relaxations. The coarse operators are re-discretisations of the shifted
operator (Remark 2.1 and Section 3.2: the same stencil on the 2h grid, with the
same omega, beta and shift alpha added to the attenuation). The coarsest level
is solved either exactly (dense or sparse LU of the coarsest operator, the paper's 2D
choice in Section 3.2), by the paper's 3D choice (Sections 3.2 and 5.3: FGMRES(5) on the
p-eliminated Schur complement, preconditioned by parallel hybrid Kaczmarz steps, to a 0.1 drop;
oracle/kaczmarz.py), or inexactly by a fixed number of red-black Vanka sweeps from a zero guess.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .discretization import Problem, assemble, coarsen, active_mask
from .transfer import restriction, prolongation
from .smoother import cell_dofs, cell_blocks, cell_colour, red_black_sweep

# Damping w by hierarchy depth (Section 5.2: 0.55, 0.35, 0.25 for 2, 3, 4 levels; 0.2 for 5 is
# a reading, since the paper stops at 4 levels).
DEFAULT_DAMPING = {1: 0.55, 2: 0.55, 3: 0.35, 4: 0.25, 5: 0.2, 6: 0.2, 7: 0.2, 8: 0.2}


class Hierarchy:
    def __init__(self, pb: Problem, levels: int, alpha: float, damping=None, nu_pre: int = 2,
                 nu_post: int = 2, coarse: str = "dense", coarse_sweeps: int = 0,
                 coarse_damping: float = 1.0, cycle: str = "V", smoother: str = "full",
                 coarse_box=2, coarse_coloured: bool = False, coarse_tol: float = 0.1,
                 coarse_steps: int = 10, coarse_kaczmarz_damping: float = 0.8, coarse_max_kaczmarz: int = 250):
        self.levels = levels
        self.cycle = cycle
        self.gamma_cycle = {"V": 1, "W": 2, "K": 2}[cycle]
        self.alpha = alpha
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.coarse, self.coarse_sweeps, self.coarse_damping = coarse, coarse_sweeps, coarse_damping
        if damping is None:
            damping = DEFAULT_DAMPING[levels]
        self.w = list(damping) if np.ndim(damping) else [float(damping)] * levels
        self.pbs = [pb]
        for _ in range(levels - 1):
            self.pbs.append(coarsen(self.pbs[-1]))
        # alpha: one shift for every level, or one per level (a deeper shift on coarse levels)
        self.alphas = list(alpha) if np.ndim(alpha) else [float(alpha)] * levels
        self.H = [assemble(p, self.alphas[l]) for l, p in enumerate(self.pbs)]
        self.R = [restriction(self.pbs[l], self.pbs[l + 1]) for l in range(levels - 1)]
        self.P = [prolongation(self.pbs[l], self.pbs[l + 1]) for l in range(levels - 1)]
        self.idx = [cell_dofs(p) for p in self.pbs]
        self.colour = [cell_colour(p) for p in self.pbs]
        self.smoother = smoother
        self.V = [cell_blocks(self.H[l], self.idx[l], economic=smoother == "economic") for l in range(levels)]
        last = levels - 1
        self.act_c = active_mask(self.pbs[last])
        if coarse == "dense":
            Hc = self.H[last][self.act_c][:, self.act_c].toarray()
            self.lu = sla.lu_factor(Hc)
        elif coarse == "sparse":
            # the same exact coarsest solve as "dense" (Sec. 3.2: LU in 2D), with a sparse LU for
            # coarsest grids whose dense matrix would not fit in memory
            self.splu = spla.splu(self.H[last][self.act_c][:, self.act_c].tocsc())
        elif coarse == "kaczmarz":
            from .kaczmarz import SchurSystem, box_partition
            self.schur = SchurSystem(self.pbs[last], self.alphas[last])
            self.kpart = box_partition(self.schur, coarse_box, coloured=coarse_coloured)
            self.kopts = dict(tol=coarse_tol, kaczmarz_steps_per_apply=coarse_steps,
                              damping=coarse_kaczmarz_damping, max_kaczmarz=coarse_max_kaczmarz)

    def smooth(self, l, b, x, count, w):
        for _ in range(count):
            x = red_black_sweep(self.H[l], self.V[l], self.idx[l], self.colour[l], b, x, w)
        return x

    def coarse_solve(self, b):
        last = self.levels - 1
        x = np.zeros_like(b)
        if self.coarse == "dense":
            x[self.act_c] = sla.lu_solve(self.lu, b[self.act_c])
        elif self.coarse == "sparse":
            x[self.act_c] = self.splu.solve(np.ascontiguousarray(b[self.act_c]))
        elif self.coarse == "kaczmarz":
            from .kaczmarz import hybrid_solve
            x, _, _ = hybrid_solve(self.schur, self.kpart, b, **self.kopts)
        else:
            x = self.smooth(last, b, x, self.coarse_sweeps, self.coarse_damping)
        return x


def vcycle(hier: Hierarchy, b, x=None, level: int = 0):
    """One V(nu_1, nu_2) cycle (or W-cycle, per the hierarchy) for H_s x = b on `level`;
    x=None means a zero initial guess."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    if level == hier.levels - 1:
        return hier.coarse_solve(b)
    x = np.zeros_like(b) if x is None else np.asarray(x, dtype=np.complex128).ravel().copy()
    H = hier.H[level]
    x = hier.smooth(level, b, x, hier.nu_pre, hier.w[level])
    r = b - H @ x
    bc = hier.R[level] @ r
    if hier.cycle == "K" and level + 1 < hier.levels - 1:
        ec = kcycle_correction(hier, bc, level + 1)
    else:
        ec = vcycle(hier, bc, None, level + 1)
        for _ in range(hier.gamma_cycle - 1):
            if level + 1 < hier.levels - 1:
                ec = vcycle(hier, bc, ec, level + 1)
    x = x + hier.P[level] @ ec
    x = hier.smooth(level, b, x, hier.nu_post, hier.w[level])
    return x


def kcycle_correction(hier: Hierarchy, r, level: int):
    """Two GCR steps for H_s e = r on `level`, each preconditioned by one recursive cycle:
    z1 = B r, q1 = A z1, a1 = <q1, r>/<q1, q1>, r2 = r - a1 q1;
    z2 = B r2, q2 = A z2, q2 -= (<q1, q2>/<q1, q1>) q1 (and z2 likewise), a2 = <q2, r2>/<q2, q2>;
    e = a1 z1 + a2 z2 (<a, b> = sum conj(a) b)."""
    A = hier.H[level]
    z1 = vcycle(hier, r, None, level)
    q1 = A @ z1
    n1 = np.vdot(q1, q1).real
    a1 = np.vdot(q1, r) / n1
    r2 = r - a1 * q1
    z2 = vcycle(hier, r2, None, level)
    q2 = A @ z2
    bt = np.vdot(q1, q2) / n1
    q2 = q2 - bt * q1
    z2 = z2 - bt * z1
    a2 = np.vdot(q2, r2) / np.vdot(q2, q2).real
    return a1 * z1 + a2 * z2
