"""Hybrid Kaczmarz-GMRES coarsest-level solve (oracle; test infrastructure only).

Section 3.2 ("coarsest grid solution") and Section 5.3: the coarsest system H_s x = b is
reduced to the displacement unknowns by the algebraic Schur complement that eliminates p
(the p-p block is diagonal, diag(1/(lambda+mu)), so it is inverted exactly),

    S u = f_u - A_up C^-1 f_p,   S = A_uu - A_up C^-1 A_pu,   C = diag(1/(lambda+mu)),
    p = C^-1 (f_p - A_pu u),

which returns to the displacement-only form Eq. (2.3). S is solved by FGMRES(5) preconditioned
by a fixed number of parallel hybrid Kaczmarz steps from a zero guess (10 steps, damping 0.8),
until the relative residual of the Schur system drops to 0.1, with at most 250 Kaczmarz steps in
all (25 preconditioner applications).

Parallel hybrid Kaczmarz (after Gordon and Gordon's component-averaged row projections, the
method the paper builds on): the domain is divided into sub-regions, boxes of cells; the rows of
a sub-region are the Schur rows of the displacement faces of its cells, swept sequentially in a
fixed order on a private copy of the unknowns the sub-region reaches; all sub-regions start from
the same iterate, and each unknown is then replaced by the mean of the sub-regions' copies of it
(oracle/kaczmarz.c holds the step itself).

Readings (the paper gives only the sub-region count of its 8-core runs):
* sub-regions are boxes of `box` cells per axis (the last box on an axis may be shorter), rows in
  a box ordered component by component, each component's faces with x1 fastest; boxes in
  lexicographic order (x1 fastest);
* the reach of a box for component c' is the box dilated by the footprint of the Schur stencil:
  1 cell down along x_c', 2 cells down along every other axis and 1 cell up along every axis
  (restricted to the domain and to active unknowns); the mean of an unknown is over the boxes
  whose reach holds it;
* a Kaczmarz step sweeps each row once, in the forward order above (no backward sweep);
* `coloured=True` instead sweeps all rows as ONE sub-region, boxes taken colour by colour
  (2^d colours by box-index parity) -- with boxes of at least 4 cells per axis, rows of
  same-coloured boxes touch disjoint unknowns, so the boxes of one colour can be swept in parallel
  and the step equals one sequential Kaczmarz sweep in that order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

from .discretization import Problem, assemble, active_mask
from .krylov import fgmres


# ---------------------------------------------------------------- Schur complement
def _eliminate(Huu, A_up, cinv, A_pu):
    """S = A_uu - A_up C^-1 A_pu."""
    return (Huu - A_up @ sp.diags(cinv) @ A_pu).tocsr()


class SchurSystem:
    """The p-eliminated form of H_s on one grid.

    S: CSR over the active displacement unknowns (u_act: their positions in the full DOF vector,
    in the full vector's order); A_up, A_pu: the coupling blocks restricted to those unknowns;
    cinv: the diagonal of C^-1 = lambda + mu per cell."""

    def __init__(self, pb: Problem, shift: float):
        self.pb = pb
        d, N = pb.dim, pb.ncell
        H = assemble(pb, shift).tocsr()
        self.nu = d * N
        act = active_mask(pb)
        self.u_act = np.flatnonzero(act[: self.nu])
        Hu = H[self.u_act]
        Huu = Hu[:, self.u_act]
        self.A_up = Hu[:, self.nu:].tocsr()
        self.A_pu = H[self.nu:][:, self.u_act].tocsr()
        Cpp = H[self.nu:, self.nu:].tocsr()
        offdiag = Cpp - sp.diags(Cpp.diagonal())
        if offdiag.count_nonzero():
            raise ValueError("p-p block is not diagonal")
        self.cinv = 1.0 / Cpp.diagonal()
        self.S = _eliminate(Huu, self.A_up, self.cinv, self.A_pu)
        self.S.sort_indices()
        self.N = N

    def reduce(self, b):
        """Schur right-hand side f_u - A_up C^-1 f_p of a full right-hand side b."""
        b = np.asarray(b, dtype=np.complex128).ravel()
        return b[self.u_act] - self.A_up @ (self.cinv * b[self.nu:])

    def recover(self, u, b):
        """Full solution vector (u, p) from the Schur solution u and the full right-hand side b."""
        b = np.asarray(b, dtype=np.complex128).ravel()
        x = np.zeros(b.size, dtype=np.complex128)
        x[self.u_act] = u
        x[self.nu:] = self.cinv * (b[self.nu:] - self.A_pu @ u)
        return x


# ---------------------------------------------------------------- sub-regions
def reach_offsets(dim: int, comp: int):
    """(low, high) dilation per axis (x1 first) of a box's reach for component `comp`."""
    low = tuple(1 if a == comp else 2 for a in range(dim))
    return low, (1,) * dim


class Partition:
    """Rows and reach of each sub-region, as indices into a SchurSystem's unknowns."""

    def __init__(self, part_ptr, part_rows, reach_ptr, reach_cols, box, coloured):
        self.part_ptr = np.ascontiguousarray(part_ptr, dtype=np.int32)
        self.part_rows = np.ascontiguousarray(part_rows, dtype=np.int32)
        self.reach_ptr = np.ascontiguousarray(reach_ptr, dtype=np.int32)
        self.reach_cols = np.ascontiguousarray(reach_cols, dtype=np.int32)
        self.box = box
        self.coloured = coloured

    @property
    def nparts(self) -> int:
        return self.part_ptr.size - 1


def _box_ranges(n, box):
    return [(s, min(s + box, n)) for s in range(0, n, box)]


def box_partition(sys: SchurSystem, box, coloured: bool = False) -> Partition:
    """Sub-regions of `box` cells per axis (an int or one value per axis), see the module text."""
    pb = sys.pb
    d, n = pb.dim, pb.n
    box = (int(box),) * d if np.ndim(box) == 0 else tuple(int(v) for v in box)
    # full DOF index -> Schur unknown index (-1: inactive)
    sidx = -np.ones(sys.nu, dtype=np.int64)
    sidx[sys.u_act] = np.arange(sys.u_act.size)
    comp_idx = sidx.reshape((d,) + tuple(n[::-1]))
    ranges = [_box_ranges(n[a], box[a]) for a in range(d)]
    shape = tuple(len(r) for r in ranges)  # boxes per axis, x1 first
    boxes = []
    for flat in range(int(np.prod(shape))):
        bi, rem = [], flat
        for a in range(d):
            bi.append(rem % shape[a])
            rem //= shape[a]
        boxes.append(tuple(bi))

    def block(c, lo, hi):
        sl = tuple(slice(max(lo[a], 0), min(hi[a], n[a])) for a in reversed(range(d)))
        v = comp_idx[(c,) + sl].ravel()
        return v[v >= 0]

    rows_of, reach_of = [], []
    for bi in boxes:
        lo = [ranges[a][bi[a]][0] for a in range(d)]
        hi = [ranges[a][bi[a]][1] for a in range(d)]
        rows_of.append(np.concatenate([block(c, lo, hi) for c in range(d)]))
        reach = []
        for c in range(d):
            dl, dh = reach_offsets(d, c)
            reach.append(block(c, [lo[a] - dl[a] for a in range(d)], [hi[a] + dh[a] for a in range(d)]))
        reach_of.append(np.concatenate(reach))
    if coloured:
        colour = [sum((bi[a] % 2) << a for a in range(d)) for bi in boxes]
        order = sorted(range(len(boxes)), key=lambda k: (colour[k], k))
        rows = np.concatenate([rows_of[k] for k in order])
        allc = np.arange(sys.S.shape[1])
        return Partition([0, rows.size], rows, [0, allc.size], allc, box, True)
    part_ptr = np.concatenate([[0], np.cumsum([r.size for r in rows_of])])
    reach_ptr = np.concatenate([[0], np.cumsum([r.size for r in reach_of])])
    return Partition(part_ptr, np.concatenate(rows_of), reach_ptr, np.concatenate(reach_of), box, False)


def row_partition(nrows: int, ncols: int, parts) -> Partition:
    """A partition given directly as lists of rows (each reaching every unknown); for tests."""
    rows = np.concatenate([np.asarray(p, dtype=np.int64) for p in parts]) if parts else np.zeros(0, np.int64)
    ptr = np.concatenate([[0], np.cumsum([len(p) for p in parts])])
    allc = np.arange(ncols)
    return Partition(ptr, rows, np.arange(len(parts) + 1) * ncols, np.tile(allc, len(parts)), None, False)


# ---------------------------------------------------------------- the Kaczmarz step (C)
_LIB = None
_STEP = None  # another build of the step (tests plant mistakes in a copy of its source)


def load_step(so: str, src: str):
    """Compiles `src` (the step's C source) to `so` when it is missing or older, and loads it."""
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", so, src], check=True)
    lib = ctypes.CDLL(so)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.carp_step.argtypes = [ctypes.c_int, ip, ip, dp, dp, dp, ctypes.c_int, ip, ip, ip, ip, ctypes.c_double,
                              dp, dp, ip, ip]
    lib.carp_step.restype = ctypes.c_int
    return lib


def _lib():
    """The compiled step (oracle/kaczmarz.c), built here on first use."""
    global _LIB
    if _LIB is None:
        here = os.path.dirname(os.path.abspath(__file__))
        _LIB = load_step(os.path.join(here, "_kaczmarz.so"), os.path.join(here, "kaczmarz.c"))
    return _LIB


def kaczmarz_steps(S, part: Partition, rhs, x, steps: int, w: float):
    """`steps` parallel hybrid Kaczmarz steps for S x = rhs starting from x (returns a new x)."""
    lib = _lib() if _STEP is None else _STEP
    S = S.tocsr()
    n = S.shape[1]
    rp = np.ascontiguousarray(S.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(S.indices, dtype=np.int32)
    v = np.ascontiguousarray(S.data, dtype=np.complex128)
    bb = np.ascontiguousarray(rhs, dtype=np.complex128)
    xx = np.array(x, dtype=np.complex128, copy=True)
    work = np.zeros(n, dtype=np.complex128)
    acc = np.zeros(n, dtype=np.complex128)
    cnt = np.zeros(n, dtype=np.int32)
    mark = np.zeros(n, dtype=np.int32)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    for _ in range(steps):
        rc = lib.carp_step(int(n), rp.ctypes.data_as(ip), ci.ctypes.data_as(ip), v.ctypes.data_as(dp),
                           bb.ctypes.data_as(dp), xx.ctypes.data_as(dp), int(part.nparts),
                           part.part_ptr.ctypes.data_as(ip), part.part_rows.ctypes.data_as(ip),
                           part.reach_ptr.ctypes.data_as(ip), part.reach_cols.ctypes.data_as(ip), float(w),
                           work.ctypes.data_as(dp), acc.ctypes.data_as(dp), cnt.ctypes.data_as(ip),
                           mark.ctypes.data_as(ip))
        if rc != 0:
            raise ValueError("a row touches an unknown outside its sub-region's reach")
    return xx


# ---------------------------------------------------------------- the hybrid solve
def hybrid_solve(sys: SchurSystem, part: Partition, b, tol: float = 0.1, restart: int = 5,
                 kaczmarz_steps_per_apply: int = 10, damping: float = 0.8, max_kaczmarz: int = 250,
                 history=None):
    """Coarsest solve of H_s x = b (full vectors): FGMRES(restart) on the Schur system from a zero
    guess, each preconditioner application `kaczmarz_steps_per_apply` Kaczmarz steps from zero,
    until the Schur residual drops by `tol` or `max_kaczmarz` steps are spent.
    Returns (x, FGMRES iterations, relative Schur residual)."""
    f = sys.reduce(b)
    S = sys.S
    M = lambda v: kaczmarz_steps(S, part, v, np.zeros_like(v), kaczmarz_steps_per_apply, damping)
    max_iter = max(1, max_kaczmarz // kaczmarz_steps_per_apply)
    u, its, rel = fgmres(lambda v: S @ v, M, f, tol=tol, max_iter=max_iter, restart=restart, history=history)
    return sys.recover(u, b), its, rel
