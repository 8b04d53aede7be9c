"""Vanka box smoother, red-black order (oracle; test infrastructure only).

Section 2.3 (last paragraph) and Section 3.2: a whole cell is relaxed at once by
inverting the (2d+1)x(2d+1) submatrix of the operator that couples the cell's
2d faces and its pressure ("full Vanka"), with a damping factor w. Red-black
order (Section 3.2): cells are coloured by the parity of the sum of their
indices; colour 0 is relaxed first, then colour 1.

Reading of the red-black step (the paper does not spell it out): within one
colour the cells are relaxed simultaneously (Jacobi within a colour) -- every
cell of the colour computes its residual from the state before the half-sweep
and the damped corrections are then added. Every face belongs to exactly one
cell of each colour, so the corrections never overlap. Faces that are not
unknowns (boundary faces, faces outside the domain) are left out of the local
system: their rows and columns become identity rows with a zero residual.

The local systems are extracted from the assembled sparse operator and solved
with a dense LU (numpy.linalg.solve); nothing exploits their block structure.
"""
from __future__ import annotations

import numpy as np

from .discretization import Problem, active_mask


def cell_dofs(pb: Problem):
    """(ncell, 2d+1) global DOF indices of each cell, in the order
    (u_1 low, u_1 high, .., u_d low, u_d high, p); -1 where the DOF is not an unknown."""
    d, N = pb.dim, pb.ncell
    grids = np.meshgrid(*[np.arange(c) for c in pb.n[::-1]], indexing="ij")
    k = [grids[d - 1 - a].ravel() for a in range(d)]  # k[a] = index along axis a
    strides = [int(np.prod(pb.n[:a])) for a in range(d)]
    flat = sum(k[a] * strides[a] for a in range(d))
    act = active_mask(pb)
    cols = []
    for c in range(d):
        low = c * N + flat
        hi_k = k[c] + 1
        if pb.periodic:
            hi_k = hi_k % pb.n[c]
            high = c * N + flat + (hi_k - k[c]) * strides[c]
        else:
            high = np.where(hi_k < pb.n[c], c * N + flat + strides[c], -1)
        low = np.where(act[np.maximum(low, 0)], low, -1)
        high = np.where((high >= 0) & act[np.maximum(high, 0)], high, -1)
        cols += [low, high]
    cols.append(d * N + flat)
    return np.stack(cols, axis=1)


def cell_colour(pb: Problem):
    d = pb.dim
    grids = np.meshgrid(*[np.arange(c) for c in pb.n[::-1]], indexing="ij")
    return (sum(g.ravel() for g in grids) % 2).astype(np.int64)


def cell_blocks(H, idx, economic=False):
    """(ncell, k, k) local matrices V_cell[a, b] = H[idx[a], idx[b]]; identity where excluded.
    economic: the displacement part (the first k-1 rows and columns) is replaced by its diagonal
    ("economic Vanka", Section 2.3); the couplings to the pressure and its diagonal are kept."""
    ncell, k = idx.shape
    V = np.zeros((ncell, k, k), dtype=np.complex128)
    for a in range(k):
        for b in range(k):
            ra, cb = idx[:, a], idx[:, b]
            ok = (ra >= 0) & (cb >= 0)
            if np.any(ok):
                V[ok, a, b] = np.asarray(H[ra[ok], cb[ok]]).ravel()
        V[idx[:, a] < 0, a, :] = 0.0
        V[:, :, a][idx[:, a] < 0] = 0.0
        V[idx[:, a] < 0, a, a] = 1.0
    if economic:
        for a in range(k - 1):
            for b in range(k - 1):
                if a != b:
                    V[:, a, b] = 0.0
    return V


def _local_residual(H, b, x, idx):
    r = b - H @ x
    rl = np.where(idx >= 0, r[np.maximum(idx, 0)], 0.0)
    return rl


def vanka_cell_update(H, V, idx, cell, b, x, w):
    """Relax one cell: x[cell DOFs] += w * V_cell^{-1} r_cell. Returns the new vector."""
    x = x.copy()
    r = b - H @ x
    ii = idx[cell]
    rl = np.where(ii >= 0, r[np.maximum(ii, 0)], 0.0)
    delta = w * np.linalg.solve(V[cell], rl)
    ok = ii >= 0
    x[ii[ok]] += delta[ok]
    return x


def half_sweep(H, V, idx, colour_of_cell, colour, b, x, w):
    """Relax every cell of one colour simultaneously from the current state."""
    sel = np.nonzero(colour_of_cell == colour)[0]
    ii = idx[sel]
    r = b - H @ x
    rl = np.where(ii >= 0, r[np.maximum(ii, 0)], 0.0)
    delta = w * np.linalg.solve(V[sel], rl[..., None])[..., 0]
    x = x.copy()
    ok = ii >= 0
    # faces of distinct same-colour cells are distinct, so plain assignment-add is exact
    np.add.at(x, ii[ok], delta[ok])
    return x


def red_black_sweep(H, V, idx, colour_of_cell, b, x, w):
    """One full smoothing step: colour 0, then colour 1."""
    x = half_sweep(H, V, idx, colour_of_cell, 0, b, x, w)
    x = half_sweep(H, V, idx, colour_of_cell, 1, b, x, w)
    return x


def _lex_lib():
    """The compiled lexicographic sweep (oracle/lexvanka.c), built here on first use."""
    import ctypes
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    so = os.path.join(here, "_lexvanka.so")
    src = os.path.join(here, "lexvanka.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", so, src], check=True)
    lib = ctypes.CDLL(so)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.lex_block_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp, ip, ip, dp, dp, dp, ctypes.c_double]
    lib.lex_block_sweep.restype = None
    return lib


def lexicographic_sweep(H, Vinv, idx, b, x, w):
    """One lexicographic Vanka sweep (Section 3.2, the ordering used for the paper's LFA and
    Table 1): cells in order, x1 fastest, each relaxed with the residual of the current iterate
    (Gauss-Seidel over cells). Vinv: (ncell, k, k) inverses of the local blocks. Returns new x."""
    import ctypes
    lib = _lex_lib()
    Hc = H.tocsr()
    indptr = np.ascontiguousarray(Hc.indptr, dtype=np.int32)
    indices = np.ascontiguousarray(Hc.indices, dtype=np.int32)
    data = np.ascontiguousarray(Hc.data, dtype=np.complex128)
    dofs = np.ascontiguousarray(idx, dtype=np.int32)
    vinv = np.ascontiguousarray(Vinv, dtype=np.complex128)
    bb = np.ascontiguousarray(b, dtype=np.complex128)
    xx = np.array(x, dtype=np.complex128, copy=True)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.lex_block_sweep(int(idx.shape[0]), int(idx.shape[1]), dofs.ctypes.data_as(ip), vinv.ctypes.data_as(dp),
                        indptr.ctypes.data_as(ip), indices.ctypes.data_as(ip), data.ctypes.data_as(dp),
                        bb.ctypes.data_as(dp), xx.ctypes.data_as(dp), float(w))
    return xx
