"""Restriction and prolongation (oracle; test infrastructure only).

Section 2.3, Eq. (2.11) pIntergrid and Eq. (2.12) u2Intergrid, with
P = blockDiag(P_u1, .., P_p) and R likewise (Eq. 2.13):

* pressure: R_p averages the 2^d child cells; P_p is (bi/tri)linear interpolation with the
  transposed stencil [1 3 3 1]/4 along every axis;
* u_d: along its own (face-normal) axis, full weighting [1 2 1]/4 for R and linear
  interpolation [1 2 1]/2 (transposed) for P; along every other axis the same factors as
  the pressure ([1 1]/2 for R, [1 3 3 1]/4 for P). In 2D this is exactly the printed
  (1/8)[1 . 1; 2 * 2; 1 . 1] and (1/8)]1 3 . 3 1; 2 6 * 6 2; 1 3 . 3 1[. The 3D operators are
  the same tensor products (the paper calls the 3D extension straightforward).

Both operators are assembled as Kronecker products of one-dimensional factors; DOFs
outside the domain count as zero and boundary faces (not unknowns) are masked.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .discretization import Problem, active_mask, _kron_axes


def _r_face(nf, per):
    """coarse face K <- fine faces 2K-1, 2K, 2K+1 with weights [1 2 1]/4."""
    nc = nf // 2
    rows, cols, vals = [], [], []
    for K in range(nc):
        for off, w in ((-1, 0.25), (0, 0.5), (1, 0.25)):
            f = 2 * K + off
            if 0 <= f < nf:
                rows.append(K); cols.append(f); vals.append(w)
            elif per:
                rows.append(K); cols.append(f % nf); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, nf))


def _r_cell(nf, per):
    """coarse cell K <- fine cells 2K, 2K+1 with weights [1 1]/2."""
    nc = nf // 2
    rows = np.repeat(np.arange(nc), 2)
    cols = np.stack([2 * np.arange(nc), 2 * np.arange(nc) + 1], axis=1).ravel()
    return sp.csr_matrix((np.full(2 * nc, 0.5), (rows, cols)), shape=(nc, nf))


def _p_face(nf, per):
    """fine face 2K <- coarse K; fine face 2K+1 <- (coarse K + coarse K+1)/2 (transposed [1 2 1]/2)."""
    nc = nf // 2
    rows, cols, vals = [], [], []
    for K in range(nc):
        for off, w in ((-1, 0.5), (0, 1.0), (1, 0.5)):
            f = 2 * K + off
            if 0 <= f < nf:
                rows.append(f); cols.append(K); vals.append(w)
            elif per:
                rows.append(f % nf); cols.append(K); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def _p_cell(nf, per):
    """transposed [1 3 3 1]/4: coarse cell K feeds fine cells 2K-1, 2K, 2K+1, 2K+2."""
    nc = nf // 2
    rows, cols, vals = [], [], []
    for K in range(nc):
        for off, w in ((-1, 0.25), (0, 0.75), (1, 0.75), (2, 0.25)):
            f = 2 * K + off
            if 0 <= f < nf:
                rows.append(f); cols.append(K); vals.append(w)
            elif per:
                rows.append(f % nf); cols.append(K); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def _component_ops(pb: Problem, comp, face_fn, cell_fn):
    ops = [face_fn(pb.n[a], pb.periodic) if a == comp else cell_fn(pb.n[a], pb.periodic)
           for a in range(pb.dim)]
    return _kron_axes(ops)


def restriction(fine: Problem, coarse: Problem):
    """R = blockDiag(R_u1, .., R_p): fine DOF vector -> coarse DOF vector."""
    d = fine.dim
    blocks = [_component_ops(fine, c, _r_face, _r_cell) for c in range(d)]
    blocks.append(_component_ops(fine, -1, _r_face, _r_cell))
    R = sp.block_diag(blocks, format="csr")
    R = sp.diags(active_mask(coarse).astype(float)) @ R @ sp.diags(active_mask(fine).astype(float))
    return sp.csr_matrix(R)


def prolongation(fine: Problem, coarse: Problem):
    """P = blockDiag(P_u1, .., P_p): coarse DOF vector -> fine DOF vector."""
    d = fine.dim
    blocks = [_component_ops(fine, c, _p_face, _p_cell) for c in range(d)]
    blocks.append(_component_ops(fine, -1, _p_face, _p_cell))
    P = sp.block_diag(blocks, format="csr")
    P = sp.diags(active_mask(fine).astype(float)) @ P @ sp.diags(active_mask(coarse).astype(float))
    return sp.csr_matrix(P)
