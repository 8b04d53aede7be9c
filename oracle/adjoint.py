"""Misfit gradient with respect to the material by the adjoint-state method (oracle; test
infrastructure only).

The paper's solver is the forward solver of frequency-domain elastic full-waveform inversion
(Section 1; its code is part of a package used for 3D elastic inversion, Section 5). Inversion
needs, besides the forward solves, the gradient of a data misfit with respect to the material
fields, which costs one more solve per source with the conjugate-transposed operator (the
adjoint-state method, e.g. Plessix 2006):

    u_s = H(m)^{-1} q_s                                (forward wavefield of source s)
    J(m) = 1/2 sum_s || S u_s - d_s ||^2                (S samples the receiver DOFs)
    a_s = H(m)^{-H} S^T (S u_s - d_s)                   (adjoint wavefield)
    dJ/dm_k = -Re sum_s a_s^H (dH/dm_k) u_s,   m in {lambda, mu, rho}, k a cell.

H is the unshifted operator of Eq. 3.10 (with the coupling sign of Eq. 4.4). It depends on the
cell fields only through
  * A_e(mu): mu at the points where each derivative d_e u_c lives (the cell mu for e = c, the
    mean of the 2 x 2 cells around the node / edge otherwise): linear in mu;
  * the face density rho_f (mean of the 2 adjacent cells) in the mass m_f = rho_f omega^2 (1 - i
    (gamma + gamma_ABL)): linear in rho;
  * diag(1/(lambda + mu)) in the continuity row.
The derivative is therefore exact and local: with the derivative matrices D (standard) and
D^beta (spread) of each term, its weight at a derivative point is (D conj(a_c)) (D^beta u_c),
mapped back to the cells by the transpose of the averaging; the mass weight is
(M^beta^T conj(a_c)) omega^2 (1 - i att) u_c at a face, mapped back by the transpose of the face
average; the continuity term gives -conj(a_p) u_p / (lambda + mu)^2 for lambda and for mu.

Solves are direct (sparse LU of the active part of the operator): the definition the iterative
GPU solves converge to.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import (Problem, assemble, active_mask, dof_shape, gamma_abl, _derivative, _mass_spread,
                             _clamp_idx)


def average_matrix(pb: Problem, lattice_axes, counts):
    """Sparse (prod(counts), ncell) matrix of the cell averaging around lattice points: along a
    lattice axis point k sits between cells k-1 and k, along the other axes point k is cell k;
    cells outside the grid are clamped to the nearest one (or wrap, if periodic)."""
    d = pb.dim
    grids = np.meshgrid(*[np.arange(c) for c in counts[::-1]], indexing="ij")
    idx = [grids[d - 1 - a].ravel() for a in range(d)]
    rows = np.arange(int(np.prod(counts)))
    shifts = [(0, -1) if a in lattice_axes else (0,) for a in range(d)]
    combos = np.array(np.meshgrid(*shifts, indexing="ij")).reshape(d, -1).T
    strides = [int(np.prod(pb.n[:a])) for a in range(d)]
    R, C = [], []
    for combo in combos:
        col = sum(_clamp_idx(idx[a] + combo[a], pb.n[a], pb.periodic) * strides[a] for a in range(d))
        R.append(rows)
        C.append(col)
    R, C = np.concatenate(R), np.concatenate(C)
    V = np.full(R.shape, 1.0 / len(combos))
    return sp.csr_matrix((V, (R, C)), shape=(int(np.prod(counts)), pb.ncell))


def _mu_points(pb: Problem, comp, e):
    counts = list(pb.n)
    if e != comp and not pb.periodic:
        counts[e] = pb.n[e] + 1
    return counts


def material_derivative(pb: Problem, u, a, shift: float = 0.0):
    """-Re a^H (dH_shift/dm_k) u for every cell k and m in (lam, mu, rho); u, a are DOF vectors.
    Returns a dict of cell arrays of shape n[::-1]."""
    d, N = pb.dim, pb.ncell
    act = active_mask(pb)
    u = np.asarray(u, dtype=np.complex128).ravel() * act
    ac = np.conj(np.asarray(a, dtype=np.complex128).ravel() * act)
    g_mu = np.zeros(N, dtype=np.complex128)
    g_rho = np.zeros(N, dtype=np.complex128)
    Ms = _mass_spread(pb)
    for c in range(d):
        uc, acc = u[c * N:(c + 1) * N], ac[c * N:(c + 1) * N]
        for e in range(d):
            w = (_derivative(pb, c, e, spread=False) @ acc) * (_derivative(pb, c, e, spread=True) @ uc)
            if e == c:
                g_mu += w
            else:
                g_mu += average_matrix(pb, (c, e), _mu_points(pb, c, e)).T @ w
        att = pb.gamma + shift + gamma_abl(pb, c).ravel()
        wm = (Ms.T @ acc) * (pb.omega ** 2 * (1.0 - 1j * att)) * uc
        g_rho -= average_matrix(pb, (c,), list(pb.n)).T @ wm
    s = 1.0 / (pb.lam + pb.mu).ravel()
    gp = -(ac[d * N:] * u[d * N:]) * s * s
    shape = tuple(pb.n[::-1])
    return {"lam": -np.real(gp).reshape(shape), "mu": -np.real(g_mu + gp).reshape(shape),
            "rho": -np.real(g_rho).reshape(shape)}


class DirectSolver:
    """Sparse LU of the active part of H (shift 0) and of its conjugate transpose."""

    def __init__(self, pb: Problem, shift: float = 0.0):
        self.pb = pb
        self.act = active_mask(pb)
        H = assemble(pb, shift).tocsr()
        Ha = H[self.act][:, self.act].tocsc()
        self.lu = spla.splu(Ha)
        self.luh = spla.splu(sp.csc_matrix(Ha.conj().T))

    def _run(self, lu, b):
        b = np.asarray(b, dtype=np.complex128).ravel()
        x = np.zeros_like(b)
        x[self.act] = lu.solve(b[self.act])
        return x

    def solve(self, b):
        return self._run(self.lu, b)

    def solve_adjoint(self, b):
        return self._run(self.luh, b)


def misfit_and_gradient(pb: Problem, sources, receivers, data):
    """J(m) and its gradient for sources q_s (DOF arrays), receiver DOF indices (flat) and data
    d_s (complex values at the receivers, one array per source)."""
    ds = DirectSolver(pb)
    J = 0.0
    grad = {k: np.zeros(tuple(pb.n[::-1])) for k in ("lam", "mu", "rho")}
    for q, dat in zip(sources, data):
        u = ds.solve(q)
        r = u[receivers] - dat
        J += 0.5 * float(np.vdot(r, r).real)
        rhs = np.zeros_like(u)
        np.add.at(rhs, receivers, r)
        a = ds.solve_adjoint(rhs)
        for k, v in material_derivative(pb, u, a).items():
            grad[k] += v
    return J, grad


def misfit(pb: Problem, sources, receivers, data):
    ds = DirectSolver(pb)
    J = 0.0
    for q, dat in zip(sources, data):
        r = ds.solve(q)[receivers] - dat
        J += 0.5 * float(np.vdot(r, r).real)
    return J


def synthetic_data(pb: Problem, sources, receivers):
    """Receiver values of the forward wavefields (the data of a 'true' medium)."""
    ds = DirectSolver(pb)
    return [ds.solve(q)[receivers] for q in sources]


def receiver_dofs(pb: Problem, comp, depth, positions):
    """Flat DOF indices of component `comp` at grid index `depth` along the last axis and the
    given positions on the other axes (x1 first)."""
    shape = dof_shape(pb)
    out = []
    for pos in positions:
        idx = tuple(pos) + (depth,)
        out.append(np.ravel_multi_index((comp,) + tuple(idx[::-1]), shape))
    return np.array(out, dtype=np.int64)
