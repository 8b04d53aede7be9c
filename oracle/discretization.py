"""Assembled FP64 operator of the paper's discretisation (oracle; test infrastructure only).

Section 3.1, Eq. (3.10) mixed-discretized, read with the sign of the homogeneous
form Eq. (4.4) mixed-discretized-homogeneous (the u-p coupling is the standard
gradient +d/dx_d, which keeps the Schur complement consistent with Eq. 2.3):

    [ grad_h^T A_e(mu) grad_h^beta - M^beta A_f(rho) m   |   +grad_h        ] [u]   [q]
    [ (div)_h^beta                                       |  diag(1/(lam+mu))] [p] = [0]

* first derivatives, Eq. (3.4) dxdyStandard and Eq. (3.5) dxSpread: the standard one is
  (1/h)[-1 * 1]; the beta-spread one mixes it with the same difference smoothed by [1 2 1]/4
  across the other axis (2D) or by [1 2 1]/4 x [1 2 1]/4 across the two other axes (3D,
  Eq. dxSkew3D, with the 1/h of the 2D form kept);
* A_e(mu): mu averaged to where d_e u_d lives -- the cell centre for e = d, the mean of the 4
  surrounding cells (2D node / 3D edge) for e != d;
* A_f(rho): rho averaged to the faces (mean of the 2 adjacent cells);
* M^beta (Eq. 3.3 massHO, 3D Eq. massHO3D): beta*[1] + (1-beta)/(2d) * (sum of the 2d
  same-component neighbours), applied to m_f u_f with the per-face complex coefficient
  m_f = rho_f omega^2 (1 - i(gamma + gamma_ABL(x_f) + alpha_s));
* the shifted operator H_s adds alpha to the attenuation (Eq. 2.9 shift and the text after it).

Grid and storage. n = (n_1, .., n_d) cells, x_1 fastest. Every component is stored as an
array of shape n[::-1]; u_d[k] is the face normal to x_d on the LOW side of cell k, at
x_d = k_d h with the other coordinates at cell centres; p sits at cell centres. The DOF
vector is the concatenation (u_1, .., u_d, p).

Boundary (the paper is silent; reading): homogeneous Dirichlet with zero extension. The
faces u_d with k_d = 0 lie on the boundary: they are not unknowns (rows and columns of H
are zero there). Every DOF outside the domain is zero; material outside is clamped to the
nearest cell. `periodic=True` wraps every axis instead (every face is an unknown); it is
used for Fourier-symbol checks only.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    n: tuple                 # cells per axis, x1 first
    h: float                 # cell size on this level
    omega: float
    gamma: float             # physical attenuation of the unshifted operator
    beta: float
    lam: np.ndarray          # cell-centred, shape n[::-1]
    mu: np.ndarray
    rho: np.ndarray
    abl_length: float = 0.0  # physical thickness of the absorbing layer (0: none)
    abl_gamma_max: float = 0.0
    domain: tuple = None     # physical domain length per axis (defaults to n*h)
    periodic: bool = False
    origin: tuple = None     # cell offset of this grid inside a larger domain (windowed evaluation)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if self.domain is None:
            self.domain = tuple(v * self.h for v in self.n)
        if self.origin is None:
            self.origin = (0,) * len(self.n)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))


def dof_shape(pb: Problem):
    return (pb.dim + 1,) + tuple(pb.n[::-1])


# ---------------------------------------------------------------- 1D factors
def _d_face_to_cell(n, h, per):
    """(v[k+1] - v[k]) / h from faces 0..n-1 (face n is zero / wraps) to cells 0..n-1."""
    rows, cols, vals = [], [], []
    for k in range(n):
        rows.append(k); cols.append(k); vals.append(-1.0 / h)
        if k + 1 < n:
            rows.append(k); cols.append(k + 1); vals.append(1.0 / h)
        elif per:
            rows.append(k); cols.append(0); vals.append(1.0 / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def _d_cell_to_node(n, h, per):
    """(v[k] - v[k-1]) / h from cells to lattice points k (n+1 of them, zero ghosts; n if periodic)."""
    m = n if per else n + 1
    rows, cols, vals = [], [], []
    for k in range(m):
        if k < n:
            rows.append(k); cols.append(k); vals.append(1.0 / h)
        if k >= 1:
            rows.append(k); cols.append(k - 1); vals.append(-1.0 / h)
        elif per:
            rows.append(k); cols.append(n - 1); vals.append(-1.0 / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, n))


def _d_cell_to_face(n, h, per):
    """(p[k] - p[k-1]) / h from cells to faces 0..n-1 (the gradient of p at the faces)."""
    return _d_cell_to_node(n, h, per)[:n, :] if not per else _d_cell_to_node(n, h, per)


def _smooth121(n, per):
    """[1 2 1]/4 along one axis, zero extension (or periodic wrap)."""
    main = np.full(n, 0.5)
    off = np.full(n - 1, 0.25)
    m = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="lil")
    if per and n > 1:
        m[0, n - 1] += 0.25
        m[n - 1, 0] += 0.25
    return m.tocsr()


def _neighbours(n, per):
    """Sum of the two neighbours along one axis."""
    off = np.ones(n - 1)
    m = sp.diags([off, off], [-1, 1], shape=(n, n), format="lil")
    if per and n > 1:
        m[0, n - 1] += 1.0
        m[n - 1, 0] += 1.0
    return m.tocsr()


def _kron_axes(ops):
    """Kronecker product of per-axis operators, ops[0] acting on x1 (the fastest index)."""
    m = ops[0]
    for a in range(1, len(ops)):
        m = sp.kron(ops[a], m, format="csr")
    return sp.csr_matrix(m)


# ---------------------------------------------------------------- coefficients
def _clamp_idx(k, n, per):
    return np.mod(k, n) if per else np.clip(k, 0, n - 1)


def _avg_cells(field, pb: Problem, lattice_axes, counts):
    """Average the cell field over the 2^|lattice_axes| cells around lattice points.

    `counts[a]` is the number of points along axis a. Along a lattice axis, point k sits at
    x_a = k h, between cells k-1 and k; along other axes point k is cell k.
    Returns an array of shape counts[::-1]."""
    d = pb.dim
    grids = np.meshgrid(*[np.arange(c) for c in counts[::-1]], indexing="ij")  # [z..x]
    idx = [grids[d - 1 - a] for a in range(d)]  # idx[a] = index along axis a
    total = np.zeros(tuple(counts[::-1]))
    shifts = [(0, -1) if a in lattice_axes else (0,) for a in range(d)]
    nterm = 0
    for combo in np.array(np.meshgrid(*shifts, indexing="ij")).reshape(d, -1).T:
        sel = tuple(_clamp_idx(idx[a] + combo[a], pb.n[a], pb.periodic) for a in range(d))
        total += field[sel[::-1]]
        nterm += 1
    return total / nterm


def _positions(pb: Problem, comp):
    """Physical coordinates (per axis) of the DOFs of component `comp` (d = pressure)."""
    d = pb.dim
    grids = np.meshgrid(*[np.arange(c) for c in pb.n[::-1]], indexing="ij")
    pos = []
    for a in range(d):
        k = grids[d - 1 - a].astype(np.float64) + pb.origin[a]
        pos.append(k * pb.h if a == comp else (k + 0.5) * pb.h)
    return pos


def gamma_abl(pb: Problem, comp):
    """Absorbing-layer attenuation at the DOFs of component `comp` (reading; the paper only
    states a 20-cell layer): gamma_max * sum_a (delta_a / L)^2, delta_a the distance into
    the layer along axis a, L its physical thickness."""
    shape = tuple(pb.n[::-1])
    if pb.abl_length <= 0.0 or pb.abl_gamma_max == 0.0:
        return np.zeros(shape)
    g = np.zeros(shape)
    L = pb.abl_length
    for a, x in enumerate(_positions(pb, comp)):
        X = pb.domain[a]
        delta = np.maximum(0.0, L - x) + np.maximum(0.0, x - (X - L))
        g += (delta / L) ** 2
    return pb.abl_gamma_max * g


def active_mask(pb: Problem):
    """Boolean DOF mask: False on the boundary faces (u_d with k_d = 0) unless periodic."""
    d = pb.dim
    m = np.ones(dof_shape(pb), dtype=bool)
    if not pb.periodic:
        for c in range(d):
            sl = [c] + [slice(None)] * d
            sl[1 + (d - 1 - c)] = 0
            m[tuple(sl)] = False
    return m.ravel()


# ---------------------------------------------------------------- assembly
def _derivative(pb: Problem, comp, e, spread):
    """Standard (spread=False) or beta-spread derivative along axis e of u_comp.

    Along e: faces->cells if e == comp else cells->lattice points; the beta-spread version
    adds (1-beta) times the same difference smoothed by [1 2 1]/4 along every other axis
    (Eq. 3.5 in 2D, Eq. dxSkew3D in 3D)."""
    d, per, h = pb.dim, pb.periodic, pb.h
    D = _d_face_to_cell(pb.n[e], h, per) if e == comp else _d_cell_to_node(pb.n[e], h, per)
    ops = [D if a == e else sp.identity(pb.n[a], format="csr") for a in range(d)]
    std = _kron_axes(ops)
    if not spread:
        return std
    ops_s = [D if a == e else _smooth121(pb.n[a], per) for a in range(d)]
    return pb.beta * std + (1.0 - pb.beta) * _kron_axes(ops_s)


def _mu_at_derivative(pb: Problem, comp, e):
    """A_e(mu): mu at the points where d_e u_comp lives."""
    if e == comp:
        return pb.mu.ravel()
    counts = list(pb.n)
    if not pb.periodic:
        counts[e] = pb.n[e] + 1
    return _avg_cells(pb.mu, pb, (comp, e), counts).ravel()


def mass_coefficient(pb: Problem, comp, shift):
    """m_f = rho_f omega^2 (1 - i(gamma + gamma_ABL + shift)) at the faces of u_comp."""
    rho_f = _avg_cells(pb.rho, pb, (comp,), list(pb.n))
    att = pb.gamma + shift + gamma_abl(pb, comp)
    return (rho_f * pb.omega ** 2 * (1.0 - 1j * att)).ravel()


def _mass_spread(pb: Problem):
    """M^beta / (omega^2 ...): beta I + (1-beta)/(2d) * (sum of the 2d neighbours)."""
    d = pb.dim
    N = pb.ncell
    acc = sp.csr_matrix((N, N))
    for a in range(d):
        ops = [_neighbours(pb.n[a], pb.periodic) if b == a else sp.identity(pb.n[b], format="csr")
               for b in range(d)]
        acc = acc + _kron_axes(ops)
    return pb.beta * sp.identity(N, format="csr") + (1.0 - pb.beta) / (2 * d) * acc


def _gradient_p(pb: Problem, comp):
    ops = [_d_cell_to_face(pb.n[a], pb.h, pb.periodic) if a == comp else sp.identity(pb.n[a], format="csr")
           for a in range(pb.dim)]
    return _kron_axes(ops)


def assemble(pb: Problem, shift: float = 0.0):
    """Sparse (d+1)N x (d+1)N matrix of H^beta (shift=0) or H^beta_s (shift=alpha)."""
    d = pb.dim
    Ms = _mass_spread(pb)
    blocks = [[None] * (d + 1) for _ in range(d + 1)]
    for c in range(d):
        lap = None
        for e in range(d):
            std = _derivative(pb, c, e, spread=False)
            spr = _derivative(pb, c, e, spread=True)
            term = std.T @ sp.diags(_mu_at_derivative(pb, c, e)) @ spr
            lap = term if lap is None else lap + term
        mass = Ms @ sp.diags(mass_coefficient(pb, c, shift))
        blocks[c][c] = (lap - mass).tocsr()
        blocks[c][d] = _gradient_p(pb, c)
        blocks[d][c] = _derivative(pb, c, c, spread=True)
    blocks[d][d] = sp.diags(1.0 / (pb.lam + pb.mu).ravel())
    H = sp.bmat(blocks, format="csr").astype(np.complex128)
    act = active_mask(pb).astype(np.float64)
    Pa = sp.diags(act)
    H = (Pa @ H @ Pa).tocsr()
    H.eliminate_zeros()
    return H


def apply(pb: Problem, x, shift: float = 0.0):
    """y = H x (or H_s x) for x of shape (d+1,) + n[::-1]."""
    H = assemble(pb, shift)
    return (H @ np.asarray(x, dtype=np.complex128).ravel()).reshape(dof_shape(pb))


def window(pb: Problem, lo, hi) -> Problem:
    """The sub-grid of cells lo[a] <= k_a < hi[a] placed at its position in `pb`'s domain.

    Rows of the window's operator that are at least 3 cells away from every cut edge equal the
    rows of `pb`'s operator (the stencil reaches 2 cells); cut edges are treated as boundaries."""
    sl = tuple(slice(lo[a], hi[a]) for a in reversed(range(pb.dim)))
    n = tuple(hi[a] - lo[a] for a in range(pb.dim))
    org = tuple(pb.origin[a] + lo[a] for a in range(pb.dim))
    return replace(pb, n=n, lam=pb.lam[sl], mu=pb.mu[sl], rho=pb.rho[sl], domain=pb.domain, origin=org)


def coarsen(pb: Problem) -> Problem:
    """Re-discretisation problem on the 2h grid (Section 3.2): same omega, beta, gamma and
    absorbing layer (physical thickness); material = arithmetic mean of the 2^d children
    (reading; the paper does not say how coarse media are formed)."""
    d = pb.dim
    if any(v % 2 for v in pb.n):
        raise ValueError("grid not divisible by 2: %s" % (pb.n,))
    nc = tuple(v // 2 for v in pb.n)

    def avg(f):
        g = f
        for ax in range(d):  # array axes (z, y, x) order does not matter for a full mean
            sh = list(g.shape)
            sh[ax:ax + 1] = [sh[ax] // 2, 2]
            g = g.reshape(sh).mean(axis=ax + 1)
        return g

    org = tuple(o // 2 for o in pb.origin)
    return replace(pb, n=nc, h=2.0 * pb.h, lam=avg(pb.lam), mu=avg(pb.mu), rho=avg(pb.rho), origin=org)
