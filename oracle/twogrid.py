"""Two-grid convergence factor in practice, and smoothing analysis (oracle; test infrastructure
only).

Section 4.3, Eq. convFactor and Table 1: the two-grid cycle of Eq. 2G for the shifted operator
(one pre- and one post-smoothing step, exact coarse solve of the re-discretised coarse operator)
is iterated on the error-residual equation (zero right-hand side, random start); after a warm-up
of 5 cycles the residual r_0 is recorded, and c_f = (||r_k|| / ||r_0||)^(1/k) for the first k
with ||r_k|| / ||r_0|| < 1e-9 (the paper's "r_k < 1e-9", read as relative).

The paper's setting: constant lambda = 500, mu = rho = 1, h = 1/1024, omega = pi / (5h), pi / (4h),
pi / (3.3h) with shifts 0.15, 0.2, 0.3, economic Vanka in lexicographic order, w = 0.65 (beta =
2/3) or 0.75 (beta = 1). Here the grid is periodic (no boundary: the setting local Fourier
analysis describes) and smaller; the factor barely depends on its size (0.229, 0.235, 0.237 for
n = 32, 64, 128 in the first case).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .discretization import Problem, assemble, active_mask, coarsen
from .transfer import restriction, prolongation
from .smoother import cell_dofs, cell_blocks, lexicographic_sweep, red_black_sweep, cell_colour


def two_grid_factor(n: int, beta: float, omega_h: float, alpha: float, w: float, lam: float = 500.0,
                    mu: float = 1.0, rho: float = 1.0, gamma: float = 0.01, smoother: str = "economic",
                    order: str = "lex", warmup: int = 5, drop: float = 1e-9, max_cycles: int = 300, seed: int = 0):
    """c_f of the two-grid cycle on an n x n periodic grid with h = 1/n (Eq. convFactor). gamma:
    the physical attenuation, 0.01 as in the paper's experiments (Sec. 5), added to the shift."""
    h = 1.0 / n
    shape = (n, n)
    pb = Problem((n, n), h, omega_h / h, gamma, beta, np.full(shape, lam), np.full(shape, mu), np.full(shape, rho),
                 abl_length=0.0, periodic=True)
    pc = coarsen(pb)
    H = assemble(pb, alpha).tocsr()
    Hc = assemble(pc, alpha).tocsc()
    R, P = restriction(pb, pc), prolongation(pb, pc)
    lu = spla.splu(Hc)
    idx = cell_dofs(pb)
    V = cell_blocks(H, idx, economic=smoother == "economic")
    Vinv = np.linalg.inv(V)
    col = cell_colour(pb)
    zero = np.zeros(H.shape[0], dtype=np.complex128)

    def smooth(x):
        if order == "lex":
            return lexicographic_sweep(H, Vinv, idx, zero, x, w)
        return red_black_sweep(H, V, idx, col, zero, x, w)

    def cycle(x):
        x = smooth(x)
        x = x + P @ lu.solve(R @ (-(H @ x)))
        return smooth(x)

    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])) * active_mask(pb)
    for _ in range(warmup):
        x = cycle(x)
    r0 = np.linalg.norm(H @ x)
    for k in range(1, max_cycles + 1):
        x = cycle(x)
        ratio = np.linalg.norm(H @ x) / r0
        if ratio < drop:
            return ratio ** (1.0 / k), k
    return ratio ** (1.0 / max_cycles), max_cycles


def smoothing_factor(n: int, beta: float, omega_h: float, alpha: float, w: float, nu: int = 1,
                     lam: float = 500.0, mu: float = 1.0, rho: float = 1.0, gamma: float = 0.01,
                     smoother: str = "economic", order: str = "lex", cycles: int = 60, seed: int = 0):
    """Smoothing analysis (Section 4.1, Definition 4.1), done numerically: the two-grid cycle
    with an IDEAL coarse-grid correction -- the projection Q that removes the low-frequency
    Fourier components (theta in [-pi/2, pi/2)^2) of every variable -- on an n x n periodic grid.
    Its asymptotic factor per cycle is mu_loc^nu (the relation the paper states for an ideal
    correction); nu = 1 applies Q S, nu = 2 applies S Q S (one pre- and one post-smoothing
    step). Computed by power iteration; returns mu_loc^nu."""
    h = 1.0 / n
    shape = (n, n)
    pb = Problem((n, n), h, omega_h / h, gamma, beta, np.full(shape, lam), np.full(shape, mu), np.full(shape, rho),
                 abl_length=0.0, periodic=True)
    H = assemble(pb, alpha).tocsr()
    idx = cell_dofs(pb)
    V = cell_blocks(H, idx, economic=smoother == "economic")
    Vinv = np.linalg.inv(V)
    col = cell_colour(pb)
    zero = np.zeros(H.shape[0], dtype=np.complex128)
    N = n * n
    k = np.fft.fftfreq(n) * 2.0 * np.pi
    low = np.abs(k) < np.pi / 2 - 1e-12
    low2 = low[:, None] & low[None, :]

    def S(x):
        if order == "lex":
            return lexicographic_sweep(H, Vinv, idx, zero, x, w)
        return red_black_sweep(H, V, idx, col, zero, x, w)

    def Q(x):
        out = x.copy()
        for c in range(3):
            f = np.fft.fft2(x[c * N:(c + 1) * N].reshape(n, n))
            f[low2] = 0.0
            out[c * N:(c + 1) * N] = np.fft.ifft2(f).ravel()
        return out

    rng = np.random.default_rng(seed)
    x = rng.standard_normal(3 * N) + 1j * rng.standard_normal(3 * N)
    fac = 0.0
    for _ in range(cycles):
        y = Q(S(x)) if nu == 1 else S(Q(S(x)))
        fac = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    return fac

