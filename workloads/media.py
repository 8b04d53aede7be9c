"""Synthetic elastic media, frequencies and point sources.

Arrays are indexed [z, y, x] (3D) or [y, x] (2D): the first grid axis x1 is the
fastest-varying one. The depth axis is the last grid axis (x2 in 2D, x3 in 3D),
i.e. the slowest array index.

Velocity relations (Section 2.1): Vp = sqrt((lambda + 2 mu)/rho), Vs = sqrt(mu/rho).
Frequency rule (Section 5): omega chosen for G_s points per minimum shear
wavelength, omega = 2 pi min(Vs) / (G_s h).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One solve: medium, frequency, source, and the solver settings it is run with."""
    name: str
    n: tuple            # cells per axis, x1 first
    h: float
    lam: np.ndarray     # cell-centred, shape n[::-1]
    mu: np.ndarray
    rho: np.ndarray
    omega: float
    rhs: np.ndarray     # complex128, shape (dim+1,) + n[::-1]; (u_1..u_d, p) components
    levels: int
    alpha: float
    damping: object     # one value for every level, or one per level
    abl_cells: int
    gamma: float = 0.01
    beta: float = 2.0 / 3.0
    abl_gamma_max: float = 2.0
    nu_pre: int = 2
    nu_post: int = 2
    restart: int = 20
    tol: float = 1e-6
    coarse: str = "dense"          # "dense", "smooth" or "kaczmarz"
    coarse_sweeps: int = 0
    coarse_damping: float = 1.0
    cycle: str = "V"               # "V" or "W"
    alpha_coarsest: float = 0.0    # shift of the coarsest level (0: alpha)
    level_alpha: tuple = None      # shift per level, finest first (overrides alpha / alpha_coarsest)
    smoother: str = "full"         # "full" or "economic" Vanka
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return len(self.n)

    def level_alphas(self):
        """Shift per level: level_alpha if given (its last value repeated below its end), else
        alpha everywhere with alpha_coarsest (if set) on the coarsest level."""
        if self.level_alpha:
            la = list(self.level_alpha)
            return [la[min(l, len(la) - 1)] for l in range(self.levels)]
        a = [self.alpha] * self.levels
        if self.alpha_coarsest > 0:
            a[-1] = self.alpha_coarsest
        return a


def lame_from_velocity(vp: np.ndarray, vs: np.ndarray, rho: np.ndarray):
    """(lambda, mu) from Vp, Vs, rho via Vs^2 = mu/rho and Vp^2 = (lambda+2mu)/rho."""
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def omega_for_points_per_wavelength(vs_min: float, h: float, g_s: float = 10.0) -> float:
    return 2.0 * np.pi * vs_min / (g_s * h)


def random_field(shape, seed: int, sigma_cells: float) -> np.ndarray:
    """White noise smoothed by a Gaussian of std `sigma_cells` (periodic wrap)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    return gaussian_filter(noise, sigma=sigma_cells, mode="wrap")


def gaussian_random_velocity(shape, seed: int, sigma_cells: float = 32.0,
                             vmin: float = 1.5, vmax: float = 4.5) -> np.ndarray:
    """Smooth random Vp field mapped affinely so that its min/max are [vmin, vmax]."""
    f = random_field(shape, seed, sigma_cells)
    lo, hi = f.min(), f.max()
    return vmin + (vmax - vmin) * (f - lo) / (hi - lo)


def point_source(n, component: int, index) -> np.ndarray:
    """Unit point force on one DOF. `index` is the DOF's grid index, x1 first."""
    dim = len(n)
    q = np.zeros((dim + 1,) + tuple(n[::-1]), dtype=np.complex128)
    q[(component,) + tuple(index[::-1])] = 1.0
    return q


def config_c1_homogeneous(n: int = 128) -> Workload:
    """2D homogeneous lambda=2, mu=1, rho=1 (Vp=2, Vs=1), 10 points per shear wavelength,
    unit force in u1 at the grid centre, 4 levels (coarsest n/8 squared, direct), ABL 16."""
    shape = (n, n)
    lam = np.full(shape, 2.0)
    mu = np.ones(shape)
    rho = np.ones(shape)
    h = 1.0
    omega = omega_for_points_per_wavelength(1.0, h)
    rhs = point_source((n, n), 0, (n // 2, n // 2))
    return Workload("c1_homogeneous_2d_%d" % n, (n, n), h, lam, mu, rho, omega, rhs,
                    levels=4, alpha=0.4, damping=0.25, abl_cells=16, coarse="dense")


def config_c2_random2d(n: int = 2048, seed: int = 0, levels: int = 5, source_depth: int = 32) -> Workload:
    """2D smooth random medium: Vp in [1.5, 4.5] (Gaussian filter sigma 32 cells, correlation
    length ~64 cells), Vs = Vp/sqrt(3), rho = 0.31 Vp^0.25; 10 points per minimum shear
    wavelength; point force in the depth component u2 at (n/2, depth 32). Solver: W(1,1) on 5
    levels (the paper's 2D cycle), shift 0.5, shift 1.0 on the coarsest level (2 red-black
    sweeps), FGMRES(5).

    Damping per level (0.7, 0.4, 0.4, 0.3, then the coarsest level's own 0.8). Two-grid Fourier
    analysis of the red-black smoother with one pre- and one post-step (alpha = 0.5, lambda =
    mu) puts the best w at 0.7-0.8 for 10 points per wavelength (the finest level), 0.5-0.6 for 5
    and 0.4 for 2.5, and a uniform 0.2 is far from all of them. Measured on this medium (FGMRES(5)
    iterations, seconds): W(2,2) with 0.2 everywhere 232, 0.94; W(2,2) with 0.5 / 0.3 / 0.3 / 0.2
    211, 0.86; W(2,1) 221-226, 0.77-0.78; W(1,1) with 0.7 / 0.4 / 0.3 / 0.25 255, 0.74; W(1,1)
    with 0.7 / 0.4 / 0.4 / 0.3 230, 0.67, the fastest."""
    shape = (n, n)
    sigma = 32.0 * n / 2048.0 if n < 2048 else 32.0
    vp = gaussian_random_velocity(shape, seed, sigma_cells=sigma)
    vs = vp / np.sqrt(3.0)
    rho = 0.31 * vp ** 0.25
    lam, mu = lame_from_velocity(vp, vs, rho)
    h = 1.0
    omega = omega_for_points_per_wavelength(float(vs.min()), h)
    rhs = point_source((n, n), 1, (n // 2, min(source_depth, n - 1)))
    return Workload("c2_random_2d_%d" % n, (n, n), h, lam, mu, rho, omega, rhs,
                    levels=levels, alpha=0.5, damping=tuple(([0.7, 0.4, 0.4, 0.3] + [0.2] * levels)[:levels]),
                    abl_cells=20, coarse="smooth", coarse_sweeps=2, coarse_damping=0.8, cycle="W",
                    alpha_coarsest=1.0, restart=5, nu_pre=1, nu_post=1)


def config_c4_batch(count: int = 64, seed0: int = 1000, sizes=(256, 384, 512, 768, 1024),
                    abl_cells: int = 20) -> list:
    """Batch of independent 2D solves: instance i draws its square grid side uniformly from
    `sizes` and its medium from the 2D random-field generator with seed seed0 + i (Gaussian
    filter sigma 32 cells, Vp in [1.5, 4.5], Vs = Vp/sqrt(3), rho = 0.31 Vp^0.25), omega for 10
    points per minimum shear wavelength, and 1-4 unit point forces in the depth component at
    random positions outside the absorbing layer (extra["sources"], the first also in rhs).
    Solver: W(2,2) on 5 levels, whose spacings h_l = 2^l h match the 2048^2 configuration's
    (coarsest n/16, 16^2 to 64^2), damping 0.5 / 0.3 / 0.3 / 0.2 by level, shift 0.5 (1.0 and 2
    red-black sweeps on the coarsest level), FGMRES(5)."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        n = int(rng.choice(sizes))
        shape = (n, n)
        vp = gaussian_random_velocity(shape, seed0 + k, sigma_cells=32.0)
        vs = vp / np.sqrt(3.0)
        rho = 0.31 * vp ** 0.25
        lam, mu = lame_from_velocity(vp, vs, rho)
        h = 1.0
        omega = omega_for_points_per_wavelength(float(vs.min()), h)
        nsrc = int(rng.integers(1, 5))
        lo, hi = abl_cells + 2, n - abl_cells - 2
        sources = [point_source((n, n), 1, (int(rng.integers(lo, hi)), int(rng.integers(lo, hi))))
                   for _ in range(nsrc)]
        w = Workload("c4_%02d_%d" % (k, n), (n, n), h, lam, mu, rho, omega, sources[0],
                     levels=5, alpha=0.5, damping=(0.5, 0.3, 0.3, 0.2, 0.2), abl_cells=abl_cells, coarse="smooth",
                     coarse_sweeps=2,
                     coarse_damping=0.8, cycle="W", alpha_coarsest=1.0, restart=5)
        w.extra["sources"] = sources
        out.append(w)
    return out


def config_c3_layered3d(n: int = 256, source=(128, 128, 24), levels: int = 4) -> Workload:
    """3D three-layer medium (Vp 2.0/3.0/4.0 for depth fractions [0,80)/[80,170)/[170,256) of
    256) plus a Gaussian inclusion Vp*(1 + 0.2 exp(-r^2/24^2)) at the centre; Vs = Vp/sqrt(3),
    rho 1.0/1.2/1.4 by layer; 10 points per minimum shear wavelength; u3 point force. Solver:
    K(1,1) on 4 levels (the paper's 3D cycle; coarsest 32^3 at n = 256), shifts 0.4 / 0.5 / 0.6 /
    0.8 from the finest level down, damping 0.35, the hybrid Kaczmarz-GMRES coarsest solve
    (Sec. 3.2, 5.3), FGMRES(8). Measured at 256^3 (FGMRES iterations, seconds): this recipe 85,
    4.28; damping 0.3 91, 4.60; 0.25 110, 5.72; 0.2 138, 7.09; one shift 0.4 on every level with
    damping 0.25 168, 9.38; 3 levels with 16 red-black sweeps on a 64^3 coarsest level shifted
    by 2.5 (the previous recipe) 193, 8.29."""
    s = n / 256.0
    z = (np.arange(n) + 0.5)
    vp1 = np.where(z < 80 * s, 2.0, np.where(z < 170 * s, 3.0, 4.0))
    rho1 = np.where(z < 80 * s, 1.0, np.where(z < 170 * s, 1.2, 1.4))
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    c = n / 2.0
    r2 = (X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2
    vp = vp1[:, None, None] * (1.0 + 0.2 * np.exp(-r2 / (24.0 * s) ** 2))
    rho = np.broadcast_to(rho1[:, None, None], vp.shape).copy()
    vs = vp / np.sqrt(3.0)
    lam, mu = lame_from_velocity(vp, vs, rho)
    h = 1.0
    omega = omega_for_points_per_wavelength(float(vs.min()), h)
    src = tuple(int(round(v * s)) for v in source)
    rhs = point_source((n, n, n), 2, src)
    return Workload("c3_layered_3d_%d" % n, (n, n, n), h, lam, mu, rho, omega, rhs,
                    levels=levels, alpha=0.4, damping=0.35, abl_cells=max(2, int(round(20 * s))),
                    coarse="kaczmarz", cycle="K", level_alpha=(0.4, 0.5, 0.6, 0.8),
                    nu_pre=1, nu_post=1, restart=8)



def config_c5_adjoint(n: int = 128, seed: int = 0, source_side: int = 4, receiver_side: int = 64,
                      depth: int = 4) -> Workload:
    """3D inversion setting for the misfit gradient: a smooth random medium built like the 2D one
    (white noise, Gaussian filter sigma n/16 cells, Vp mapped onto [1.5, 4.5], Vs = Vp/sqrt(3),
    rho = 0.31 Vp^0.25) as the current model; the data model adds a Gaussian blob of +5 % in Vp
    (radius n/8, at the grid centre, Vs and rho following Vp). source_side^2 unit point forces in
    the depth component u3 on a regular grid at depth index `depth`, receiver_side^2 receivers of
    u3 on a regular grid at the same depth; 10 points per minimum shear wavelength of the
    current model. extra: "sources" (DOF arrays), "receivers" ((comp, (i, j, k)) tuples, x1
    first), "true" (lam, mu, rho of the data model). Solver: the 3D recipe (K(1,1) on 4 levels at
    n >= 64, fewer below so that the coarsest level keeps at least 8^3 cells; shifts 0.4 / 0.5 /
    0.6 / 0.8; the hybrid Kaczmarz-GMRES coarsest solve; FGMRES(8)) with damping 0.25. Measured at 128^3 per source (FGMRES iterations, seconds, forward / adjoint):
    35 / 35, 0.65 / 0.69; damping 0.3 35 / 35, 0.67 / 0.70; the previous 3-level recipe with 16
    red-black sweeps on a 32^3 coarsest level shifted by 2.5, 240 / 239, 1.74 / 2.00."""
    shape = (n, n, n)
    vp = gaussian_random_velocity(shape, seed, sigma_cells=n / 16.0)
    z = np.arange(n) + 0.5
    Z, Y, X = np.meshgrid(z, z, z, indexing="ij")
    c = n / 2.0
    blob = 1.0 + 0.05 * np.exp(-((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) / (n / 8.0) ** 2)

    def model(v):
        vs = v / np.sqrt(3.0)
        rho = 0.31 * v ** 0.25
        lam, mu = lame_from_velocity(v, vs, rho)
        return lam, mu, rho

    lam, mu, rho = model(vp)
    h = 1.0
    omega = omega_for_points_per_wavelength(float(vp.min() / np.sqrt(3.0)), h)
    grid = lambda k: [int((i + 0.5) * n / k) for i in range(k)]
    sources = [point_source(shape, 2, (i, j, depth)) for j in grid(source_side) for i in grid(source_side)]
    receivers = [(2, (i, j, depth)) for j in grid(receiver_side) for i in grid(receiver_side)]
    levels = min(4, max(2, int(np.log2(n)) - 2))  # coarsest level of at least 8^3 below 128^3
    w = Workload("c5_adjoint_3d_%d" % n, shape, h, lam, mu, rho, omega, sources[0],
                 levels=levels, alpha=0.4, damping=0.25, abl_cells=max(2, int(round(20 * n / 256.0))),
                 coarse="kaczmarz", cycle="K", level_alpha=(0.4, 0.5, 0.6, 0.8),
                 nu_pre=1, nu_post=1, restart=8)
    w.extra["sources"] = sources
    w.extra["receivers"] = receivers
    w.extra["true"] = model(vp * blob)
    return w

def small_heterogeneous(n, seed: int = 1, sigma_cells: float = 2.0, abl_cells: int = 2,
                        levels: int = 2, omega_ppw: float = 10.0) -> Workload:
    """A small random heterogeneous medium for parity tests (any dimension)."""
    n = tuple(n)
    shape = n[::-1]
    vp = gaussian_random_velocity(shape, seed, sigma_cells=sigma_cells, vmin=1.5, vmax=3.0)
    vs = vp / np.sqrt(3.0)
    rho = 0.31 * vp ** 0.25
    lam, mu = lame_from_velocity(vp, vs, rho)
    h = 1.0
    omega = omega_for_points_per_wavelength(float(vs.min()), h, omega_ppw)
    rng = np.random.default_rng(seed + 7)
    rhs = (rng.standard_normal((len(n) + 1,) + shape)
           + 1j * rng.standard_normal((len(n) + 1,) + shape))
    return Workload("small_%s_s%d" % ("x".join(map(str, n)), seed), n, h, lam, mu, rho, omega, rhs,
                    levels=levels, alpha=0.4, damping=0.5, abl_cells=abl_cells, coarse="dense")
