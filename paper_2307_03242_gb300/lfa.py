"""Local Fourier analysis of the two-grid cycle for the 2D mixed elastic Helmholtz discretisation
(Section 4): the tool that tunes beta, the damping w and the shift alpha before a solve.

This is host-side analysis on small dense symbol matrices (numpy); it is not part of the solve
path and launches nothing on the GPU.

Setting (Section 4.2): constant lambda, mu, rho on an infinite grid with spacing h, the operator of
Eq. 4.4 (mixed-discretized-homogeneous) with the beta-spread Laplacian, mass and divergence, the
standard gradient of p, and the complex mass coefficient m = rho omega^2 (1 - i(gamma + alpha)).
Grid conventions: u_1[k] sits on the low x-face of cell k, u_2[k] on its low y-face, p[k] at its
centre; a Fourier mode of frequency theta has the value a_c exp(i theta . k) at index k of
component c (index phases: the staggered offsets only multiply every symbol by fixed diagonal
phase matrices, which leaves every spectral radius unchanged).

Operators, as stencils over index offsets (a row at index k couples to index k + d):
  * d_e u_c: along e == c, (v[k+1] - v[k]) / h (faces to cells); along e != c,
    (v[k] - v[k-1]) / h (to the lattice points); the beta-spread version is
    beta D + (1 - beta) D smoothed by [1 2 1]/4 across (Eq. 3.5 dxSpread);
  * u_c block: sum_e D_ce^T mu D_ce^beta - m M^beta, M^beta = beta + (1 - beta)/4 (4 neighbours);
  * u_c <- p: (p[k] - p[k-1]) / h along c; p <- u_c: the spread D_cc^beta; p <- p: 1/(lambda+mu).

Vanka smoother symbol (Section 4.1 and 4.2; the paper omits the derivation and points to the
overlapping-smoother technique of MacLachlan and Oosterlee): every cell k receives a correction
c exp(i theta . k) of its five unknowns (u_1 low/high face, u_2 low/high face, p). With the local
block V (economic: its displacement part reduced to the diagonal), damping w, and L(theta) the
coupling of a cell's rows to the corrections of the cells relaxed before it, the lexicographic
sweep (x fastest) satisfies (V/w + L) c = -Phi H a, so that
    S(theta) = I - G (V/w + L)^{-1} Phi H(theta),
with Phi picking a cell's rows out of a mode and G summing the two cells that correct every face.
The red-black sweep relaxes one colour at a time with the pre-half-sweep residual (Jacobi within a
colour); its half-sweeps couple theta with theta + (pi, pi).

Two-grid symbol (Eq. symbolTG) on the four harmonics of Definition 4.3:
    TG = S^nu2 (I - P A_2h^{-1} R A_h) S^nu1,
with R and P the tensor-product transfers of Eq. 2.11-2.12 and A_2h the re-discretised coarse
operator at 2h. rho_loc (Definition 4.2) is the supremum of rho(TG) over T_low; mu_loc
(Definition 4.1) the supremum of rho(S) over T_high (for red-black, the ideal-correction form
rho(S^nu2 Q S^nu1)^(1/nu) with Q removing the low harmonic).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

U1, U2, P = 0, 1, 2
# the cell's unknowns in the order of the library's block solve: (component, index offset)
CELL = ((U1, (0, 0)), (U1, (1, 0)), (U2, (0, 0)), (U2, (0, 1)), (P, (0, 0)))
# the harmonics of Definition 4.3: theta, theta + (pi, pi), theta + (pi, 0), theta + (0, pi)
HARMONICS = ((0, 0), (1, 1), (1, 0), (0, 1))


@dataclass(frozen=True)
class Setting:
    """Constant-coefficient problem and smoother. omega_h = omega * h (pi/5 is 10 points per
    wavelength of the slowest wave when the shear velocity is 1)."""
    beta: float = 2.0 / 3.0
    omega_h: float = np.pi / 5.0
    alpha: float = 0.1
    w: float = 0.65
    lam: float = 500.0
    mu: float = 1.0
    rho: float = 1.0
    gamma: float = 0.0
    h: float = 1.0 / 1024.0
    smoother: str = "economic"   # "economic" | "full"
    order: str = "lex"           # "lex" | "red-black"
    nu1: int = 1
    nu2: int = 1


# ------------------------------------------------------------------ stencils
def _conv(a, b):
    out = {}
    for da, ca in a.items():
        for db, cb in b.items():
            d = (da[0] + db[0], da[1] + db[1])
            out[d] = out.get(d, 0.0) + ca * cb
    return out


def _add(a, b, sa=1.0, sb=1.0):
    out = {d: sa * c for d, c in a.items()}
    for d, c in b.items():
        out[d] = out.get(d, 0.0) + sb * c
    return out


def _transpose(a):
    return {(-d[0], -d[1]): c for d, c in a.items()}


def _along(axis, taps):
    return {((o, 0) if axis == 0 else (0, o)): c for o, c in taps.items()}


def _derivative(comp, e, h, beta=None):
    """d_e u_comp as a stencil; beta given: the spread version."""
    taps = {0: -1.0 / h, 1: 1.0 / h} if e == comp else {0: 1.0 / h, -1: -1.0 / h}
    D = _along(e, taps)
    if beta is None:
        return D
    smooth = _along(1 - e, {-1: 0.25, 0: 0.5, 1: 0.25})
    return _add(D, _conv(smooth, D), beta, 1.0 - beta)


def operator_stencil(s: Setting, h: float):
    """{(row component, column component): {offset: coefficient}} of the shifted operator on a
    grid of spacing h (the same omega and shift on every grid: re-discretisation)."""
    m = s.rho * (s.omega_h / s.h) ** 2 * (1.0 - 1j * (s.gamma + s.alpha))
    mass = {(0, 0): s.beta, (1, 0): (1 - s.beta) / 4, (-1, 0): (1 - s.beta) / 4, (0, 1): (1 - s.beta) / 4,
            (0, -1): (1 - s.beta) / 4}
    st = {}
    for c in (U1, U2):
        lap = {}
        for e in (0, 1):
            lap = _add(lap, _conv(_transpose(_derivative(c, e, h)), _derivative(c, e, h, s.beta)), 1.0, s.mu)
        st[(c, c)] = _add(lap, mass, 1.0, -m)
        st[(c, P)] = _along(c, {0: 1.0 / h, -1: -1.0 / h})
        st[(P, c)] = _derivative(c, c, h, s.beta)
    st[(P, P)] = {(0, 0): 1.0 / (s.lam + s.mu)}
    return st


def _symbol(st, theta):
    """(N, 3, 3) matrix of symbols for theta of shape (N, 2)."""
    out = np.zeros((theta.shape[0], 3, 3), dtype=np.complex128)
    for (r, c), taps in st.items():
        for d, coef in taps.items():
            out[:, r, c] += coef * np.exp(1j * (theta[:, 0] * d[0] + theta[:, 1] * d[1]))
    return out


def operator_symbol(s: Setting, theta, coarse=False):
    """H(theta), (N, 3, 3), on the fine grid (spacing h) or the coarse one (2h)."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    return _symbol(operator_stencil(s, 2 * s.h if coarse else s.h), theta)


# ------------------------------------------------------------------ Vanka
def cell_block(s: Setting):
    """The 5x5 local block V of one cell (economic: displacement part reduced to its diagonal)."""
    st = operator_stencil(s, s.h)
    V = np.zeros((5, 5), dtype=np.complex128)
    for a, (ca, oa) in enumerate(CELL):
        for b, (cb, ob) in enumerate(CELL):
            V[a, b] = st.get((ca, cb), {}).get((ob[0] - oa[0], ob[1] - oa[1]), 0.0)
    if s.smoother == "economic":
        for a in range(4):
            for b in range(4):
                if a != b:
                    V[a, b] = 0.0
    elif s.smoother != "full":
        raise ValueError("smoother must be 'full' or 'economic'")
    return V


def _phase(theta, o):
    return np.exp(1j * (theta[:, 0] * o[0] + theta[:, 1] * o[1]))


def _pick_and_spread(theta):
    """Phi (N, 5, 3): a mode's values at a cell's unknowns; G (N, 3, 5): the mode amplitudes of
    the faces that cell corrections of the form c exp(i theta . k) change."""
    N = theta.shape[0]
    Phi = np.zeros((N, 5, 3), dtype=np.complex128)
    G = np.zeros((N, 3, 5), dtype=np.complex128)
    for l, (c, o) in enumerate(CELL):
        Phi[:, l, c] = _phase(theta, o)
        G[:, c, l] = np.conj(_phase(theta, o))
    return Phi, G


def _earlier_coupling(s: Setting, theta):
    """L (N, 5, 5): rows of a cell against the corrections of the cells relaxed before it in
    lexicographic order (x fastest), i.e. offsets (dx, dy) with dy < 0, or dy == 0 and dx < 0."""
    st = operator_stencil(s, s.h)
    L = np.zeros((theta.shape[0], 5, 5), dtype=np.complex128)
    for a, (ca, oa) in enumerate(CELL):
        for b, (cb, ob) in enumerate(CELL):
            for d, coef in st.get((ca, cb), {}).items():
                # the cell at offset e couples through d = e + ob - oa
                e = (d[0] - ob[0] + oa[0], d[1] - ob[1] + oa[1])
                if e[1] < 0 or (e[1] == 0 and e[0] < 0):
                    L[:, a, b] += coef * _phase(theta, e)
    return L


def smoother_symbol(s: Setting, theta):
    """Lexicographic Vanka: S(theta), (N, 3, 3)."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    H = operator_symbol(s, theta)
    Phi, G = _pick_and_spread(theta)
    M = cell_block(s)[None] / s.w + _earlier_coupling(s, theta)
    return np.eye(3)[None] - G @ np.linalg.solve(M, Phi @ H)


def red_black_symbol(s: Setting, theta):
    """Red-black Vanka (colour 0 then colour 1, Jacobi within a colour): (N, 6, 6) acting on the
    amplitudes (a_theta, a_{theta + (pi, pi)})."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    Vi = np.linalg.inv(cell_block(s))
    pair = (theta, theta + np.pi)
    GB = []
    for ph in pair:
        Phi, G = _pick_and_spread(ph)
        GB.append((G, -s.w * (Vi[None] @ Phi @ operator_symbol(s, ph))))
    N = theta.shape[0]
    sweep = np.broadcast_to(np.eye(6, dtype=np.complex128), (N, 6, 6)).copy()
    for colour in (0, 1):
        sg = -1.0 if colour else 1.0
        K = np.broadcast_to(np.eye(6, dtype=np.complex128), (N, 6, 6)).copy()
        for i in range(2):
            for j in range(2):
                f = 0.5 if i == j else 0.5 * sg
                K[:, 3 * i:3 * i + 3, 3 * j:3 * j + 3] += f * (GB[i][0] @ GB[j][1])
        sweep = K @ sweep
    return sweep


# ------------------------------------------------------------------ transfers
def _transfer_taps(comp, axis, kind):
    """1-D weights along `axis` for component `comp`: R: coarse K <- fine 2K + d; P: fine 2K + d
    <- coarse K (Eq. 2.11 pIntergrid, Eq. 2.12 u2Intergrid)."""
    face = comp == axis
    if kind == "R":
        return {-1: 0.25, 0: 0.5, 1: 0.25} if face else {0: 0.5, 1: 0.5}
    return {-1: 0.5, 0: 1.0, 1: 0.5} if face else {-1: 0.25, 0: 0.75, 1: 0.75, 2: 0.25}


def _transfer_symbol(comp, kind, theta):
    tx, ty = _transfer_taps(comp, 0, kind), _transfer_taps(comp, 1, kind)
    sg = 1.0 if kind == "R" else -1.0
    out = np.zeros(theta.shape[0], dtype=np.complex128)
    for dx, cx in tx.items():
        for dy, cy in ty.items():
            out += cx * cy * np.exp(sg * 1j * (theta[:, 0] * dx + theta[:, 1] * dy))
    return out if kind == "R" else 0.25 * out


def harmonics(theta):
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    return [theta + np.pi * np.array(a, dtype=np.float64) for a in HARMONICS]


def coarse_correction_symbol(s: Setting, theta):
    """I - P A_2h^{-1} R A_h on the four harmonics: (N, 12, 12), index 3 * harmonic + component;
    the coarse mode has index frequency 2 theta."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    N = theta.shape[0]
    hs = harmonics(theta)
    Ah = np.zeros((N, 12, 12), dtype=np.complex128)
    R = np.zeros((N, 3, 12), dtype=np.complex128)
    Pm = np.zeros((N, 12, 3), dtype=np.complex128)
    for a, th in enumerate(hs):
        Ah[:, 3 * a:3 * a + 3, 3 * a:3 * a + 3] = operator_symbol(s, th)
        for c in range(3):
            R[:, c, 3 * a + c] = _transfer_symbol(c, "R", th)
            Pm[:, 3 * a + c, c] = _transfer_symbol(c, "P", th)
    A2h = operator_symbol(s, 2 * theta, coarse=True)
    return np.eye(12)[None] - Pm @ np.linalg.solve(A2h, R @ Ah)


def smoothing_symbol_12(s: Setting, theta):
    """The smoother on the four harmonics, (N, 12, 12)."""
    theta = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    N = theta.shape[0]
    S = np.zeros((N, 12, 12), dtype=np.complex128)
    hs = harmonics(theta)
    if s.order == "lex":
        for a, th in enumerate(hs):
            S[:, 3 * a:3 * a + 3, 3 * a:3 * a + 3] = smoother_symbol(s, th)
    elif s.order == "red-black":
        # theta pairs with theta + (pi, pi) (harmonics 0, 1); theta + (pi, 0) with theta + (0, pi) (2, 3)
        for first, second in ((0, 1), (2, 3)):
            rb = red_black_symbol(s, hs[first])
            ix = np.r_[3 * first:3 * first + 3, 3 * second:3 * second + 3]
            S[:, ix[:, None], ix[None, :]] = rb
    else:
        raise ValueError("order must be 'lex' or 'red-black'")
    return S


def two_grid_symbol(s: Setting, theta):
    """TG(theta) of Eq. symbolTG, (N, 12, 12)."""
    S = smoothing_symbol_12(s, theta)
    K = coarse_correction_symbol(s, theta)
    out = K
    for _ in range(s.nu1):
        out = out @ S
    for _ in range(s.nu2):
        out = S @ out
    return out


# ------------------------------------------------------------------ factors
def low_frequencies(step=0.01):
    """Samples of T_low = [-pi/2, pi/2)^2 with the given spacing."""
    t = np.arange(-np.pi / 2, np.pi / 2, step)
    T1, T2 = np.meshgrid(t, t, indexing="ij")
    return np.stack([T1.ravel(), T2.ravel()], axis=1)


def _spectral_radius(M, chunk=20000):
    out = np.empty(M.shape[0])
    for i in range(0, M.shape[0], chunk):
        out[i:i + chunk] = np.abs(np.linalg.eigvals(M[i:i + chunk])).max(axis=-1)
    return out


def rho_loc(s: Setting, step=0.01, theta=None):
    """Definition 4.2: sup over T_low of rho(TG(theta)); returns (rho_loc, maximising theta)."""
    theta = low_frequencies(step) if theta is None else np.atleast_2d(theta)
    r = _spectral_radius(two_grid_symbol(s, theta))
    i = int(np.argmax(r))
    return float(r[i]), theta[i]


def mu_loc(s: Setting, step=0.01, nu=1):
    """Definition 4.1 (lexicographic: sup over T_high of rho(S(theta)), sampled as the three high
    harmonics of every sample of T_low); for red-black, the ideal-correction form
    sup rho(S^(nu - 1) Q S)^(1/nu) over the harmonics, Q removing the low one."""
    theta = low_frequencies(step)
    S = smoothing_symbol_12(s, theta)
    Q = np.eye(12)
    Q[0:3, 0:3] = 0.0
    M = Q @ S
    for _ in range(nu - 1):
        M = S @ M
    return float(_spectral_radius(M).max() ** (1.0 / nu))


def minimal_shift(s: Setting, lo=0.0, hi=1.0, step=0.02, tol=1e-3):
    """Smallest alpha with rho_loc < 1 (Figure 4.2 left), by bisection on [lo, hi]."""
    if rho_loc(replace(s, alpha=hi), step)[0] >= 1.0:
        raise ValueError("rho_loc >= 1 even at alpha = %g" % hi)
    if rho_loc(replace(s, alpha=lo), step)[0] < 1.0:
        return lo
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if rho_loc(replace(s, alpha=mid), step)[0] < 1.0:
            hi = mid
        else:
            lo = mid
    return hi


def sweep(s: Setting, field, values, fn="rho_loc", step=0.02):
    """rho_loc (or mu_loc) as one parameter of the setting varies (Figure 4.1)."""
    f = rho_loc if fn == "rho_loc" else mu_loc
    out = []
    for v in values:
        r = f(replace(s, **{field: v}), step)
        out.append(r[0] if isinstance(r, tuple) else r)
    return np.array(out)


def damping_by_level(s: Setting, levels: int, candidates=None, step=0.04):
    """Damping per level of a hierarchy whose finest level is described by `s` (its omega_h,
    shift, material, smoother and sweep counts): level l has spacing 2^l h, hence omega_h 2^l,
    and gets the candidate w with the smallest two-grid factor. The coarsest level is solved
    separately and gets none. Returns [(w, rho_loc), ...] for levels 0 .. levels - 2."""
    cands = np.round(np.arange(0.1, 1.0001, 0.05), 2) if candidates is None else candidates
    out = []
    for l in range(levels - 1):
        sl = replace(s, omega_h=s.omega_h * 2 ** l, h=s.h * 2 ** l)
        r = sweep(sl, "w", cands, step=step)
        i = int(np.argmin(r))
        out.append((float(cands[i]), float(r[i])))
    return out


def _table():
    rows = []
    for beta, w in ((1.0, 0.75), (2.0 / 3.0, 0.65)):
        for omega_h, alpha in ((np.pi / 5, 0.15), (np.pi / 4, 0.2), (np.pi / 3.3, 0.3)):
            s = Setting(beta=beta, w=w, omega_h=omega_h, alpha=alpha)
            rows.append((beta, omega_h, alpha, rho_loc(s)[0], mu_loc(s) ** 2))
    return rows


if __name__ == "__main__":
    print("beta    omega*h  alpha  rho_loc  mu_loc^2   (lambda=500, mu=rho=1, economic Vanka, lex, V(1,1))")
    for beta, omega_h, alpha, r, m2 in _table():
        print("%.4f  %.4f   %.2f   %.3f    %.3f" % (beta, omega_h, alpha, r, m2))
