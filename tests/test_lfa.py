"""The LFA tool (paper_2307_03242_gb300.lfa) against the oracle and against Section 4's numbers.

Parity with the oracle (exact up to rounding): on an n x n periodic grid every operator of the
two-grid cycle is translation invariant, so a field made of the four harmonics of Definition 4.3
stays in their span. The oracle's assembled operator, red-black sweep, transfers and two-grid
cycle applied to such a field must give what the tool's symbol matrices predict. The
lexicographic sweep is not translation invariant on a periodic grid (the first row and column
see unrelaxed neighbours); away from them it converges to the infinite-grid sweep the symbol
describes, so it is compared on an interior window.

Against the paper: the smoothing factors (Table 1's mu_loc^2, Section 4.2's optimal mu_loc) and
the frequency, shift and beta limits stated in Section 4.2; the printed rho_loc of Table 1 for
beta = 1. For beta = 2/3 the tool's rho_loc (0.25 / 0.30 / 0.43) lies between the two-grid factor
measured in practice (0.24 / 0.27 / 0.35, which the oracle reproduces) and the printed 0.37 /
0.40 / 0.47; that case is checked for its bounds and ordering only.
"""
import os

import numpy as np
import pytest

import oracle
from oracle.smoother import cell_dofs, cell_blocks, cell_colour, red_black_sweep, lexicographic_sweep
from paper_2307_03242_gb300 import lfa

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            out.append(line.split())
    return out


def _periodic(n, beta, omega_h, alpha, smoother="full", lam=500.0):
    h = 1.0 / n
    sh = (n, n)
    pb = oracle.Problem((n, n), h, omega_h / h, 0.0, beta, np.full(sh, lam), np.full(sh, 1.0), np.full(sh, 1.0),
                        periodic=True)
    H = oracle.assemble(pb, alpha).tocsr()
    idx = cell_dofs(pb)
    V = cell_blocks(H, idx, economic=smoother == "economic")
    s = lfa.Setting(beta=beta, omega_h=omega_h, alpha=alpha, lam=lam, smoother=smoother, h=h)
    return pb, H, idx, V, s


def _field(n, modes):
    """sum over (theta, amplitude[3]) of amplitude[c] exp(i theta . k), DOF layout (3, ny, nx)."""
    ky, kx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out = np.zeros((3, n, n), dtype=np.complex128)
    for th, a in modes:
        out += a[:, None, None] * np.exp(1j * (th[0] * kx + th[1] * ky))[None]
    return out.ravel()


def _project(n, x, th):
    ky, kx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ph = np.exp(-1j * (th[0] * kx + th[1] * ky))
    return np.array([(x.reshape(3, n, n)[c] * ph).mean() for c in range(3)])


def _amp(rng, k):
    return rng.standard_normal(k) + 1j * rng.standard_normal(k)


SETTINGS = [(2.0 / 3.0, np.pi / 5, 0.15), (1.0, np.pi / 4, 0.2), (0.8, np.pi / 3.3, 0.3)]


@pytest.mark.parametrize("beta,omega_h,alpha", SETTINGS)
def test_operator_symbol_matches_oracle(beta, omega_h, alpha):
    n = 16
    pb, H, _, _, s = _periodic(n, beta, omega_h, alpha)
    rng = np.random.default_rng(1)
    for m in [(0, 0), (3, 1), (8, 8), (5, 12), (15, 2)]:
        th = 2 * np.pi * np.array(m) / n
        a = _amp(rng, 3)
        y = H @ _field(n, [(th, a)])
        want = lfa.operator_symbol(s, th)[0] @ a
        assert np.allclose(_project(n, y, th), want, rtol=0, atol=1e-11 * np.abs(want).max())
        # and nothing leaks into other frequencies
        assert np.allclose(y, _field(n, [(th, want)]), rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("smoother", ["full", "economic"])
@pytest.mark.parametrize("beta,omega_h,alpha", SETTINGS)
def test_red_black_symbol_matches_oracle_sweep(smoother, beta, omega_h, alpha):
    n = 16
    pb, H, idx, V, s = _periodic(n, beta, omega_h, alpha, smoother)
    s = lfa.Setting(**{**s.__dict__, "w": 0.55})
    col = cell_colour(pb)
    rng = np.random.default_rng(2)
    for m in [(1, 2), (4, 0), (7, 3), (2, 6)]:
        th = 2 * np.pi * np.array(m) / n
        thb = th + np.pi
        a, b = _amp(rng, 3), _amp(rng, 3)
        y = red_black_sweep(H, V, idx, col, np.zeros(3 * n * n), _field(n, [(th, a), (thb, b)]), s.w)
        want = lfa.red_black_symbol(s, th)[0] @ np.r_[a, b]
        got = np.r_[_project(n, y, th), _project(n, y, thb)]
        assert np.allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max()), (m, got, want)


@pytest.mark.parametrize("smoother", ["full", "economic"])
def test_lexicographic_symbol_matches_oracle_sweep_away_from_the_start(smoother):
    n = 64
    beta, omega_h, alpha = 2.0 / 3.0, np.pi / 5, 0.15
    pb, H, idx, V, s = _periodic(n, beta, omega_h, alpha, smoother)
    s = lfa.Setting(**{**s.__dict__, "w": 0.65})
    Vinv = np.linalg.inv(V)
    rng = np.random.default_rng(3)
    win = (slice(None), slice(n // 2, 3 * n // 4), slice(n // 2, 3 * n // 4))
    for m in [(20, 5), (32, 32), (10, 40), (40, 17), (3, 2)]:
        th = 2 * np.pi * np.array(m) / n
        a = _amp(rng, 3)
        y = lexicographic_sweep(H, Vinv, idx, np.zeros(3 * n * n), _field(n, [(th, a)]), s.w)
        pred = lfa.smoother_symbol(s, th)[0] @ a
        want = _field(n, [(th, pred)]).reshape(3, n, n)
        err = np.abs(y.reshape(3, n, n)[win] - want[win]).max() / np.abs(pred).max()
        # the start-up disturbance decays geometrically away from the first row and column; a
        # wrong coupling would leave an O(1) difference
        assert err < 1e-5, (m, err)


def _harmonic_field(n, th, A):
    return _field(n, [(h[0], A[3 * i:3 * i + 3]) for i, h in enumerate(lfa.harmonics(th))])


def _harmonic_project(n, x, th):
    return np.concatenate([_project(n, x, h[0]) for h in lfa.harmonics(th)])


@pytest.mark.parametrize("beta,omega_h,alpha", SETTINGS)
def test_coarse_correction_symbol_matches_oracle(beta, omega_h, alpha):
    n = 16
    pb, H, _, _, s = _periodic(n, beta, omega_h, alpha)
    pc = oracle.coarsen(pb)
    Hc = oracle.assemble(pc, alpha).toarray()
    R, P = oracle.restriction(pb, pc), oracle.prolongation(pb, pc)
    rng = np.random.default_rng(4)
    for m in [(0, 0), (1, 3), (-3, 2), (2, -1)]:
        th = 2 * np.pi * np.array(m) / n
        A = _amp(rng, 12)
        x = _harmonic_field(n, th, A)
        y = x - P @ np.linalg.solve(Hc, R @ (H @ x))
        want = lfa.coarse_correction_symbol(s, th)[0] @ A
        assert np.allclose(_harmonic_project(n, y, th), want, rtol=0, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("smoother", ["full", "economic"])
def test_two_grid_symbol_matches_oracle_red_black_cycle(smoother):
    """Eq. symbolTG with nu1 = nu2 = 1 against the oracle's two-grid cycle (pre-sweep, exact
    coarse correction, post-sweep) on the error equation."""
    n = 16
    beta, omega_h, alpha = 2.0 / 3.0, np.pi / 4, 0.2
    pb, H, idx, V, s = _periodic(n, beta, omega_h, alpha, smoother)
    s = lfa.Setting(**{**s.__dict__, "w": 0.5, "order": "red-black"})
    pc = oracle.coarsen(pb)
    Hc = oracle.assemble(pc, alpha).toarray()
    R, P = oracle.restriction(pb, pc), oracle.prolongation(pb, pc)
    col = cell_colour(pb)
    zero = np.zeros(3 * n * n)
    rng = np.random.default_rng(5)
    for m in [(1, 1), (3, -2), (0, 2)]:
        th = 2 * np.pi * np.array(m) / n
        A = _amp(rng, 12)
        x = red_black_sweep(H, V, idx, col, zero, _harmonic_field(n, th, A), s.w)
        x = x - P @ np.linalg.solve(Hc, R @ (H @ x))
        x = red_black_sweep(H, V, idx, col, zero, x, s.w)
        want = lfa.two_grid_symbol(s, th)[0] @ A
        assert np.allclose(_harmonic_project(n, x, th), want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_symbols_are_2pi_periodic_and_lex_equals_red_black_to_first_order_in_w():
    s = lfa.Setting(beta=2.0 / 3.0, omega_h=np.pi / 5, alpha=0.15)
    th = np.array([[0.3, -1.1], [2.0, 0.4]])
    for f in (lfa.operator_symbol, lfa.smoother_symbol):
        assert np.allclose(f(s, th), f(s, th + 2 * np.pi), atol=1e-9)
    # with a tiny damping both sweeps are I - w (sum of the cell corrections) + O(w^2)
    eps = 1e-6
    se = lfa.Setting(**{**s.__dict__, "w": eps})
    lex = (lfa.smoother_symbol(se, th) - np.eye(3)) / eps
    rb = lfa.red_black_symbol(se, th)
    assert np.allclose((rb[:, :3, :3] - np.eye(3)) / eps, lex, rtol=1e-4, atol=1e-4 * np.abs(lex).max())


# ------------------------------------------------------------ Section 4 numbers
def _table1():
    return [tuple(float(v) for v in r) for r in _rows("table1_cf.txt")]


@pytest.mark.parametrize("row", _table1())
def test_smoothing_factor_matches_table1(row):
    beta, w, omega_h, alpha, _, mu2 = row
    s = lfa.Setting(beta=beta, w=w, omega_h=omega_h, alpha=alpha)
    assert abs(lfa.mu_loc(s, step=0.02) ** 2 - mu2) <= 0.02


@pytest.mark.parametrize("row", [tuple(float(v) for v in r) for r in _rows("sec42_mu_opt.txt")])
def test_optimal_smoothing_factor_matches_section_4_2(row):
    beta, w, omega_h, alpha, mu = row
    s = lfa.Setting(beta=beta, w=w, omega_h=omega_h, alpha=alpha)
    assert abs(lfa.mu_loc(s, step=0.02) - mu) <= 0.015


@pytest.fixture(scope="module")
def table1_rho():
    out = {}
    for r in _rows("table1_rho_loc.txt"):
        beta, w, omega_h, alpha, printed = (float(v) for v in r)
        s = lfa.Setting(beta=beta, w=w, omega_h=omega_h, alpha=alpha)
        out[(beta, omega_h)] = (lfa.rho_loc(s, step=0.04)[0], printed)
    return out


def test_two_grid_factor_table1(table1_rho):
    for (beta, omega_h), (got, printed) in table1_rho.items():
        if beta == 1.0:
            assert abs(got - printed) <= 0.05, (beta, omega_h, got, printed)
        else:
            # at most the printed value, at least the factor measured in practice (Table 1's c_f)
            c_f = [r[4] for r in _table1() if r[0] == beta and abs(r[2] - omega_h) < 1e-12][0]
            assert c_f <= got <= printed + 0.01, (beta, omega_h, got, printed)
            assert got < table1_rho[(1.0, omega_h)][0] - 0.3
    spread = [table1_rho[k][0] for k in sorted(k for k in table1_rho if k[0] != 1.0)]
    assert spread == sorted(spread)


def _limits():
    return {r[0]: float(r[1]) for r in _rows("sec42_lfa_limits.txt")}


def test_beta_two_thirds_is_near_optimal():
    s = lfa.Setting(beta=2.0 / 3.0, w=0.7, omega_h=np.pi / 5, alpha=0.1)
    betas = np.arange(0.5, 1.0001, 0.04)
    r = lfa.sweep(s, "beta", betas, step=0.04)
    best = betas[int(np.argmin(r))]
    assert abs(best - _limits()["beta_opt"]) <= 0.1, (best, r)
    assert lfa.rho_loc(s, step=0.04)[0] <= r.min() + 0.01   # 2/3 within 0.01 of the optimum
    assert r[-1] > 2.5 * r.min()                             # the standard stencil is far worse


def test_minimal_shift_and_points_per_wavelength():
    lim = _limits()
    base = lfa.Setting(omega_h=np.pi / 5, alpha=0.1)
    a23 = lfa.minimal_shift(lfa.Setting(**{**base.__dict__, "beta": 2.0 / 3.0, "w": 0.65}), 0.0, 0.5, step=0.04,
                            tol=4e-3)
    a1 = lfa.minimal_shift(lfa.Setting(**{**base.__dict__, "beta": 1.0, "w": 0.75}), 0.0, 0.5, step=0.04, tol=4e-3)
    assert abs(a23 - lim["alpha_min_beta_2_3"]) <= 0.025 and abs(a1 - lim["alpha_min_beta_1"]) <= 0.025
    assert a23 < a1

    def rho_at(beta, w, ppw):
        return lfa.rho_loc(lfa.Setting(beta=beta, w=w, omega_h=2 * np.pi / ppw, alpha=0.1), step=0.04)[0]

    p23, p1 = lim["ppw_min_beta_2_3"], lim["ppw_min_beta_1"]
    assert rho_at(2.0 / 3.0, 0.65, p23) < 1.0 < rho_at(2.0 / 3.0, 0.65, p23 - 1.0)
    assert rho_at(1.0, 0.75, p1) < 1.0 < rho_at(1.0, 0.75, p1 - 2.0)


def test_damping_by_level_decreases_towards_the_coarse_grids():
    """Coarser levels have fewer points per wavelength; their best damping is smaller and their
    two-grid factor larger (Section 5.2 uses a smaller w on coarser grids for the same reason)."""
    s = lfa.Setting(beta=2.0 / 3.0, omega_h=np.pi / 5, alpha=0.5, lam=1.0, smoother="full", order="red-black",
                    nu1=1, nu2=1, h=1.0)
    rec = lfa.damping_by_level(s, 4, candidates=np.array([0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8]), step=0.08)
    ws, rhos = [r[0] for r in rec], [r[1] for r in rec]
    assert len(rec) == 3
    assert ws[0] >= ws[1] >= ws[2] and ws[0] > ws[2], rec
    assert rhos[0] < rhos[1] < rhos[2] < 1.0, rec


def test_smoothing_factor_is_smallest_near_the_printed_damping():
    """Figure 4.1 (left) and its text: mu_loc is smallest near w = 0.65 (beta = 2/3) and w = 0.75
    (beta = 1), and nearly so for every beta at w = 0.7 (omega = pi/(5h), alpha = 0.1)."""
    ws = np.round(np.arange(0.5, 0.91, 0.05), 2)
    for r in _rows("sec42_mu_opt.txt"):
        beta, w_opt, omega_h, alpha, _ = (float(v) for v in r)
        s = lfa.Setting(beta=beta, omega_h=omega_h, alpha=alpha)
        mus = lfa.sweep(s, "w", ws, fn="mu_loc", step=0.04)
        assert abs(ws[int(np.argmin(mus))] - w_opt) <= 0.05 + 1e-9, (beta, list(zip(ws, mus)))
        assert mus[list(ws).index(0.7)] <= mus.min() + 0.01


def test_red_black_order_is_no_worse_than_lexicographic_at_table1_settings():
    """The GPU smoother's red-black order against the lexicographic order of the paper's analysis
    (economic Vanka, one pre- and one post-step): the two-grid factor is not larger."""
    for r in _table1():
        beta, w, omega_h, alpha = r[:4]
        base = dict(beta=beta, w=w, omega_h=omega_h, alpha=alpha)
        lex = lfa.rho_loc(lfa.Setting(**base), step=0.04)[0]
        rb = lfa.rho_loc(lfa.Setting(order="red-black", **base), step=0.04)[0]
        assert rb <= lex + 1e-3, (r, lex, rb)
