"""Pins of the oracle's smoother, V-cycle and FGMRES against properties fixed by the method
and by dense direct solves (the plain definition x = H^{-1} q the iteration converges to)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle.discretization import Problem
from oracle.smoother import cell_colour, half_sweep
from workloads import small_heterogeneous
from _paper_symbols import operator_symbol, mode


def _problem(w, periodic=False):
    return Problem(w.n, w.h, w.omega, w.gamma, w.beta, w.lam, w.mu, w.rho,
                   abl_length=0.0 if periodic else w.abl_cells * w.h,
                   abl_gamma_max=w.abl_gamma_max, periodic=periodic)


def _direct(H, b, act):
    x = np.zeros_like(b)
    x[act] = spla.spsolve(H[act][:, act].tocsc(), b[act])
    return x


@pytest.mark.parametrize("n", [(8, 6), (4, 4, 4)])
def test_vanka_single_cell_with_unit_damping_zeroes_its_residuals(n):
    """Full Vanka (Section 2.3): with w = 1 one cell update solves the cell's (2d+1) equations."""
    w = small_heterogeneous(n, levels=1)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.4)
    idx = oracle.cell_dofs(pb)
    V = oracle.cell_blocks(H, idx)
    rng = np.random.default_rng(0)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    x = (rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)) * act
    for cell in (0, pb.ncell // 2 + 1, pb.ncell - 1):
        y = oracle.vanka_cell_update(H, V, idx, cell, b, x, 1.0)
        r = b - H @ y
        ii = idx[cell][idx[cell] >= 0]
        assert np.abs(r[ii]).max() < 1e-12 * np.abs(b).max()
        changed = np.nonzero(y != x)[0]
        assert set(changed) <= set(ii)


def test_red_black_half_sweep_touches_each_face_once_and_only_its_colour_pressures():
    w = small_heterogeneous((8, 8), levels=1)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.4)
    idx = oracle.cell_dofs(pb)
    V = oracle.cell_blocks(H, idx)
    col = cell_colour(pb)
    for c in (0, 1):
        ii = idx[col == c]
        faces = ii[:, :-1][ii[:, :-1] >= 0]
        assert len(faces) == len(set(faces))
        act = oracle.active_mask(pb)
        nact_faces = act[:2 * pb.ncell].sum()
        assert len(faces) == nact_faces
    b = w.rhs.ravel() * oracle.active_mask(pb)
    x0 = np.zeros_like(b)
    x1 = half_sweep(H, V, idx, col, 0, b, x0, 0.7)
    p_changed = np.nonzero(x1[2 * pb.ncell:] != 0)[0]
    assert np.all(col[p_changed] == 0)


def test_smoother_fixed_point_is_the_solution():
    w = small_heterogeneous((8, 8), levels=1)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.4)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    xs = _direct(H, b, act)
    idx = oracle.cell_dofs(pb)
    V = oracle.cell_blocks(H, idx)
    y = oracle.red_black_sweep(H, V, idx, cell_colour(pb), b, xs, 0.5)
    assert np.linalg.norm(y - xs) < 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("n,levels", [((8, 8), 2), ((16, 16), 3), ((16, 8), 2), ((4, 4, 4), 2), ((8, 8, 8), 2)])
def test_fgmres_vcycle_converges_to_dense_direct_solution(n, levels):
    """The solve (FGMRES + V-cycle on H_s, Sections 3.2 and 5) converges to H^{-1} q."""
    w = small_heterogeneous(n, levels=levels, abl_cells=2)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.0)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    xd = _direct(H, b, act)
    hier = oracle.Hierarchy(pb, levels, 0.4, 0.5, coarse="dense")
    x, its, res = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b,
                                tol=1e-11, restart=20, max_iter=300)
    assert res <= 1e-11
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert its < 100


def test_single_level_exact_preconditioner_converges_in_one_iteration():
    w = small_heterogeneous((8, 8), levels=1)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.0)
    hier = oracle.Hierarchy(pb, 1, 0.0, 1.0, coarse="dense")
    b = w.rhs.ravel() * oracle.active_mask(pb)
    x, its, res = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-12)
    assert its == 1 and res < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_plane_wave_solution_on_periodic_grid(dim):
    """Manufactured discrete plane wave: b = H~(theta) u^ e^{i theta x}; the solve returns
    u^ e^{i theta x}, with H~ the closed-form symbol of Eq. (4.4)."""
    n = (16, 16) if dim == 2 else (8, 8, 8)
    h, beta, lam, mu, rho, omega, gamma = 1.0, 2.0 / 3.0, 2.0, 1.0, 1.0, 0.5, 0.01
    shape = tuple(n[::-1])
    pb = Problem(n, h, omega, gamma, beta, np.full(shape, lam), np.full(shape, mu), np.full(shape, rho),
                 periodic=True)
    kidx = [3, 1] if dim == 2 else [1, 2, 1]
    k = [2 * np.pi * kidx[a] / (n[a] * h) for a in range(dim)]
    A = operator_symbol(k, h, beta, lam, mu, rho, omega, gamma)
    uhat = np.arange(1, dim + 2) * (1 + 0.5j)
    bhat = A @ uhat
    b = np.concatenate([bhat[c] * mode(n, h, c, dim, k).ravel() for c in range(dim + 1)])
    want = np.concatenate([uhat[c] * mode(n, h, c, dim, k).ravel() for c in range(dim + 1)])
    H = oracle.assemble(pb, 0.0)
    hier = oracle.Hierarchy(pb, 2, 0.5, 0.5, coarse="dense")
    x, its, res = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-12,
                                restart=30, max_iter=300)
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)


def test_fgmres_with_identity_preconditioner_matches_numpy_solve():
    rng = np.random.default_rng(5)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3 + 1j * rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, its, res = oracle.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, restart=10, max_iter=500)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11)
    x2, its2, _ = oracle.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-13, restart=60, max_iter=500)
    assert its2 <= n


def test_vcycle_is_linear_and_deterministic():
    w = small_heterogeneous((16, 16), levels=3)
    pb = _problem(w)
    hier = oracle.Hierarchy(pb, 3, 0.4, 0.35, coarse="smooth", coarse_sweeps=4, coarse_damping=0.8)
    rng = np.random.default_rng(2)
    act = oracle.active_mask(pb)
    b1 = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    b2 = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    a = 0.3 - 1.7j
    lhs = oracle.vcycle(hier, a * b1 + b2)
    rhs = a * oracle.vcycle(hier, b1) + oracle.vcycle(hier, b2)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)
    assert np.array_equal(oracle.vcycle(hier, b1), oracle.vcycle(hier, b1))
    assert np.all(lhs[~act] == 0)


@pytest.mark.parametrize("n", [(24, 20), (12, 10, 8)])
def test_windowed_operator_matches_full_operator_away_from_cuts(n):
    """oracle.window: rows >= 3 cells from a cut edge equal the full operator's rows (incl. ABL)."""
    w = small_heterogeneous(n, abl_cells=3)
    pb = _problem(w)
    rng = np.random.default_rng(4)
    shape = oracle.dof_shape(pb)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    y = oracle.apply(pb, x, shift=0.3)
    d = pb.dim
    lo = tuple(0 if a == 0 else 2 for a in range(d))
    hi = tuple(n[a] - 1 if a == 0 else n[a] for a in range(d))
    wp = oracle.window(pb, lo, hi)
    sl = tuple(slice(lo[a], hi[a]) for a in reversed(range(d)))
    yw = oracle.apply(wp, x[(slice(None),) + sl], shift=0.3)
    inner = []
    for a in reversed(range(d)):
        s0 = 0 if lo[a] == 0 else 3
        s1 = (hi[a] - lo[a]) - (0 if hi[a] == n[a] else 3)
        inner.append(slice(s0, s1))
    full_inner = tuple(slice(lo[a] + inner[d - 1 - a].start, lo[a] + inner[d - 1 - a].stop)
                       for a in reversed(range(d)))
    np.testing.assert_allclose(yw[(slice(None),) + tuple(inner)], y[(slice(None),) + full_inner], atol=1e-12)


def test_wcycle_converges_to_dense_direct_solution_in_fewer_iterations():
    """W-cycle (two recursive calls, Sec. 2.2) as preconditioner: same solution, no more iterations."""
    w = small_heterogeneous((32, 32), levels=4, abl_cells=3)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.0)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    xd = _direct(H, b, act)
    its = {}
    for cyc in ("V", "W"):
        hier = oracle.Hierarchy(pb, 4, 0.5, 0.3, coarse="smooth", coarse_sweeps=8, coarse_damping=0.8, cycle=cyc)
        x, its[cyc], res = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-10,
                                         restart=20, max_iter=400)
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert its["W"] <= its["V"]


def test_kcycle_gcr_steps_minimise_the_coarse_residual_and_converge():
    """K-cycle (Sec. 2.2): the GCR(2) correction leaves a residual orthogonal to both search
    directions A z1, A z2, and the preconditioned solve converges to the direct solution."""
    from oracle.multigrid import kcycle_correction
    w = small_heterogeneous((32, 32), levels=4, abl_cells=3)
    pb = _problem(w)
    hier = oracle.Hierarchy(pb, 4, 0.5, 0.3, coarse="smooth", coarse_sweeps=8, coarse_damping=0.8, cycle="K")
    rng = np.random.default_rng(8)
    act = oracle.active_mask(hier.pbs[1])
    r = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    e = kcycle_correction(hier, r, 1)
    A = hier.H[1]
    res = r - A @ e
    z1 = oracle.vcycle(hier, r, None, 1)
    q1 = A @ z1
    assert abs(np.vdot(q1, res)) <= 1e-10 * np.linalg.norm(q1) * np.linalg.norm(r)
    assert np.linalg.norm(res) <= np.linalg.norm(r - (np.vdot(q1, r) / np.vdot(q1, q1)) * q1) * (1 + 1e-12)
    H = oracle.assemble(pb, 0.0)
    b = w.rhs.ravel() * oracle.active_mask(pb)
    xd = _direct(H, b, oracle.active_mask(pb))
    x, its, res2 = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-10, restart=20,
                                 max_iter=300)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_kcycle_correction_is_the_least_squares_combination_of_its_two_cycles():
    """K-cycle (Sec. 2.2): with z1 = B r and z2 = B r2 (r2 the residual after the first step), the
    two GCR steps return the combination e = c1 z1 + c2 z2 that minimises ||r - A e||; computed
    here by a least-squares solve (numpy lstsq) on [A z1, A z2], not by the GCR recurrences."""
    import oracle.multigrid as mg
    w = small_heterogeneous((32, 32), levels=4, abl_cells=3)
    pb = _problem(w)
    hier = oracle.Hierarchy(pb, 4, 0.5, 0.3, coarse="smooth", coarse_sweeps=8, coarse_damping=0.8, cycle="K")
    rng = np.random.default_rng(9)
    act = oracle.active_mask(hier.pbs[1])
    r = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    A = hier.H[1]
    e = mg.kcycle_correction(hier, r, 1)
    z1 = oracle.vcycle(hier, r, None, 1)
    c1 = np.linalg.lstsq((A @ z1)[:, None], r, rcond=None)[0][0]  # the first step: min over span{z1}
    z2 = oracle.vcycle(hier, r - c1 * (A @ z1), None, 1)
    Z = np.stack([z1, z2], axis=1)
    c = np.linalg.lstsq(A @ Z, r, rcond=None)[0]
    e_ls = Z @ c
    assert np.linalg.norm(e - e_ls) <= 1e-10 * np.linalg.norm(e_ls)


@pytest.mark.parametrize("n", [(8, 6), (4, 4, 4)])
def test_economic_vanka_keeps_the_pressure_coupling_and_solves_the_pressure_row(n):
    """Economic Vanka (Section 2.3): the displacement part of the cell block becomes its diagonal,
    the couplings to the pressure stay. With w = 1 one cell update therefore zeroes the cell's
    pressure residual exactly, and leaves on its faces the residual of the dropped off-diagonal
    displacement couplings, -(V_full - V_econ) delta."""
    w = small_heterogeneous(n, levels=1)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.4)
    idx = oracle.cell_dofs(pb)
    Vf = oracle.cell_blocks(H, idx)
    Ve = oracle.cell_blocks(H, idx, economic=True)
    k = idx.shape[1]
    off = ~np.eye(k - 1, dtype=bool)
    assert np.all(Ve[:, :k - 1, :k - 1][:, off] == 0)
    assert np.allclose(np.diagonal(Ve, axis1=1, axis2=2), np.diagonal(Vf, axis1=1, axis2=2))
    assert np.array_equal(Ve[:, k - 1, :], Vf[:, k - 1, :]) and np.array_equal(Ve[:, :, k - 1], Vf[:, :, k - 1])
    assert np.abs(Vf[:, :k - 1, :k - 1][:, off]).max() > 0  # something was dropped
    rng = np.random.default_rng(1)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    x = (rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)) * act
    for cell in (0, pb.ncell // 2 + 1, pb.ncell - 1):
        y = oracle.vanka_cell_update(H, Ve, idx, cell, b, x, 1.0)
        ii = idx[cell]
        ok = ii >= 0
        r = b - H @ x
        rl = np.where(ok, r[np.maximum(ii, 0)], 0.0)
        delta = np.linalg.solve(Ve[cell], rl)
        r_new = b - H @ y
        assert abs(r_new[ii[-1]]) < 1e-12 * np.abs(b).max()
        expect = -(Vf[cell] - Ve[cell]) @ delta
        assert np.allclose(r_new[ii[:-1][ok[:-1]]], expect[:-1][ok[:-1]], atol=1e-12 * np.abs(b).max())


def test_economic_vanka_cycle_fixes_the_solution_and_converges():
    w = small_heterogeneous((16, 16), levels=2)
    pb = _problem(w)
    H = oracle.assemble(pb, 0.0)
    act = oracle.active_mask(pb)
    b = w.rhs.ravel() * act
    xs = _direct(H, b, act)
    hier = oracle.Hierarchy(pb, 2, 0.3, smoother="economic")
    idx, col = hier.idx[0], hier.colour[0]
    y = oracle.red_black_sweep(hier.H[0], hier.V[0], idx, col, hier.H[0] @ xs, xs, 0.5)
    assert np.linalg.norm(y - xs) < 1e-12 * np.linalg.norm(xs)
    x, its, res = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-10, restart=30,
                                max_iter=300)
    assert res <= 1e-10 and np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)
