"""Pins of the hybrid Kaczmarz-GMRES coarsest solve (oracle/kaczmarz.py, Sections 3.2 and 5.3).

Each pin checks the oracle against something other than itself: the full system's direct solve
(the Schur reduction), the row-projection property of a Kaczmarz update, the Bjorck-Elfving
identity (a Kaczmarz sweep is an SOR sweep on A A^H y = b with x = A^H y, solved here by
scipy's triangular solver), hand-computed component averages, the exact solution as a fixed
point, the monotone error decrease of row projections, the stencil footprint behind the
sub-regions' reach, and order independence of same-coloured boxes."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import kaczmarz as kz
from oracle.discretization import Problem
from workloads import small_heterogeneous


def _problem(w):
    return Problem(w.n, w.h, w.omega, w.gamma, w.beta, w.lam, w.mu, w.rho, abl_length=w.abl_cells * w.h,
                   abl_gamma_max=w.abl_gamma_max)


def _system(n, seed=1, shift=0.4):
    w = small_heterogeneous(n, seed=seed, levels=1)
    pb = _problem(w)
    return kz.SchurSystem(pb, shift), w.rhs.ravel().copy(), pb


def _crand(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ---------------------------------------------------------------- Schur reduction
@pytest.mark.parametrize("n", [(10, 8), (6, 5, 4)])
def test_schur_reduction_reproduces_the_direct_solve(n):
    """Eliminating p (diagonal p-p block) and recovering it gives the full system's solution."""
    sysm, b, pb = _system(n)
    H = oracle.assemble(pb, 0.4)
    act = oracle.active_mask(pb)
    x_ref = np.zeros_like(b)
    x_ref[act] = spla.spsolve(H[act][:, act].tocsc(), b[act])
    u = spla.spsolve(sysm.S.tocsc(), sysm.reduce(b))
    x = sysm.recover(u, b)
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_schur_residual_has_zero_pressure_rows():
    """For any u, recover() satisfies the continuity rows exactly, and the displacement rows of
    the full residual equal the Schur residual (the elimination is exact)."""
    sysm, b, pb = _system((6, 5, 4))
    H = oracle.assemble(pb, 0.4)
    u = _crand(np.random.default_rng(3), sysm.S.shape[0])
    x = sysm.recover(u, b)
    r = b - H @ x
    assert np.abs(r[sysm.nu:]).max() <= 1e-12 * np.abs(b).max()
    rs = sysm.reduce(b) - sysm.S @ u
    assert np.linalg.norm(r[sysm.u_act] - rs) <= 1e-12 * np.linalg.norm(rs)


# ---------------------------------------------------------------- a single Kaczmarz update
def test_hand_examples_of_projection_and_component_average():
    """Rows [1, 1] and [1, -1], rhs (2, 0), one row per sub-region, both reaching both unknowns:
    the first projects 0 onto x1 + x2 = 2, i.e. (1, 1); the second leaves 0 (residual 0); the
    mean is (1/2, 1/2); with damping 0.8 it is (0.4, 0.4). A complex row [i, 1] with rhs 1 moves
    0 to (1/2) conj([i, 1]) = (-i/2, 1/2)."""
    S = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]], dtype=complex))
    part = kz.row_partition(2, 2, [[0], [1]])
    x = kz.kaczmarz_steps(S, part, np.array([2.0, 0.0], complex), np.zeros(2, complex), 1, 1.0)
    assert np.allclose(x, [0.5, 0.5], atol=1e-15)
    x = kz.kaczmarz_steps(S, part, np.array([2.0, 0.0], complex), np.zeros(2, complex), 1, 0.8)
    assert np.allclose(x, [0.4, 0.4], atol=1e-15)
    # one sub-region with both rows in order: (1, 1), then the second row's residual is 0
    seq = kz.row_partition(2, 2, [[0, 1]])
    x = kz.kaczmarz_steps(S, seq, np.array([2.0, 0.0], complex), np.zeros(2, complex), 1, 1.0)
    assert np.allclose(x, [1.0, 1.0], atol=1e-15)
    Sc = sp.csr_matrix(np.array([[1j, 1.0]]))
    x = kz.kaczmarz_steps(Sc, kz.row_partition(1, 2, [[0]]), np.array([1.0 + 0j]), np.zeros(2, complex), 1, 1.0)
    assert np.allclose(x, [-0.5j, 0.5], atol=1e-15)


@pytest.mark.parametrize("n", [(10, 8), (6, 5, 4)])
def test_projection_property_on_the_schur_rows(n):
    """With damping 1, a sub-region whose rows touch pairwise disjoint unknowns ends its sweep
    with zero residual on all of them, moves x only within the span of conj(a_i), and leaves
    every other unknown unchanged; with overlapping rows, the last row swept has zero residual."""
    sysm, b, _ = _system(n)
    S = sysm.S.tocsr()
    rng = np.random.default_rng(5)
    rhs = _crand(rng, S.shape[0])
    x0 = _crand(rng, S.shape[1])
    # greedily pick rows with disjoint supports
    used, rows = set(), []
    for i in rng.permutation(S.shape[0]):
        cols = set(S.indices[S.indptr[i]:S.indptr[i + 1]])
        if not cols & used:
            rows.append(int(i))
            used |= cols
    assert len(rows) >= 4
    part = kz.row_partition(S.shape[0], S.shape[1], [rows])
    x1 = kz.kaczmarz_steps(S, part, rhs, x0, 1, 1.0)
    res = rhs[rows] - S[rows] @ x1
    assert np.abs(res).max() <= 1e-11 * np.abs(rhs[rows]).max()
    untouched = np.setdiff1d(np.arange(S.shape[1]), np.fromiter(used, int))
    assert np.array_equal(x1[untouched], x0[untouched])
    A = S[rows].toarray().conj().T
    coef = np.linalg.lstsq(A, x1 - x0, rcond=None)[0]
    assert np.linalg.norm(A @ coef - (x1 - x0)) <= 1e-12 * np.linalg.norm(x1 - x0)
    # overlapping rows: a box's rows in order, the last one projected exactly
    box = kz.box_partition(sysm, 2)
    rows_b = box.part_rows[box.part_ptr[0]:box.part_ptr[1]]
    one = kz.row_partition(S.shape[0], S.shape[1], [list(rows_b)])
    x2 = kz.kaczmarz_steps(S, one, rhs, x0, 1, 1.0)
    last = rows_b[-1]
    assert abs(rhs[last] - S[last] @ x2) <= 1e-11 * abs(rhs[last])
    assert np.abs(rhs[rows_b[:-1]] - S[rows_b[:-1]] @ x2).max() > 1e-6


@pytest.mark.parametrize("w", [1.0, 0.8, 1.3])
def test_bjorck_elfving_sor_identity(w):
    """One sub-region holding every row in order: from x = A^H y0, Kaczmarz sweeps are SOR sweeps
    on (A A^H) y = b with x = A^H y (Bjorck and Elfving 1979). Two sweeps from zero:
    (D + wL) y1 = w b;  (D + wL) y2 = w b - (w U + (w - 1) D) y1."""
    sysm, _, _ = _system((8, 6))
    S = sysm.S.tocsr()
    rng = np.random.default_rng(7)
    b = _crand(rng, S.shape[0])
    M = (S @ S.conj().T).tocsr()
    D = sp.diags(M.diagonal())
    L = sp.tril(M, k=-1)
    U = sp.triu(M, k=1)
    lower = (D + w * L).tocsr()
    y1 = spla.spsolve_triangular(lower, w * b, lower=True)
    y2 = spla.spsolve_triangular(lower, w * b - (w * U + (w - 1.0) * D) @ y1, lower=True)
    part = kz.row_partition(S.shape[0], S.shape[1], [list(range(S.shape[0]))])
    x1 = kz.kaczmarz_steps(S, part, b, np.zeros(S.shape[1], complex), 1, w)
    x2 = kz.kaczmarz_steps(S, part, b, np.zeros(S.shape[1], complex), 2, w)
    ref1 = S.conj().T @ y1
    ref2 = S.conj().T @ y2
    assert np.linalg.norm(x1 - ref1) <= 1e-11 * np.linalg.norm(ref1)
    assert np.linalg.norm(x2 - ref2) <= 1e-11 * np.linalg.norm(ref2)


# ---------------------------------------------------------------- the parallel step
@pytest.mark.parametrize("n,box", [((10, 8), 2), ((10, 8), 3), ((6, 5, 4), 2)])
def test_exact_solution_is_a_fixed_point(n, box):
    """Every row has zero residual at the solution, so every copy keeps it and every mean equals
    it, whatever the partition and damping."""
    sysm, b, _ = _system(n)
    f = sysm.reduce(b)
    u = spla.spsolve(sysm.S.tocsc(), f)
    part = kz.box_partition(sysm, box)
    for w in (0.8, 1.5):
        x = kz.kaczmarz_steps(sysm.S, part, f, u, 1, w)
        assert np.linalg.norm(x - u) <= 1e-10 * np.linalg.norm(u)


@pytest.mark.parametrize("n,box", [((10, 8), 2), ((12, 10), 4), ((6, 5, 4), 2)])
def test_error_decreases_monotonically(n, box):
    """Component-averaged row projections with 0 < w < 2 never increase the distance to the
    solution of a consistent system (Gordon and Gordon 2005: a Kaczmarz method in a superspace)."""
    sysm, b, _ = _system(n)
    f = sysm.reduce(b)
    u = spla.spsolve(sysm.S.tocsc(), f)
    part = kz.box_partition(sysm, box)
    for w in (0.8, 1.6):
        x = np.zeros_like(u)
        prev = np.linalg.norm(x - u)
        for _ in range(8):
            x = kz.kaczmarz_steps(sysm.S, part, f, x, 1, w)
            err = np.linalg.norm(x - u)
            assert err <= prev * (1 + 1e-12)
            prev = err
        assert prev < 0.999 * np.linalg.norm(u)


@pytest.mark.parametrize("n", [(10, 8), (6, 5, 4)])
def test_reach_is_the_schur_stencil_footprint(n):
    """Every nonzero of S at (row comp c, cell k; column comp c', cell k') has k' - k within the
    reach offsets of c' (low: 1 along x_c', 2 along the other axes; high: 1), and the bounds are
    attained, so single-cell boxes never step outside their reach and the reach is no larger than
    needed."""
    sysm, _, pb = _system(n)
    d, N = pb.dim, pb.ncell
    S = sysm.S.tocoo()
    full_r, full_c = sysm.u_act[S.row], sysm.u_act[S.col]
    cr, kr = np.divmod(full_r, N)
    cc, kc = np.divmod(full_c, N)

    def coords(k):
        out = []
        for a in range(d):
            out.append(k % pb.n[a])
            k = k // pb.n[a]
        return out

    pr, pc = coords(kr), coords(kc)
    for c2 in range(d):
        low, high = kz.reach_offsets(d, c2)
        sel = cc == c2
        for a in range(d):
            off = pc[a][sel] - pr[a][sel]
            assert off.min() == -low[a] and off.max() == high[a]
    part = kz.box_partition(sysm, 1)
    kz.kaczmarz_steps(sysm.S, part, np.ones(sysm.S.shape[0], complex), np.zeros(sysm.S.shape[1], complex), 1, 1.0)


def test_partition_covers_every_row_once():
    sysm, _, _ = _system((9, 7, 5))
    for box in (2, 3, (4, 2, 3)):
        part = kz.box_partition(sysm, box)
        assert np.array_equal(np.sort(part.part_rows), np.arange(sysm.S.shape[0]))
        for p in range(part.nparts):
            reach = part.reach_cols[part.reach_ptr[p]:part.reach_ptr[p + 1]]
            assert np.unique(reach).size == reach.size
    col = kz.box_partition(sysm, 4, coloured=True)
    assert col.nparts == 1 and np.array_equal(np.sort(col.part_rows), np.arange(sysm.S.shape[0]))


@pytest.mark.parametrize("n", [(16, 12), (9, 8, 8)])
def test_same_coloured_boxes_commute(n):
    """With boxes of 4 cells, the rows of two boxes of the same colour touch disjoint unknowns, so
    the coloured sweep does not depend on the order of the boxes within a colour (what lets a GPU
    sweep them at once)."""
    sysm, b, _ = _system(n)
    S = sysm.S.tocsr()
    part = kz.box_partition(sysm, 4, coloured=True)
    boxes = kz.box_partition(sysm, 4)
    d = len(n)
    shape = [-(-n[a] // 4) for a in range(d)]
    colour = []
    for p in range(boxes.nparts):
        bi, rem = [], p
        for a in range(d):
            bi.append(rem % shape[a])
            rem //= shape[a]
        colour.append(sum((bi[a] % 2) << a for a in range(d)))
    rows_of = [boxes.part_rows[boxes.part_ptr[p]:boxes.part_ptr[p + 1]] for p in range(boxes.nparts)]
    for c in range(2 ** d):
        members = [p for p in range(boxes.nparts) if colour[p] == c]
        supports = [set(S[rows_of[p]].indices) for p in members]
        for i in range(len(members)):
            for j in range(i + 1, len(members)):
                assert not supports[i] & supports[j]
    rev = np.concatenate([rows_of[p] for c in range(2 ** d)
                          for p in reversed([q for q in range(boxes.nparts) if colour[q] == c])])
    perm = kz.Partition([0, rev.size], rev, part.reach_ptr, part.reach_cols, 4, True)
    f = sysm.reduce(b)
    x0 = np.zeros(S.shape[1], complex)
    xa = kz.kaczmarz_steps(S, part, f, x0, 2, 0.8)
    xb = kz.kaczmarz_steps(S, perm, f, x0, 2, 0.8)
    assert np.linalg.norm(xa - xb) <= 1e-13 * np.linalg.norm(xa)


# ---------------------------------------------------------------- the hybrid solve
def test_hybrid_solve_reaches_the_drop_and_is_consistent():
    """FGMRES(5) + 10 Kaczmarz steps at 0.8 stops at a 0.1 drop of the Schur residual; the full
    residual of the recovered (u, p) has that same norm on the displacement rows and zero on the
    continuity rows."""
    sysm, b, pb = _system((8, 8, 6))
    part = kz.box_partition(sysm, 2)
    x, its, rel = kz.hybrid_solve(sysm, part, b)
    assert rel <= 0.1 and 1 <= its <= 25
    H = oracle.assemble(pb, 0.4)
    r = b - H @ x
    f = sysm.reduce(b)
    assert abs(np.linalg.norm(r[sysm.u_act]) / np.linalg.norm(f) - rel) <= 1e-10
    assert np.abs(r[sysm.nu:]).max() <= 1e-12 * np.abs(b).max()
    # tighter tolerance: the 250-step cap (25 preconditioner applications) ends the solve
    x, its, rel = kz.hybrid_solve(sysm, part, b, tol=1e-14)
    assert its == 25 and rel > 1e-14


def test_hierarchy_kaczmarz_coarsest_matches_the_hybrid_solve():
    """Multigrid's coarsest level in "kaczmarz" mode is exactly the hybrid solve on the coarsest
    re-discretisation, and a V-cycle with it reduces the residual."""
    w = small_heterogeneous((16, 16, 8), levels=2)
    pb = _problem(w)
    hier = oracle.Hierarchy(pb, 2, 0.4, damping=0.5, coarse="kaczmarz", coarse_box=2)
    rng = np.random.default_rng(11)
    bc = _crand(rng, hier.H[1].shape[0]) * oracle.active_mask(hier.pbs[1])
    ref, _, _ = kz.hybrid_solve(kz.SchurSystem(hier.pbs[1], 0.4), kz.box_partition(kz.SchurSystem(hier.pbs[1], 0.4), 2),
                                bc)
    got = hier.coarse_solve(bc)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    b = w.rhs.ravel() * oracle.active_mask(pb)
    x = oracle.vcycle(hier, b)
    r1 = np.linalg.norm(b - hier.H[0] @ x) / np.linalg.norm(b)
    assert r1 < 0.9
