"""The oracle's adjoint-state misfit gradient (oracle/adjoint.py) against central finite
differences of the misfit, each misfit evaluated with direct solves in FP64.

What it catches: a wrong sign or conjugation in the gradient formula, a missing term (the
continuity row's 1/(lambda+mu), the node average of mu, the face average of rho, the absorbing
layer inside the mass), an averaging transpose that misplaces cells at the clamped boundary."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import (average_matrix, material_derivative, misfit, misfit_and_gradient, receiver_dofs,
                            synthetic_data, DirectSolver)
from oracle.discretization import _avg_cells, replace
from workloads import small_heterogeneous, point_source
from _gpu_helpers import oracle_problem


@pytest.mark.parametrize("n", [(7, 5), (5, 4, 3)])
@pytest.mark.parametrize("periodic", [False, True])
def test_average_matrix_equals_the_cell_average(n, periodic):
    w = small_heterogeneous(n, seed=3, abl_cells=1)
    pb = replace(oracle_problem(w), periodic=periodic)
    d = len(n)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(tuple(n[::-1]))
    for axes in [(0,), (d - 1,), (0, 1), (1, d - 1)]:
        counts = list(n)
        if not periodic:
            for a in axes[1:]:
                counts[a] += 1
        A = average_matrix(pb, axes, counts)
        # the same average up to the order of the additions
        assert np.allclose(A @ f.ravel(), _avg_cells(f, pb, axes, counts).ravel(), rtol=0, atol=1e-15)


def _setup(n, nsrc, seed):
    w = small_heterogeneous(n, seed=seed, abl_cells=2)
    pb = oracle_problem(w)
    d = len(n)
    rng = np.random.default_rng(seed)
    srcs = []
    for _ in range(nsrc):
        idx = tuple(int(rng.integers(1, v - 1)) for v in n[:-1]) + (1,)
        srcs.append(point_source(n, d - 1, idx).ravel())
    pos = [p for p in np.ndindex(*n[:-1])]
    rec = receiver_dofs(pb, d - 1, 1, pos)
    # data from a medium with a density and stiffness bump
    true = replace(pb, mu=pb.mu * (1 + 0.1 * rng.random(pb.mu.shape)), rho=pb.rho * (1 + 0.1 * rng.random(pb.rho.shape)))
    return pb, srcs, rec, synthetic_data(true, srcs, rec)


def _perturbed(pb, field, delta, eps):
    return replace(pb, **{field: getattr(pb, field) + eps * delta})


@pytest.mark.parametrize("n,nsrc", [((12, 10), 2), ((6, 5, 4), 1)])
@pytest.mark.parametrize("field", ["lam", "mu", "rho"])
def test_gradient_matches_central_differences_in_a_random_direction(n, nsrc, field):
    pb, srcs, rec, data = _setup(n, nsrc, seed=5)
    J, g = misfit_and_gradient(pb, srcs, rec, data)
    assert J > 0
    rng = np.random.default_rng(11)
    delta = rng.standard_normal(getattr(pb, field).shape) * getattr(pb, field)
    eps = 1e-5
    fd = (misfit(_perturbed(pb, field, delta, eps), srcs, rec, data)
          - misfit(_perturbed(pb, field, delta, -eps), srcs, rec, data)) / (2 * eps)
    an = float(np.sum(g[field] * delta))
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-30), (field, an, fd)


@pytest.mark.parametrize("field", ["lam", "mu", "rho"])
def test_gradient_matches_central_differences_cell_by_cell(field):
    """Single cells in a corner (clamped averages), on an edge inside the absorbing layer and in
    the interior."""
    n = (10, 8)
    pb, srcs, rec, data = _setup(n, 2, seed=8)
    _, g = misfit_and_gradient(pb, srcs, rec, data)
    for cell in [(0, 0), (9, 7), (0, 4), (5, 3), (6, 1)]:
        delta = np.zeros(getattr(pb, field).shape)
        delta[cell[::-1]] = getattr(pb, field)[cell[::-1]]
        eps = 1e-5
        fd = (misfit(_perturbed(pb, field, delta, eps), srcs, rec, data)
              - misfit(_perturbed(pb, field, delta, -eps), srcs, rec, data)) / (2 * eps)
        an = g[field][cell[::-1]] * delta[cell[::-1]]
        assert abs(an - fd) <= 1e-6 * np.abs(g[field] * getattr(pb, field)).max(), (field, cell, an, fd)


def test_adjoint_solve_is_the_conjugate_transpose_solve():
    w = small_heterogeneous((9, 7), seed=2, abl_cells=2)
    pb = oracle_problem(w)
    ds = DirectSolver(pb)
    act = oracle.active_mask(pb)
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    y = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    # <H^-1 x, y> = <x, H^-H y>
    assert abs(np.vdot(ds.solve(x), y) - np.vdot(x, ds.solve_adjoint(y))) <= 1e-12 * np.linalg.norm(x) * \
        np.linalg.norm(ds.solve_adjoint(y))


def test_derivative_is_linear_in_the_wavefield_and_conjugate_linear_in_the_adjoint():
    w = small_heterogeneous((6, 5), seed=4, abl_cells=1)
    pb = oracle_problem(w)
    act = oracle.active_mask(pb)
    rng = np.random.default_rng(6)
    u = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    a = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    g1 = material_derivative(pb, u, a)
    # scaling u by i and a by i leaves -Re(a^H dH u) unchanged; scaling u alone by i changes it
    g2 = material_derivative(pb, 1j * u, 1j * a)
    g3 = material_derivative(pb, 1j * u, a)
    for k in g1:
        assert np.allclose(g1[k], g2[k], rtol=1e-13, atol=1e-13 * np.abs(g1[k]).max())
        assert not np.allclose(g1[k], g3[k])


def test_gradient_points_towards_the_data_model_on_a_small_inversion_instance():
    """The 3D inversion setting at 8^3 (4 sources, 16 receivers): to first order in the model
    difference dm (data model minus current model) the receiver residual is r = F' dm, so the
    gradient satisfies -grad . dm = Re <r, F' dm> = |r|^2 = 2 J."""
    from workloads import config_c5_adjoint
    w = config_c5_adjoint(8, source_side=2, receiver_side=4, depth=2)
    pb = oracle_problem(w)
    rec = np.array([np.ravel_multi_index((c,) + tuple(idx[::-1]), oracle.dof_shape(pb)) for c, idx in w.extra["receivers"]])
    srcs = [q.ravel() for q in w.extra["sources"]]
    lam_t, mu_t, rho_t = w.extra["true"]
    data = synthetic_data(replace(pb, lam=lam_t, mu=mu_t, rho=rho_t), srcs, rec)
    J, g = misfit_and_gradient(pb, srcs, rec, data)
    assert J > 0
    descent = -(np.sum(g["lam"] * (lam_t - pb.lam)) + np.sum(g["mu"] * (mu_t - pb.mu))
                + np.sum(g["rho"] * (rho_t - pb.rho)))
    # first order: -grad . dm = |r|^2 = 2 J (measured 1.012 x 2J for a 5 % blob)
    assert abs(descent / (2 * J) - 1.0) < 0.05, (descent, J)


def test_conjugate_transpose_is_the_sign_conjugated_operator_at_beta_one():
    """H^H = S conj(H) S with S = diag(I, -I) when beta = 1 (any medium); with the beta-spread
    stencils the two differ, for a homogeneous medium only in the u-p coupling blocks. The GPU
    adjoint solve preconditions H^H with the forward cycle mapped through this relation."""
    import scipy.sparse as sp
    for beta in (1.0, 2.0 / 3.0):
        w = small_heterogeneous((8, 6), seed=5, abl_cells=2)
        pb = replace(oracle_problem(w), beta=beta)
        H = oracle.assemble(pb, 0.0)
        N, d = pb.ncell, pb.dim
        S = sp.diags(np.r_[np.ones(d * N), -np.ones(N)])
        D = (H.conj().T - S @ H.conj() @ S).tocsr()
        if beta == 1.0:
            assert abs(D).max() <= 1e-12 * abs(H).max()
        else:
            assert abs(D).max() > 1e-3 * abs(H).max()
    # homogeneous medium, beta = 2/3: the displacement block and the p-p block agree
    pb = replace(oracle_problem(w), beta=2.0 / 3.0, lam=np.full(w.lam.shape, 2.0), mu=np.ones(w.lam.shape),
                 rho=np.ones(w.lam.shape), abl_length=0.0)
    H = oracle.assemble(pb, 0.0)
    D = (H.conj().T - S @ H.conj() @ S).tocsr()
    uu = D[:d * N][:, :d * N]
    assert abs(uu).max() <= 1e-12 * abs(H).max() and abs(D[d * N:, d * N:]).max() == 0.0


@pytest.mark.parametrize("n,levels", [((24, 16), 2), ((8, 8, 8), 2)])
def test_mapped_forward_cycle_preconditions_the_adjoint_operator(n, levels):
    """FGMRES on H^H with the preconditioner S conj(M(conj(S r))), M the forward cycle, needs at
    most twice the iterations of the forward solve (measured 28 vs 21 in 2D, 14 vs 10 in 3D)."""
    from _gpu_helpers import oracle_hierarchy
    w = small_heterogeneous(n, seed=3, levels=levels, abl_cells=2, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    H = oracle.assemble(pb, 0.0)
    Hh = H.conj().T.tocsr()
    act = oracle.active_mask(pb)
    S = np.r_[np.ones(pb.dim * pb.ncell), -np.ones(pb.ncell)]
    rng = np.random.default_rng(4)
    b = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    M = lambda v: oracle.vcycle(hier, v)
    _, its, _ = oracle.fgmres(lambda v: H @ v, M, b, tol=1e-10, restart=20, max_iter=500)
    x, its_a, _ = oracle.fgmres(lambda v: Hh @ v, lambda r: S * np.conj(M(np.conj(S * r))), b, tol=1e-10,
                                restart=20, max_iter=500)
    assert np.linalg.norm(b - Hh @ x) <= 1e-9 * np.linalg.norm(b)
    assert its_a <= 2 * its, (its, its_a)
