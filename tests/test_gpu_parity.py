"""GPU vs oracle parity for every row of the cycle, in FP64 and FP32, 2D and 3D.

Sizes span several thread tiles with ragged tails; the oracle runs in seconds on them. Tolerances:
FP64 kernels 1e-12 (max-norm relative), FP64 cycle 1e-11; FP32 kernels 2e-6, FP32 cycle 1e-5
(2-norm relative), i.e. a few FP32 roundings amplified by the stencil's cancellation."""
import numpy as np
import pytest

import oracle
from oracle.smoother import cell_colour
from workloads import small_heterogeneous
from _gpu_helpers import (oracle_problem, oracle_hierarchy, gpu_solver, random_field, to_gpu, to_np, rel, rel_max,
                          TOL, TOL_CYCLE)

pytestmark = pytest.mark.gpu

CASES = {
    "2d": dict(n=(72, 40), levels=3, abl_cells=5),
    "2d_odd_coarse": dict(n=(36, 20), levels=3, abl_cells=3),
    "3d": dict(n=(40, 12, 8), levels=2, abl_cells=2),
}


def _w(case, seed=1):
    c = CASES[case]
    return small_heterogeneous(c["n"], seed=seed, levels=c["levels"], abl_cells=c["abl_cells"], sigma_cells=2.0)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("shifted", [False, True])
def test_apply_fp64_matches_oracle(case, shifted):
    w = _w(case)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    x = random_field(pb, 11)
    y_ref = oracle.apply(pb, x, shift=w.alpha if shifted else 0.0)
    import torch
    xt = to_gpu(x, 64)
    yt = torch.empty_like(xt)
    s.apply(xt, yt, shifted=shifted)
    assert rel_max(to_np(yt), y_ref) < TOL[64]
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("level", [0, 1])
def test_red_black_vanka_matches_oracle(case, prec, sweeps, level):
    # level 0 runs one launch per half-sweep; the small coarse levels of these cases run all
    # half-sweeps in one cooperative launch (2D)
    w = _w(case)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    pl = hier.pbs[level]
    b = random_field(pl, 21)
    x = random_field(pl, 22)
    ref = x.ravel()
    for _ in range(sweeps):
        ref = oracle.red_black_sweep(hier.H[level], hier.V[level], hier.idx[level], hier.colour[level], b.ravel(), ref,
                                     hier.w[level])
    xt = to_gpu(x, prec)
    s.smooth(level, to_gpu(b, prec), xt, sweeps)
    tol = TOL[prec] * (10 if prec == 64 else 5)
    assert rel_max(to_np(xt), ref) < tol
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("level", [0, 1])
def test_economic_vanka_matches_oracle(case, prec, level):
    """Economic Vanka (the displacement part of each cell block replaced by its diagonal,
    Sec. 2.3) in the red-black order of the full smoother."""
    w = _w(case)
    w.smoother = "economic"
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    pl = hier.pbs[level]
    b = random_field(pl, 23)
    x = random_field(pl, 24)
    ref = x.ravel()
    for _ in range(2):
        ref = oracle.red_black_sweep(hier.H[level], hier.V[level], hier.idx[level], hier.colour[level], b.ravel(), ref,
                                     hier.w[level])
    xt = to_gpu(x, prec)
    s.smooth(level, to_gpu(b, prec), xt, 2)
    assert rel_max(to_np(xt), ref) < TOL[prec] * (10 if prec == 64 else 5)
    # and a whole cycle
    bb = random_field(pb, 25)
    ref_c = oracle.vcycle(hier, bb.ravel())
    import torch
    xc = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    s.vcycle(to_gpu(bb, prec), xc, zero_guess=True)
    assert rel(to_np(xc).ravel() * oracle.active_mask(pb), ref_c) < TOL_CYCLE[prec]
    s.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_cooperative_sweeps_match_per_launch_sweeps(prec):
    """Level 1 of a 1024x800 grid whose material is constant on 2x2 blocks is, cell for cell, the
    level 0 of a 512x400 grid with twice the spacing (same physical absorbing layer, shift and
    damping). Its sweeps run in one cooperative launch whose threads each take several cells
    (102 400 cells per colour); the 512x400 level 0 runs one launch per half-sweep, the path
    the oracle parity tests pin."""
    from paper_2307_03242_gb300 import emg
    import torch
    rng = np.random.default_rng(7)
    nb = (512, 400)
    shape_b = (nb[1], nb[0])
    mu_b = rng.uniform(0.5, 2.0, shape_b)
    rho_b = rng.uniform(0.8, 1.5, shape_b)
    lam_b = mu_b * rng.uniform(1.0, 2.0, shape_b)
    up = lambda a: np.repeat(np.repeat(a, 2, axis=0), 2, axis=1)
    common = dict(omega=0.3, gamma=0.01, alpha=0.5, beta=2.0 / 3.0, abl_gamma_max=2.0, damping=[0.3, 0.3],
                  cycle_precision=prec, coarse_solver=emg.COARSE_SMOOTH, coarse_sweeps=2)
    sa = emg.Solver(emg.Params(n=(2 * nb[0], 2 * nb[1]), h=1.0, abl_cells=12, levels=2, **common),
                    up(lam_b), up(mu_b), up(rho_b))
    sb = emg.Solver(emg.Params(n=nb, h=2.0, abl_cells=6, levels=1, **common), lam_b, mu_b, rho_b)
    assert sa.vec_shape(1) == sb.vec_shape(0)
    dt = sa.cdtype
    g = torch.Generator(device="cuda").manual_seed(3)
    b = torch.randn(sb.vec_shape(0), dtype=dt, device="cuda", generator=g)
    x0 = torch.randn(sb.vec_shape(0), dtype=dt, device="cuda", generator=g)
    x0[0, :, 0] = 0  # faces on the boundary are not unknowns
    x0[1, 0, :] = 0
    for sweeps in (1, 2):
        xa, xb = x0.clone(), x0.clone()
        sa.smooth(1, b, xa, sweeps)
        sb.smooth(0, b, xb, sweeps)
        assert rel_max(to_np(xa), to_np(xb)) < TOL[prec]
    sa.close()
    sb.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_residual_restriction_matches_oracle(case, prec):
    w = _w(case)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    b = random_field(pb, 31)
    x = random_field(pb, 32)
    ref = hier.R[0] @ (b.ravel() - hier.H[0] @ x.ravel())
    import torch
    bc = torch.zeros(s.vec_shape(1), dtype=s.cdtype, device="cuda")
    s.residual_restrict(0, to_gpu(b, prec), to_gpu(x, prec), bc)
    assert rel_max(to_np(bc), ref) < TOL[prec] * 10
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_prolongation_correction_matches_oracle(case, prec):
    w = _w(case)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    e = random_field(hier.pbs[1], 41)
    x = random_field(pb, 42)
    ref = x.ravel() + hier.P[0] @ e.ravel()
    xt = to_gpu(x, prec)
    s.prolong_correct(0, to_gpu(e, prec), xt)
    assert rel_max(to_np(xt), ref) < TOL[prec]
    s.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("coarse", ["dense", "smooth"])
def test_coarsest_solve_matches_oracle(case, prec, coarse):
    w = _w(case)
    w.coarse, w.coarse_sweeps, w.coarse_damping = coarse, 3, 0.8
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    last = w.levels - 1
    b = random_field(hier.pbs[last], 51)
    ref = hier.coarse_solve(b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(last), dtype=s.cdtype, device="cuda")
    s.coarse_solve(to_gpu(b, prec), xt)
    assert rel(to_np(xt), ref) < TOL_CYCLE[prec] * 10
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("coarse", ["dense", "smooth"])
def test_vcycle_matches_oracle(case, prec, coarse):
    w = _w(case)
    w.coarse, w.coarse_sweeps, w.coarse_damping = coarse, 4, 0.8
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    b = random_field(pb, 61)
    ref = oracle.vcycle(hier, b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    xt.fill_(3.0)  # ignored with a zero initial guess
    s.vcycle(to_gpu(b, prec), xt, zero_guess=True)
    got = to_np(xt).ravel() * oracle.active_mask(pb)
    assert rel(got, ref) < TOL_CYCLE[prec]
    # non-zero initial guess path
    x0 = random_field(pb, 62)
    ref2 = oracle.vcycle(hier, b.ravel(), x0.ravel())
    xt2 = to_gpu(x0, prec)
    s.vcycle(to_gpu(b, prec), xt2, zero_guess=False)
    assert rel(to_np(xt2), ref2) < TOL_CYCLE[prec]
    s.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("cycle", ["W", "K"])
def test_wcycle_and_kcycle_match_oracle(case, prec, cycle):
    """W-cycle (two recursive calls) and K-cycle (the two calls precondition two GCR steps of the
    coarse problem), Sec. 2.2, with a smoothed coarsest level."""
    c = dict(CASES[case])
    w = small_heterogeneous(c["n"], seed=5, levels=3, abl_cells=c["abl_cells"], sigma_cells=2.0)
    w.cycle, w.coarse, w.coarse_sweeps, w.coarse_damping = cycle, "smooth", 3, 0.8
    w.alpha_coarsest = 1.1  # per-level shift on the coarsest level
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    b = random_field(pb, 63)
    ref = oracle.vcycle(hier, b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    s.vcycle(to_gpu(b, prec), xt, zero_guess=True)
    assert rel(to_np(xt).ravel() * oracle.active_mask(pb), ref) < TOL_CYCLE[prec]
    s.close()


@pytest.mark.parametrize("case", ["2d", "2d_odd_coarse"])
@pytest.mark.parametrize("prec", [64, 32])
def test_per_level_damping_matches_oracle(case, prec):
    """A different damping on every level (the coarsest level keeps its own): a W-cycle whose
    levels each read their own entry."""
    w = _w(case)
    w.coarse, w.coarse_sweeps, w.coarse_damping, w.cycle = "smooth", 3, 0.8, "W"
    w.damping = [0.6, 0.35, 0.2][:w.levels]
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, prec)
    b = random_field(pb, 67)
    ref = oracle.vcycle(hier, b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    s.vcycle(to_gpu(b, prec), xt, zero_guess=True)
    assert rel(to_np(xt).ravel() * oracle.active_mask(pb), ref) < TOL_CYCLE[prec]
    # the same cycle with one damping everywhere differs: the entries are not all read from one slot
    hier1 = oracle_hierarchy(w, pb, damping=w.damping[0])
    assert rel(oracle.vcycle(hier1, b.ravel()), ref) > 100 * TOL_CYCLE[32]
    s.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_vcycle_is_deterministic(case):
    w = _w(case)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    import torch
    bt = to_gpu(random_field(pb, 71), 32)
    x1 = torch.zeros_like(bt)
    x2 = torch.zeros_like(bt)
    s.vcycle(bt, x1)
    s.vcycle(bt, x2)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    s.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("prec", [64, 32])
def test_fgmres_solve_matches_oracle(case, prec):
    """Outer FGMRES(20) in FP64 around the V-cycle: same iteration count as the oracle (FP64
    cycle: +-1; FP32 cycle: within 10%), true FP64 residual <= tol, solution within 1e-5 of the
    oracle's FP64 solution solved to 1e-10."""
    w = _w(case)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    H = oracle.assemble(pb, 0.0)
    b = w.rhs.ravel() * oracle.active_mask(pb)
    x_ref, its_ref, _ = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-6, restart=20,
                                      max_iter=500)
    x_tight, _, _ = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b, tol=1e-10, restart=20,
                                  max_iter=500)
    s = gpu_solver(w, prec)
    import torch
    bt = to_gpu(b.reshape(oracle.dof_shape(pb)), 64)
    xt = torch.zeros_like(bt)
    st = s.solve(bt, xt, tol=1e-6, max_iter=500, restart=20)
    x = to_np(xt).ravel()
    assert st["converged"]
    true_res = np.linalg.norm(b - H @ x) / np.linalg.norm(b)
    assert true_res <= 1e-6 and abs(true_res - st["rel_residual"]) < 1e-9
    if prec == 64:
        assert abs(st["iterations"] - its_ref) <= 1
    else:
        assert abs(st["iterations"] - its_ref) <= max(1, int(0.1 * its_ref))
    xt2 = torch.zeros_like(bt)
    st2 = s.solve(bt, xt2, tol=1e-10, max_iter=800, restart=20)
    assert rel(to_np(xt2), x_tight) < 1e-5 * (1 if prec == 64 else 10) and st2["converged"]
    s.close()


def test_solve_host_buffers_match_device_solve():
    w = _w("2d")
    pb = oracle_problem(w)
    b = (w.rhs.ravel() * oracle.active_mask(pb)).astype(np.complex128)
    s = gpu_solver(w, 32)
    import torch
    bt = to_gpu(b.reshape(oracle.dof_shape(pb)), 64)
    xt = torch.zeros_like(bt)
    st = s.solve(bt, xt, tol=1e-6)
    xh = np.zeros_like(b)
    sh = s.solve_host(b, xh, tol=1e-6)
    assert st["iterations"] == sh["iterations"]
    np.testing.assert_array_equal(xh, to_np(xt).ravel())
    s.close()


def test_solve_edge_cases():
    """Zero right-hand side (x = 0 at once, 0 iterations); max_iter = 0 (the initial guess comes
    back untouched, EMG_NOT_CONVERGED with its true residual); a non-zero initial guess reaches
    the same solution as a zero one."""
    import torch
    w = _w("2d")
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    act = oracle.active_mask(pb)
    zero = torch.zeros(s.vec_shape(0), dtype=torch.complex128, device="cuda")
    x = to_gpu(random_field(pb, 81), 64)
    st = s.solve(zero, x, tol=1e-6, max_iter=50, restart=5)
    assert st["converged"] and st["iterations"] == 0 and st["rel_residual"] == 0.0
    assert torch.count_nonzero(x) == 0
    b = w.rhs.ravel() * act
    bt = to_gpu(b.reshape(oracle.dof_shape(pb)), 64)
    x0 = to_gpu(random_field(pb, 82), 64)
    x1 = x0.clone()
    st = s.solve(bt, x1, tol=1e-6, max_iter=0, restart=5)
    assert not st["converged"] and st["iterations"] == 0
    assert torch.equal(x1, x0)
    H = oracle.assemble(pb, 0.0)
    r_true = np.linalg.norm(b - H @ to_np(x0).ravel()) / np.linalg.norm(b)
    assert abs(st["rel_residual"] - r_true) < 1e-10 * r_true
    xa = torch.zeros_like(bt)
    s.solve(bt, xa, tol=1e-10, max_iter=500, restart=5)
    xb = x0.clone()
    s.solve(bt, xb, tol=1e-10, max_iter=500, restart=5)
    assert rel(to_np(xb), to_np(xa)) < 1e-7
    s.close()


def test_single_level_hierarchy_is_an_exact_preconditioner():
    """levels = 1 with the dense coarsest solve: the preconditioner is H_s^{-1} itself; with no
    shift (alpha on the only level = the physical attenuation only, via a tiny alpha) FGMRES
    converges in a couple of iterations (FP32 inverse, FP64 outer)."""
    import torch
    w = small_heterogeneous((16, 12), seed=4, levels=1, abl_cells=2, sigma_cells=2.0)
    w.alpha = 1e-12
    pb = oracle_problem(w)
    s = gpu_solver(w, 64)
    b = w.rhs.ravel() * oracle.active_mask(pb)
    bt = to_gpu(b.reshape(oracle.dof_shape(pb)), 64)
    xt = torch.zeros_like(bt)
    st = s.solve(bt, xt, tol=1e-10, max_iter=10, restart=5)
    assert st["converged"] and st["iterations"] <= 2
    s.close()
