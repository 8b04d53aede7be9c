"""Parity at the full configuration sizes (2048^2 2D heterogeneous, 256^3 3D layered), in the
solver configuration bench.py times. The oracle cannot assemble these grids, so it checks
sampled windows: the operator rows, a red-black sweep and the residual restriction are local
(a half-sweep reaches 2 cells, a full sweep 4), so the oracle evaluated on a window with a
6-cell margin reproduces the interior of the window exactly. The full solve is checked by its
true FP64 residual and by the oracle's residual of the GPU solution on sampled windows."""
import numpy as np
import pytest

import oracle
from oracle.smoother import cell_dofs, cell_blocks, red_black_sweep
from workloads import config_c2_random2d, config_c3_layered3d
from _gpu_helpers import oracle_problem, gpu_solver, to_gpu, to_np, TOL

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
MARGIN = 6


@pytest.fixture(scope="module", params=["c2", "c3"])
def case(request):
    w = config_c2_random2d(2048) if request.param == "c2" else config_c3_layered3d(256)
    return request.param, w, oracle_problem(w)


def _windows(w):
    n = w.n
    d = len(n)
    size = 28 if d == 2 else 14
    starts = []
    # corners / edges / interior, each low corner with an even index sum (global red-black parity)
    for frac in ((0.0,) * d, (0.5,) * d, tuple(1.0 if a == 0 else 0.3 for a in range(d)), (1.0,) * d):
        lo = [int(min(max(0, round(f * (n[a] - size))), n[a] - size)) for a, f in enumerate(frac)]
        if sum(lo) % 2:
            lo[0] = lo[0] - 1 if lo[0] > 0 else lo[0] + 1
        starts.append(tuple(lo))
    return [(lo, tuple(lo[a] + size for a in range(d))) for lo in starts]


def _inner(w, lo, hi):
    """Slices (array order, leading component axis) of the window interior that is exact."""
    d = len(w.n)
    sl_local, sl_global = [], []
    for a in reversed(range(d)):
        s0 = 0 if lo[a] == 0 else MARGIN
        s1 = (hi[a] - lo[a]) - (0 if hi[a] == w.n[a] else MARGIN)
        sl_local.append(slice(s0, s1))
        sl_global.append(slice(lo[a] + s0, lo[a] + s1))
    return (slice(None),) + tuple(sl_local), (slice(None),) + tuple(sl_global)


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_fullsize_apply_fp64_on_sampled_windows(case):
    name, w, pb = case
    s = gpu_solver(w, 32)
    shape = oracle.dof_shape(pb)
    x = _rand(shape, 1)
    import torch
    xt = to_gpu(x, 64)
    yt = torch.empty_like(xt)
    s.apply(xt, yt, shifted=False)
    y = to_np(yt)
    for lo, hi in _windows(w):
        wp = oracle.window(pb, lo, hi)
        sl = tuple(slice(lo[a], hi[a]) for a in reversed(range(len(w.n))))
        yw = oracle.apply(wp, x[(slice(None),) + sl], shift=0.0)
        li, gi = _inner(w, lo, hi)
        ref = yw[li]
        assert np.abs(y[gi] - ref).max() <= 1e-12 * np.abs(ref).max(), (name, lo)
    s.close()


def test_fullsize_red_black_sweep_on_sampled_windows(case):
    name, w, pb = case
    s = gpu_solver(w, 32)
    shape = oracle.dof_shape(pb)
    b, x = _rand(shape, 2), _rand(shape, 3)
    xt = to_gpu(x, 32)
    s.smooth(0, to_gpu(b, 32), xt, 1)
    got = to_np(xt)
    alpha0 = w.level_alphas()[0]
    wdamp = s.params.damping if np.ndim(s.params.damping) == 0 else s.params.damping[0]
    for lo, hi in _windows(w):
        wp = oracle.window(pb, lo, hi)
        sl = (slice(None),) + tuple(slice(lo[a], hi[a]) for a in reversed(range(len(w.n))))
        H = oracle.assemble(wp, alpha0)
        idx = cell_dofs(wp)
        V = cell_blocks(H, idx)
        from oracle.smoother import cell_colour
        act = oracle.active_mask(wp)
        ref = red_black_sweep(H, V, idx, cell_colour(wp), b[sl].ravel() * act, x[sl].ravel() * act, wdamp)
        ref = ref.reshape(oracle.dof_shape(wp))
        li, gi = _inner(w, lo, hi)
        err = np.abs(got[gi] - ref[li]).max() / np.abs(ref[li]).max()
        assert err < 5 * TOL[32], (name, lo, err)
    s.close()


def test_fullsize_residual_restriction_on_sampled_windows(case):
    name, w, pb = case
    s = gpu_solver(w, 32)
    shape = oracle.dof_shape(pb)
    b, x = _rand(shape, 4), _rand(shape, 5)
    import torch
    bc = torch.zeros(s.vec_shape(1), dtype=torch.complex64, device="cuda")
    s.residual_restrict(0, to_gpu(b, 32), to_gpu(x, 32), bc)
    got = to_np(bc)
    alpha0 = w.level_alphas()[0]
    d = len(w.n)
    for lo, hi in _windows(w):
        lo2 = tuple(v - v % 2 for v in lo)
        hi2 = tuple(v - v % 2 for v in hi)
        wp = oracle.window(pb, lo2, hi2)
        cp = oracle.coarsen(wp)
        sl = (slice(None),) + tuple(slice(lo2[a], hi2[a]) for a in reversed(range(d)))
        act = oracle.active_mask(wp)
        r = (b[sl].ravel() - oracle.assemble(wp, alpha0) @ (x[sl].ravel() * act)) * act
        ref = (oracle.restriction(wp, cp) @ r).reshape(oracle.dof_shape(cp))
        sl_l, sl_g = [], []
        for a in reversed(range(d)):
            c0 = 0 if lo2[a] == 0 else MARGIN // 2
            c1 = (hi2[a] - lo2[a]) // 2 - (0 if hi2[a] == w.n[a] else MARGIN // 2)
            sl_l.append(slice(c0, c1))
            sl_g.append(slice(lo2[a] // 2 + c0, lo2[a] // 2 + c1))
        gl = (slice(None),) + tuple(sl_g)
        ll = (slice(None),) + tuple(sl_l)
        err = np.abs(got[gl] - ref[ll]).max() / np.abs(ref[ll]).max()
        assert err < 10 * TOL[32], (name, lo, err)
    s.close()


def test_fullsize_solve_reaches_tolerance_and_satisfies_the_oracle_rows(case):
    """FP32-cycle FGMRES(20) to 1e-6 in the bench configuration: the reported residual is the
    true FP64 residual, and on sampled windows the oracle's residual b - H x of the GPU solution
    equals the GPU's own residual (so x solves the oracle's equations to the stated tolerance)."""
    name, w, pb = case
    s = gpu_solver(w, 32)
    import torch
    bt = to_gpu(w.rhs, 64)
    xt = torch.zeros_like(bt)
    st = s.solve(bt, xt, tol=1e-6, max_iter=1500, restart=20)
    assert st["converged"] and st["rel_residual"] <= 1e-6, (name, st["iterations"], st["rel_residual"])
    rt = torch.empty_like(xt)
    s.apply(xt, rt, shifted=False)
    r_gpu = w.rhs - to_np(rt)
    x = to_np(xt)
    assert np.linalg.norm(r_gpu) / np.linalg.norm(w.rhs) <= 1.01e-6
    bmax = np.abs(w.rhs).max()
    for lo, hi in _windows(w):
        wp = oracle.window(pb, lo, hi)
        sl = (slice(None),) + tuple(slice(lo[a], hi[a]) for a in reversed(range(len(w.n))))
        rw = w.rhs[sl] - oracle.apply(wp, x[sl], shift=0.0)
        li, gi = _inner(w, lo, hi)
        assert np.abs(rw[li] - r_gpu[gi]).max() <= 1e-10 * bmax, (name, lo)
    s.close()
