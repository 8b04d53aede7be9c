"""Every sweep path of 2D FP32 levels against the oracle: one launch per colour (half), all
sweeps in one cooperative launch (coop), and the one-pass shared-memory tiled sweep with tiles of
60 x 24, 60 x 8 and 60 x 4 cells (tile24, tile8, tile4), forced on every level; and the autotuned
choice.

The grids reach several tiles in each direction with a ragged last tile (200 x 72: four tile
columns, the last 20 cells wide), tiles inside the absorbing layer, on the boundary and, for the
finest level, interior tiles without attenuation (the specialised variant). Tolerances as in
test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from workloads import small_heterogeneous
from _gpu_helpers import oracle_problem, oracle_hierarchy, gpu_solver, random_field, to_gpu, to_np, rel, rel_max, \
    TOL, TOL_CYCLE

pytestmark = pytest.mark.gpu

PATHS = {"half": 1, "coop": 2, "tile24": 3, "tile8": 4, "tile4": 5}


def _w(n=(200, 72), levels=3, abl=5):
    w = small_heterogeneous(n, seed=4, levels=levels, abl_cells=abl, sigma_cells=2.0)
    w.cycle, w.nu_pre, w.nu_post = "W", 1, 1
    w.coarse, w.coarse_sweeps, w.coarse_damping = "smooth", 2, 0.8
    return w


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("level", [0, 1, 2])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_forced_sweep_path_matches_the_oracle(path, level, sweeps):
    w = _w()
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, 32, sweep_path=PATHS[path])
    got_path, _ = s.sweep_path(level)
    n0 = hier.pbs[level].n[0]
    if path.startswith("tile") and n0 % 4:
        assert got_path != PATHS[path]  # the tiled kernel needs n_x divisible by 4
    else:
        assert got_path == PATHS[path]
    pl = hier.pbs[level]
    b, x = random_field(pl, 71 + level), random_field(pl, 81 + sweeps)
    ref = x.ravel()
    for _ in range(sweeps):
        ref = oracle.red_black_sweep(hier.H[level], hier.V[level], hier.idx[level], hier.colour[level], b.ravel(), ref,
                                     hier.w[level])
    xt = to_gpu(x, 32)
    s.smooth(level, to_gpu(b, 32), xt, sweeps)
    assert rel_max(to_np(xt), ref) < 5 * TOL[32]
    s.close()


@pytest.mark.parametrize("path", list(PATHS) + ["auto"])
def test_wcycle_along_each_path_matches_the_oracle(path):
    """W(1,1) with two inexact coarsest sweeps: the tiled post-sweeps add the prolonged coarse
    correction while loading their tiles."""
    w = _w()
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    s = gpu_solver(w, 32, sweep_path=PATHS.get(path, 0))
    b = random_field(pb, 91)
    ref = oracle.vcycle(hier, b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    s.vcycle(to_gpu(b, 32), xt, zero_guess=True)
    assert rel(to_np(xt).ravel() * oracle.active_mask(pb), ref) < TOL_CYCLE[32]
    x0 = random_field(pb, 92)
    ref2 = oracle.vcycle(hier, b.ravel(), x0.ravel())
    xt2 = to_gpu(x0, 32)
    s.vcycle(to_gpu(b, 32), xt2, zero_guess=False)
    assert rel(to_np(xt2), ref2) < TOL_CYCLE[32]
    s.close()


def test_autotuner_reports_a_timed_choice_per_level():
    w = _w((2048, 512), levels=5, abl=20)
    s = gpu_solver(w, 32)
    for l in range(5):
        p, us = s.sweep_path(l)
        assert p in PATHS.values()
        assert us > 0
    # the same sizes tune once per process: a second handle reuses the choices
    s2 = gpu_solver(w, 32)
    assert [s2.sweep_path(l) for l in range(5)] == [s.sweep_path(l) for l in range(5)]
    s.close()
    s2.close()
