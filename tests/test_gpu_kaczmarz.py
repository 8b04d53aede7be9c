"""GPU parity of the hybrid Kaczmarz-GMRES coarsest solve (EMG_COARSE_KACZMARZ; Sections 3.2 and
5.3) against the oracle (oracle/kaczmarz.py): the Schur rows the library forms by probing its
coarsest operator, the coarsest solve at a fixed iteration count and at the paper's 0.1 drop,
its determinism, a V-cycle that uses it, and a full 3D K-cycle solve with it."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import kaczmarz as kz
from workloads import small_heterogeneous
from _gpu_helpers import oracle_problem, random_field, to_gpu, to_np, rel

pytestmark = pytest.mark.gpu

# name -> (finest cells, levels, box)
CASES = {"3d_box2": ((16, 16, 12), 2, (2, 2, 2)), "3d_ragged": ((20, 16, 12), 2, (4, 3, 2)),
         "2d_box2": ((48, 40), 2, (2, 2)), "3d_three_levels": ((24, 24, 16), 3, (2, 2, 2)),
         "3d_box1": ((16, 12, 12), 2, (1, 1, 1)), "2d_box1": ((40, 36), 2, (1, 1))}


@pytest.fixture(scope="module")
def hc():
    from paper_2307_03242_gb300.build import build_hostcheck
    lib = ctypes.CDLL(build_hostcheck())
    lib.emg_hc_kz_steps.restype = ctypes.c_long
    return lib


def _setup(case, prec, **over):
    from paper_2307_03242_gb300 import emg
    n, levels, box = CASES[case]
    w = small_heterogeneous(n, seed=4, levels=levels, abl_cells=2, sigma_cells=2.0)
    pb = oracle_problem(w)
    alphas = [0.4] * levels
    hier = oracle.Hierarchy(pb, levels, alphas, damping=0.5, nu_pre=1, nu_post=1, coarse="kaczmarz",
                            coarse_box=box, coarse_tol=over.get("coarse_tol", 0.1),
                            coarse_max_kaczmarz=over.get("kaczmarz_max", 250))
    p = emg.Params(n=n, h=w.h, omega=w.omega, gamma=w.gamma, alpha=0.4, beta=w.beta, abl_cells=w.abl_cells,
                   abl_gamma_max=w.abl_gamma_max, levels=levels, nu_pre=1, nu_post=1, damping=0.5,
                   coarse_solver=emg.COARSE_KACZMARZ, cycle_precision=prec, kaczmarz_box=box, **over)
    s = emg.Solver(p, w.lam, w.mu, w.rho)
    return w, pb, hier, s


@pytest.mark.parametrize("case", ["3d_box2", "3d_ragged", "2d_box2", "3d_box1"])
@pytest.mark.parametrize("prec", [64, 32])
def test_probed_schur_rows_match_the_oracle(hc, case, prec):
    from test_host_kaczmarz import stored_rows
    _, _, hier, s = _setup(case, prec)
    last = hier.levels - 1
    ref = stored_rows(hc, kz.SchurSystem(hier.pbs[last], 0.4))
    got = s.coarse_schur_rows().astype(np.complex128)
    tol = 1e-12 if prec == 64 else 2e-6
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert np.array_equal(got != 0, ref != 0) or prec == 32
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_coarsest_solve_at_fixed_iterations_matches_the_oracle(case, prec):
    """30 Kaczmarz steps (3 FGMRES iterations, restart 5) with no early stop on both sides."""
    _, _, hier, s = _setup(case, prec, coarse_tol=1e-30, kaczmarz_max=30)
    last = hier.levels - 1
    b = random_field(hier.pbs[last], 71)
    ref = hier.coarse_solve(b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(last), dtype=s.cdtype, device="cuda")
    s.coarse_solve(to_gpu(b, prec), xt)
    its, relres, steps = s.coarse_stats()
    assert its == 3 and steps == 30
    assert rel(to_np(xt), ref) < (1e-10 if prec == 64 else 2e-4)
    sysm = hier.schur
    f = sysm.reduce(b.ravel())
    u = to_np(xt).ravel()[sysm.u_act]
    ref_rel = np.linalg.norm(f - sysm.S @ u) / np.linalg.norm(f)
    assert abs(relres - ref_rel) <= (1e-9 if prec == 64 else 1e-4) * max(ref_rel, 1e-3)
    s.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_coarsest_solve_reaches_the_paper_drop(case, prec):
    """Default settings (Sec. 5.3): FGMRES(5), 10 steps at 0.8, stop at a 0.1 drop of the Schur
    residual; the iteration count equals the oracle's and the drop holds for the returned (u, p)."""
    _, _, hier, s = _setup(case, prec)
    last = hier.levels - 1
    b = random_field(hier.pbs[last], 72)
    hist = []
    sysm = hier.schur
    ref, its_ref, _ = kz.hybrid_solve(sysm, hier.kpart, b.ravel(), history=hist)
    import torch
    xt = torch.zeros(s.vec_shape(last), dtype=s.cdtype, device="cuda")
    s.coarse_solve(to_gpu(b, prec), xt)
    its, relres, steps = s.coarse_stats()
    if prec == 64:
        assert its == its_ref
        assert rel(to_np(xt), ref) < 1e-9
    else:
        assert abs(its - its_ref) <= 1
    x = to_np(xt).ravel()
    f = sysm.reduce(b.ravel())
    got = np.linalg.norm(f - sysm.S @ x[sysm.u_act]) / np.linalg.norm(f)
    if its_ref < 25:
        assert got <= 0.1 * (1 + 1e-4)
    else:  # the oracle too spent the 250 Kaczmarz steps (1-cell boxes in 2D converge slowly)
        assert its == 25 and abs(got - relres) <= (1e-9 if prec == 64 else 1e-4)
    # the pressure is recovered exactly from u: the continuity rows of the full residual vanish
    r = b.ravel() - hier.H[last] @ x
    assert np.abs(r[sysm.nu:]).max() <= (1e-10 if prec == 64 else 1e-4) * np.abs(b).max()
    s.close()


def test_coarsest_solve_is_deterministic():
    _, _, hier, s = _setup("3d_box2", 32)
    last = hier.levels - 1
    import torch
    bt = to_gpu(random_field(hier.pbs[last], 73), 32)
    x1 = torch.zeros(s.vec_shape(last), dtype=s.cdtype, device="cuda")
    x2 = torch.zeros_like(x1)
    s.coarse_solve(bt, x1)
    s.coarse_solve(bt, x2)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    s.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_vcycle_with_kaczmarz_coarsest_matches_the_oracle(prec):
    _, pb, hier, s = _setup("3d_three_levels", prec, coarse_tol=1e-30, kaczmarz_max=20)
    b = random_field(pb, 74)
    ref = oracle.vcycle(hier, b.ravel())
    import torch
    xt = torch.zeros(s.vec_shape(0), dtype=s.cdtype, device="cuda")
    s.vcycle(to_gpu(b, prec), xt, zero_guess=True)
    assert rel(to_np(xt), ref) < (1e-10 if prec == 64 else 1e-4)
    s.close()


def test_k_cycle_solve_with_kaczmarz_coarsest_converges():
    """A 3D K(1,1)-cycle solve to 1e-6 with the Kaczmarz coarsest solve on 4 levels (coarsest 4^3
    scaled up: 32^3 finest, 4^3 coarsest), checked with the oracle's FP64 operator."""
    from paper_2307_03242_gb300 import emg
    import torch
    n = (32, 32, 32)
    w = small_heterogeneous(n, seed=8, levels=4, abl_cells=3, sigma_cells=4.0)
    pb = oracle_problem(w)
    p = emg.Params(n=n, h=w.h, omega=w.omega, gamma=w.gamma, alpha=0.4, beta=w.beta, abl_cells=w.abl_cells,
                   abl_gamma_max=w.abl_gamma_max, levels=4, nu_pre=1, nu_post=1, damping=0.3,
                   coarse_solver=emg.COARSE_KACZMARZ, cycle_precision=32, cycle_type=emg.CYCLE_K)
    s = emg.Solver(p, w.lam, w.mu, w.rho)
    b = w.rhs.ravel() * oracle.active_mask(pb)
    bt = torch.from_numpy(b.reshape(oracle.dof_shape(pb))).to("cuda")
    xt = torch.zeros_like(bt)
    st = s.solve(bt, xt, tol=1e-6, max_iter=400, restart=20)
    x = to_np(xt).ravel()
    res = np.linalg.norm(b - oracle.assemble(pb, 0.0) @ x) / np.linalg.norm(b)
    assert st["rel_residual"] <= 1e-6 and res <= 2e-6
    s.close()
