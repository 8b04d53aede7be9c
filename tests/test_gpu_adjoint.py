"""GPU adjoint-state gradient against the FP64 oracle: y = H^H x, the per-cell material
derivative, the adjoint solve, and the misfit gradient through torch.autograd, including central
finite differences of the GPU misfit on a 32^3 instance with 2 sources."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import material_derivative, misfit_and_gradient, synthetic_data, DirectSolver
from oracle.discretization import replace
from workloads import small_heterogeneous, config_c5_adjoint
from _gpu_helpers import oracle_problem, gpu_solver, to_gpu, to_np, rel_max

pytestmark = pytest.mark.gpu

CASES = {"2d": ((24, 16), 2, 3), "3d": ((8, 8, 8), 2, 2)}  # n, levels, absorbing-layer cells


def _w(case, seed=3):
    n, levels, abl = CASES[case]
    return small_heterogeneous(n, seed=seed, levels=levels, abl_cells=abl, sigma_cells=2.0)


def _rand(pb, seed):
    act = oracle.active_mask(pb)
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act
    return v.reshape(oracle.dof_shape(pb))


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_apply_matches_the_oracle(case):
    import torch
    w = _w(case)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    x = _rand(pb, 1)
    ref = (oracle.assemble(pb, 0.0).conj().T @ x.ravel()).reshape(x.shape)
    xt = to_gpu(x, 64)
    yt = torch.empty_like(xt)
    s.apply_adjoint(xt, yt)
    assert rel_max(to_np(yt), ref) < 1e-12
    s.close()


@pytest.mark.slow
def test_adjoint_apply_at_128_cubed_on_sampled_windows():
    """H^H x of the 3D inversion setting (128^3, float-float on the forward apply's coefficients)
    on sampled windows: H^H is as local as H, so the oracle's conjugate transpose on a window
    with a 6-cell margin reproduces the window's interior rows."""
    import torch
    w = config_c5_adjoint(128)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    x = _rand(pb, 5)
    xt = to_gpu(x, 64)
    yt = torch.empty_like(xt)
    s.apply_adjoint(xt, yt)
    y = to_np(yt)
    size, margin = 16, 6
    ymax = np.abs(y).max()
    for lo in ((0, 0, 0), (56, 56, 56), (112, 40, 0), (112, 112, 112)):
        hi = tuple(l + size for l in lo)
        wp = oracle.window(pb, lo, hi)
        sl = (slice(None),) + tuple(slice(lo[a], hi[a]) for a in (2, 1, 0))
        xw = x[sl]
        yw = (oracle.assemble(wp, 0.0).conj().T @ xw.ravel()).reshape(xw.shape)
        inner = tuple(slice(0 if lo[a] == 0 else margin, size - (0 if hi[a] == 128 else margin)) for a in (2, 1, 0))
        glob = tuple(slice(lo[a] + inner[2 - a].start, lo[a] + inner[2 - a].stop) for a in (2, 1, 0))
        got = y[(slice(None),) + glob]
        ref = yw[(slice(None),) + inner]
        assert np.abs(got - ref).max() <= 1e-12 * ymax, lo
    s.close()


@pytest.mark.parametrize("case", list(CASES))
def test_material_gradient_kernel_matches_the_oracle(case):
    w = _w(case)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    u, a = _rand(pb, 2), _rand(pb, 3)
    ref = material_derivative(pb, u, a)
    g = s.material_gradient(to_gpu(u, 64), to_gpu(a, 64))
    for got, name in zip(g, ("lam", "mu", "rho")):
        assert rel_max(got.cpu().numpy(), ref[name]) < 1e-12, name
    # accumulate adds
    g2 = s.material_gradient(to_gpu(u, 64), to_gpu(a, 64), out=tuple(t.clone() for t in g), accumulate=True)
    for got, name in zip(g2, ("lam", "mu", "rho")):
        assert rel_max(got.cpu().numpy(), 2 * ref[name]) < 1e-12, name
    s.close()


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_solve_matches_the_oracle_direct_solve(case):
    import torch
    w = _w(case)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    b = _rand(pb, 4)
    ref = DirectSolver(pb).solve_adjoint(b.ravel()).reshape(b.shape)
    xt = torch.zeros(s.vec_shape(0), dtype=torch.complex128, device="cuda")
    st = s.solve_adjoint(to_gpu(b, 64), xt, tol=1e-10, max_iter=2000, restart=20)
    assert st["converged"] and st["rel_residual"] <= 1e-10, st
    assert np.linalg.norm(to_np(xt) - ref) <= 1e-7 * np.linalg.norm(ref)
    s.close()


def _inversion_instance(n, source_side, receiver_side):
    import torch
    w = config_c5_adjoint(n, source_side=source_side, receiver_side=receiver_side, depth=2)
    pb = oracle_problem(w)
    shape = oracle.dof_shape(pb)
    rec = np.array([np.ravel_multi_index((c,) + tuple(idx[::-1]), shape) for c, idx in w.extra["receivers"]])
    srcs = [q for q in w.extra["sources"]]
    lam_t, mu_t, rho_t = w.extra["true"]
    data = synthetic_data(replace(pb, lam=lam_t, mu=mu_t, rho=rho_t), [q.ravel() for q in srcs], rec)
    dev = "cuda"
    return w, pb, rec, srcs, data, dict(
        sources=[torch.from_numpy(q).to(dev) for q in srcs], receivers=torch.from_numpy(rec).to(dev),
        data=[torch.from_numpy(d).to(dev) for d in data])


@pytest.mark.parametrize("keep_fields", [True, False])
def test_misfit_gradient_through_autograd_matches_the_oracle(keep_fields):
    """keep_fields=False: the backward pass recomputes each forward field (and checks that the
    recomputing solve converged) instead of keeping it."""
    import torch
    from paper_2307_03242_gb300 import emg, inversion
    w, pb, rec, srcs, data, t = _inversion_instance(16, 2, 4)
    J_ref, g_ref = misfit_and_gradient(pb, [q.ravel() for q in srcs], rec, data)
    lam, mu, rho = (torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(True) for a in (w.lam, w.mu, w.rho))
    params = emg.params_from_workload(w, 32)
    # J is small (the data model differs from the current one by a 5 % blob), so the solves must
    # be tighter than J's tolerance: a 1e-12 residual leaves J within ~1e-9 of the direct solve
    J = inversion.misfit(lam, mu, rho, params, t["sources"], t["receivers"], t["data"], tol=1e-12,
                         keep_fields=keep_fields)
    J.backward()
    assert abs(J.item() - J_ref) <= 1e-8 * J_ref
    for got, name in zip((lam.grad, mu.grad, rho.grad), ("lam", "mu", "rho")):
        assert rel_max(got.cpu().numpy(), g_ref[name]) < 1e-6, name


def test_misfit_gradient_matches_central_differences_at_32_cubed():
    """The finite-difference check of the inversion setting: 32^3, 2 sources, 64 receivers, data
    from the +5 % blob model computed by the GPU solver, FP64 outer solves to 1e-11, one random
    direction per field."""
    import torch
    from paper_2307_03242_gb300 import emg, inversion
    w = config_c5_adjoint(32, source_side=2, receiver_side=8, depth=2)
    shape = (w.dim + 1,) + tuple(w.n[::-1])
    rec = torch.tensor([np.ravel_multi_index((c,) + tuple(idx[::-1]), shape) for c, idx in w.extra["receivers"]],
                       device="cuda")
    sources = [torch.from_numpy(q).cuda() for q in w.extra["sources"][:2]]
    params = emg.params_from_workload(w, 32)
    true = emg.Solver(params, *w.extra["true"])
    data = []
    for q in sources:
        u = torch.zeros_like(q)
        assert true.solve(q, u, tol=1e-11, max_iter=4000, restart=20)["converged"]
        data.append(u.reshape(-1)[rec].clone())
    true.close()
    base = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w.lam, w.mu, w.rho)]
    leaves = [b.clone().requires_grad_(True) for b in base]
    J = inversion.misfit(*leaves, params, sources, rec, data, tol=1e-11)
    J.backward()
    assert J.item() > 0
    rng = np.random.default_rng(9)
    for k, name in enumerate(("lam", "mu", "rho")):
        delta = torch.from_numpy(rng.standard_normal(w.lam.shape)).cuda() * base[k]
        eps = 1e-4

        def J_at(sgn):
            m = [b.clone() for b in base]
            m[k] = m[k] + sgn * eps * delta
            with torch.no_grad():
                return inversion.misfit(*m, params, sources, rec, data, tol=1e-11).item()

        fd = (J_at(1) - J_at(-1)) / (2 * eps)
        an = float(torch.sum(leaves[k].grad * delta))
        assert abs(an - fd) <= 1e-4 * abs(fd), (name, an, fd)
