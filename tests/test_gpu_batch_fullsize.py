"""Instances of the 64-instance batch at the sizes it runs (256^2 and 1024^2), in the batch's
solver configuration (W(2,2) on 5 levels, two coarsest sweeps, FGMRES(5), FP32 cycle, the
autotuned sweep paths), solved through emg_solve_batch together with a second instance.

256^2: the solution against the oracle's sparse direct solve of its assembled operator.
1024^2 (too large for a direct solve): the reported residual is the true FP64 residual, and on
sampled windows the oracle's rows b - H x of the GPU solution equal the GPU's own residual."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from workloads import config_c4_batch
from _gpu_helpers import oracle_problem, to_gpu, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _instance(n):
    for w in config_c4_batch(64):
        if w.n[0] == n:
            return w
    raise AssertionError("no instance of size %d" % n)


def _batch(ws, tol):
    from paper_2307_03242_gb300 import emg
    import torch
    solvers = [emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=torch.cuda.Stream()) for w in ws]
    jobs = []
    for s, w in zip(solvers, ws):
        b = to_gpu(w.extra["sources"][0], 64)
        jobs.append((s, b, torch.zeros_like(b)))
    res = emg.solve_batch(jobs, tol=tol, max_iter=4000, restart=5)
    torch.cuda.synchronize()
    return solvers, jobs, res


def test_batch_instance_256_matches_the_oracle_direct_solve():
    w256, w1024 = _instance(256), _instance(1024)
    # solved further than the batch's 1e-6 so that the solution error is far below the tolerance
    solvers, jobs, res = _batch([w256, w1024], 1e-10)
    assert all(r["converged"] for r in res)
    pb = oracle_problem(w256)
    H = oracle.assemble(pb, 0.0)
    act = oracle.active_mask(pb)
    b = w256.extra["sources"][0].ravel()
    xd = np.zeros_like(b)
    xd[act] = spla.spsolve(H[act][:, act].tocsc(), b[act])
    x = to_np(jobs[0][2]).ravel()
    assert np.linalg.norm(H @ x - b) <= 1.01e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    for s in solvers:
        s.close()


def test_batch_instance_1024_satisfies_the_oracle_rows_on_windows():
    w1024, w256 = _instance(1024), _instance(256)
    solvers, jobs, res = _batch([w1024, w256], 1e-6)
    assert all(r["converged"] for r in res)
    s, bt, xt = jobs[0]
    import torch
    rt = torch.empty_like(xt)
    s.apply(xt, rt, shifted=False)
    b = w1024.extra["sources"][0]
    r_gpu = b - to_np(rt)
    assert np.linalg.norm(r_gpu) / np.linalg.norm(b) <= 1.01e-6
    pb = oracle_problem(w1024)
    x = to_np(xt)
    scale = np.abs(b).max()
    margin, size = 6, 28
    for lo in ((0, 0), (500, 500), (996, 300), (996, 996)):
        hi = (lo[0] + size, lo[1] + size)
        wp = oracle.window(pb, lo, hi)
        sl = (slice(None), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        rw = b[sl] - oracle.apply(wp, x[sl], shift=0.0)
        inner = tuple(slice(0 if lo[a] == 0 else margin, size - (0 if hi[a] == 1024 else margin)) for a in (1, 0))
        glob = tuple(slice(lo[a] + inner[1 - a].start, lo[a] + inner[1 - a].stop) for a in (1, 0))
        assert np.abs(rw[(slice(None),) + inner] - r_gpu[(slice(None),) + glob]).max() <= 1e-10 * scale, lo
    for s in solvers:
        s.close()
