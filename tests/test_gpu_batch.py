"""Concurrent batch of independent solves (emg_solve_batch): every job matches the same solve run
on its own, bit for bit, and the solutions match the oracle's; a failing job reports its own
status without disturbing the others."""
import numpy as np
import pytest

import oracle
from workloads import small_heterogeneous, point_source
from _gpu_helpers import oracle_problem, rel

pytestmark = pytest.mark.gpu

SIZES = [((48, 32), 3, 2), ((40, 40), 3, 1), ((64, 24), 3, 2), ((32, 32), 2, 1)]  # (n, levels, sources)


def _instances():
    out = []
    for k, (n, levels, nsrc) in enumerate(SIZES):
        w = small_heterogeneous(n, seed=20 + k, levels=levels, abl_cells=3, sigma_cells=2.0)
        rng = np.random.default_rng(40 + k)
        srcs = [point_source(n, 1, (int(rng.integers(4, n[0] - 4)), int(rng.integers(4, n[1] - 4))))
                for _ in range(nsrc)]
        out.append((w, srcs))
    return out


def _jobs(insts):
    import torch
    from paper_2307_03242_gb300 import emg
    solvers, jobs = [], []
    for w, srcs in insts:
        s = emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=torch.cuda.Stream())
        solvers.append(s)
        for q in srcs:
            b = torch.from_numpy(q).cuda()
            jobs.append((s, b, torch.zeros_like(b)))
    torch.cuda.synchronize()
    return solvers, jobs


@pytest.mark.parametrize("workers", [0, 2])
def test_batch_matches_individual_solves_and_the_oracle(workers):
    import torch
    from paper_2307_03242_gb300 import emg
    insts = _instances()
    solvers, jobs = _jobs(insts)
    seq = []
    for s, b, x in jobs:
        seq.append((s.solve(b, x, tol=1e-8, max_iter=400, restart=5), x.clone()))
        x.zero_()
    torch.cuda.synchronize()
    res = emg.solve_batch(jobs, tol=1e-8, max_iter=400, restart=5, workers=workers)
    for (st_seq, x_seq), st, (_, _, x) in zip(seq, res, jobs):
        assert st["status"] == 0 and st["converged"]
        assert st["iterations"] == st_seq["iterations"]
        assert torch.equal(x, x_seq)
    # each solution against the plain definition x = H^-1 b on the oracle's assembled operator
    import scipy.sparse.linalg as sla
    k = 0
    for w, srcs in insts:
        pb = oracle_problem(w)
        H = oracle.assemble(pb, 0.0).tocsr()
        act = oracle.active_mask(pb).astype(bool)
        Haa = H[act][:, act].tocsc()  # faces on the boundary are not unknowns
        for q in srcs:
            x_dir = sla.spsolve(Haa, q.ravel()[act])
            assert rel(jobs[k][2].cpu().numpy().ravel()[act], x_dir) < 1e-5
            k += 1
    for s in solvers:
        s.close()


def test_batch_reports_a_failing_job_without_disturbing_the_others():
    import torch
    from paper_2307_03242_gb300 import emg
    insts = _instances()[:2]
    solvers, jobs = _jobs(insts)
    bad = 1
    jobs[bad][1][0, 3, 5] = float("nan")  # a non-finite right-hand side
    res = emg.solve_batch(jobs, tol=1e-8, max_iter=400, restart=5, raise_errors=False)
    for k, st in enumerate(res):
        if k == bad:
            assert st["status"] == 4  # EMG_ERR_NONFINITE
        else:
            assert st["status"] == 0 and st["converged"]
    with pytest.raises(emg.EmgError):
        emg.solve_batch(jobs, tol=1e-8, max_iter=400, restart=5)
    for s in solvers:
        s.close()


def test_graph_replayed_cycles_match_eager_cycles():
    """A handle on a stream of its own replays the preconditioner cycle as a captured CUDA graph
    (from the second use of each Krylov slot on); a handle on the legacy default stream, where
    capture is not possible, runs it launch by launch. Same iterate bit for bit, same kernel
    count; with the instrumentation on, the graphs carry its event pairs, so both report the same
    number of timed launches per kernel class."""
    import torch
    from paper_2307_03242_gb300 import emg
    w, srcs = _instances()[0]
    p = emg.params_from_workload(w, 32)
    sg = emg.Solver(p, w.lam, w.mu, w.rho, stream=torch.cuda.Stream())
    se = emg.Solver(p, w.lam, w.mu, w.rho)  # torch's current stream: the legacy default stream
    assert se.stream.cuda_stream == 0
    b = torch.from_numpy(srcs[0]).cuda()
    torch.cuda.synchronize()
    out = {}
    for name, s in (("graph", sg), ("eager", se)):
        x = torch.zeros_like(b)
        s.solve(b, x, tol=1e-8, max_iter=60, restart=5)  # captures (graph handle)
        s.profile_read(emg.K_ALL)
        x.zero_()
        torch.cuda.synchronize()
        s.profile(True)
        st = s.solve(b, x, tol=1e-8, max_iter=60, restart=5)  # timed graphs are captured here
        s.profile_read(emg.K_SMOOTH)
        x.zero_()
        torch.cuda.synchronize()
        st = s.solve(b, x, tol=1e-8, max_iter=60, restart=5)  # ... and replayed here
        sm = s.profile_read(emg.K_SMOOTH)
        s.profile(False)
        out[name] = (st, x.clone(), s.profile_read(emg.K_ALL)["launches"], sm)
    (stg, xg, ng, smg), (ste, xe, ne, sme) = out["graph"], out["eager"]
    assert stg["iterations"] == ste["iterations"]
    assert torch.equal(xg, xe)
    assert ng == ne
    assert smg["launches"] == sme["launches"] > 0 and smg["ms"] > 0
    assert smg["bytes"] == sme["bytes"]
    sg.close()
    se.close()


def test_batch_with_handles_sharing_a_stream():
    """Handles on one stream (a stream pool hands the same stream to several callers) are driven
    by one worker, one after another: results equal the individual solves."""
    import torch
    from paper_2307_03242_gb300 import emg
    insts = _instances()
    shared = torch.cuda.Stream()
    solvers, jobs = [], []
    for k, (w, srcs) in enumerate(insts):
        st = shared if k % 2 == 0 else torch.cuda.Stream()
        s = emg.Solver(emg.params_from_workload(w, 32), w.lam, w.mu, w.rho, stream=st)
        solvers.append(s)
        b = torch.from_numpy(srcs[0]).cuda()
        jobs.append((s, b, torch.zeros_like(b)))
    torch.cuda.synchronize()
    ref = []
    for s, b, x in jobs:
        s.solve(b, x, tol=1e-8, max_iter=400, restart=5)
        ref.append(x.clone())
        x.zero_()
    torch.cuda.synchronize()
    res = emg.solve_batch(jobs, tol=1e-8, max_iter=400, restart=5)
    for st, r, (_, _, x) in zip(res, ref, jobs):
        assert st["status"] == 0
        assert torch.equal(x, r)
    for s in solvers:
        s.close()
