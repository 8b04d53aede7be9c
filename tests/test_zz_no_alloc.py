"""The allocation-free smoothing entry point (emg_smooth_noalloc).

Callers that cannot allocate device memory -- code running while a stream is captured into a
CUDA graph, applications whose device memory is owned by their own allocator -- use this entry
point instead of a handle: it runs the red-black Vanka sweeps of emg_smooth on caller-provided
material and vectors, with a fixed file-scope work array. This file is collected last so that a
run that stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from workloads import small_heterogeneous
from _gpu_helpers import oracle_problem, gpu_solver, random_field, to_gpu, to_np, rel_max, TOL


def _params_and_material(w):
    from paper_2307_03242_gb300 import emg
    import torch
    prm = emg.params_from_workload(w, cycle_precision=32)
    mu = torch.from_numpy(w.mu.astype(np.float32).ravel()).cuda()
    rho = torch.from_numpy(w.rho.astype(np.float32).ravel()).cuda()
    cp = torch.from_numpy((1.0 / (w.lam + w.mu)).astype(np.float32).ravel()).cuda()
    return prm, mu, rho, cp


@pytest.mark.gpu
def test_noalloc_smoothing_matches_the_handle_smoother_on_two_calls_in_a_row():
    """Same sweeps as emg_smooth (level 0 of a handle built from the same parameters), twice in a
    row with different inputs -- the second call reuses the shared work array."""
    from paper_2307_03242_gb300 import emg
    w = small_heterogeneous((72, 40), seed=9, levels=3, abl_cells=4, sigma_cells=2.0)
    pb = oracle_problem(w)
    s = gpu_solver(w, 32)
    prm, mu, rho, cp = _params_and_material(w)
    for call in range(2):
        b = random_field(pb, 100 + call)
        x0 = random_field(pb, 200 + call)
        x_ref = to_gpu(x0, 32)
        s.smooth(0, to_gpu(b, 32), x_ref, 2)
        x_new = to_gpu(x0, 32)
        emg.smooth_noalloc(prm, mu, rho, cp, to_gpu(b, 32), x_new, 2)
        assert rel_max(to_np(x_new), to_np(x_ref)) < TOL[32]
    s.close()


def test_noalloc_rejects_grids_beyond_its_work_array():
    from paper_2307_03242_gb300 import emg
    prm = emg.Params(n=(1024, 512), levels=1, cycle_precision=32).to_c()
    st = emg.LIB.emg_smooth_noalloc(ctypes.byref(prm), None, None, None, None, None, 1, None)
    assert st == 1
    prm2 = emg.Params(n=(1024, 512), levels=1, cycle_precision=32).to_c()
    dummy = ctypes.c_void_p(16)
    st = emg.LIB.emg_smooth_noalloc(ctypes.byref(prm2), dummy, dummy, dummy, dummy, dummy, 1, None)
    assert st == 1 and b"limited to 262144" in emg.LIB.emg_last_error()


@pytest.mark.parametrize("field,value", [("h", 0.0), ("h", float("nan")), ("omega", float("inf")),
                                         ("abl_cells", -1)])
def test_noalloc_rejects_parameters_that_emg_create_rejects(field, value):
    """The parameter checks of emg_create run before any device work (no GPU needed)."""
    from paper_2307_03242_gb300 import emg
    prm = emg.Params(n=(64, 64), levels=1, cycle_precision=32).to_c()
    setattr(prm, field, value)
    dummy = ctypes.c_void_p(16)
    st = emg.LIB.emg_smooth_noalloc(ctypes.byref(prm), dummy, dummy, dummy, dummy, dummy, 1, None)
    assert st == 1, emg.LIB.emg_last_error()
