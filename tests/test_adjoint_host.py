"""The adjoint's per-cell functions (csrc/adjoint.cuh), compiled for the host and looped over the
cells (libemg_hostcheck.so), against the FP64 oracle: y = H^H x against the oracle's assembled
conjugate transpose, and the material derivative -Re a^H (dH/dm) u against oracle/adjoint.py.
These are the functions the GPU kernels run; the GPU tests check the launches."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.adjoint import material_derivative
from workloads import small_heterogeneous
from _gpu_helpers import oracle_problem

DP = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def hc():
    from paper_2307_03242_gb300.build import build_hostcheck
    return ctypes.CDLL(build_hostcheck())


def _args(pb):
    n = np.array(list(pb.n) + [1] * (3 - pb.dim), dtype=np.int32)
    mats = [np.ascontiguousarray(pb.mu.ravel()), np.ascontiguousarray(pb.rho.ravel()),
            np.ascontiguousarray((1.0 / (pb.lam + pb.mu)).ravel())]
    head = [pb.dim, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h), ctypes.c_double(pb.beta),
            ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma), ctypes.c_double(pb.abl_length),
            ctypes.c_double(pb.abl_gamma_max)] + [m.ctypes.data_as(DP) for m in mats]
    return head, (n, mats)


def _cvec(v):
    return v.view(np.float64).ctypes.data_as(DP)


def _rand(act, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(act.size) + 1j * rng.standard_normal(act.size)) * act


CASES = [((9, 7), 2), ((16, 10), 3), ((6, 5, 4), 2), ((7, 6, 5), 1)]


@pytest.mark.parametrize("n,abl", CASES)
def test_host_adjoint_apply_matches_the_oracle_conjugate_transpose(hc, n, abl):
    w = small_heterogeneous(n, seed=2, abl_cells=abl)
    pb = oracle_problem(w)
    act = oracle.active_mask(pb)
    x = _rand(act, 1)
    ref = oracle.assemble(pb, 0.0).conj().T @ x
    y = np.zeros_like(x)
    head, keep = _args(pb)
    assert hc.emg_hc_adjoint_apply(*head, _cvec(x), _cvec(y)) == 0
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n,abl", CASES)
def test_host_material_derivative_matches_the_oracle(hc, n, abl):
    w = small_heterogeneous(n, seed=4, abl_cells=abl)
    pb = oracle_problem(w)
    act = oracle.active_mask(pb)
    u, a = _rand(act, 2), _rand(act, 3)
    ref = material_derivative(pb, u, a)
    g = [np.zeros(pb.ncell) for _ in range(3)]
    head, keep = _args(pb)
    assert hc.emg_hc_material_gradient(*head, _cvec(u), _cvec(a), *[v.ctypes.data_as(DP) for v in g]) == 0
    for got, name in zip(g, ("lam", "mu", "rho")):
        r = ref[name].ravel()
        assert np.abs(got - r).max() <= 1e-13 * np.abs(r).max(), name
