"""Shared helpers for the GPU parity tests: build the oracle problem and the GPU solver from the
same seeded workload, move vectors between numpy and CUDA tensors, compare."""
import numpy as np

import oracle
from oracle.discretization import Problem


def oracle_problem(w):
    return Problem(w.n, w.h, w.omega, w.gamma, w.beta, w.lam, w.mu, w.rho,
                   abl_length=w.abl_cells * w.h, abl_gamma_max=w.abl_gamma_max)


def oracle_hierarchy(w, pb=None, damping=None):
    pb = pb or oracle_problem(w)
    return oracle.Hierarchy(pb, w.levels, w.level_alphas(), w.damping if damping is None else damping,
                            nu_pre=w.nu_pre, nu_post=w.nu_post, coarse=w.coarse,
                            coarse_sweeps=w.coarse_sweeps, coarse_damping=w.coarse_damping, cycle=w.cycle,
                            smoother=w.smoother)


def gpu_solver(w, prec, **over):
    from paper_2307_03242_gb300 import emg
    return emg.Solver(emg.params_from_workload(w, cycle_precision=prec, **over), w.lam, w.mu, w.rho)


def random_field(pb, seed):
    rng = np.random.default_rng(seed)
    shape = oracle.dof_shape(pb)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return (v.ravel() * oracle.active_mask(pb)).reshape(shape)


def to_gpu(a, prec):
    import torch
    dt = torch.complex64 if prec == 32 else torch.complex128
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dt).contiguous()


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.to(torch.complex128).cpu().numpy()


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rel_max(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


TOL = {64: 1e-12, 32: 2e-6}       # single kernels (max-norm relative)
TOL_CYCLE = {64: 1e-11, 32: 1e-5}  # composed cycle (2-norm relative)
