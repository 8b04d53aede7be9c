"""Data misfit of frequency-domain inversion and its gradient with respect to the material, as a
torch.autograd.Function over libemg's solves (the adjoint-state method, e.g. Plessix 2006; the
paper's solver is the forward solver of such an inversion, Sections 1 and 5).

    J(lambda, mu, rho) = 1/2 sum_s || u_s[receivers] - d_s ||^2,   u_s = H^{-1} q_s
    dJ/dm = -Re sum_s a_s^H (dH/dm) u_s,                           a_s = H^{-H} S^T (u_s[receivers] - d_s)

Every solve and the derivative kernel run in the library (emg_solve, emg_solve_adjoint,
emg_material_gradient); this module only sequences the calls and gathers the receiver values.
The forward fields are kept for the backward pass (one complex128 field per source), or
recomputed there with `keep_fields=False` when memory is short.
"""
from __future__ import annotations

import torch

from . import emg


class Misfit(torch.autograd.Function):
    """J = Misfit.apply(lam, mu, rho, params, sources, receivers, data, tol, keep_fields, solver, stats,
    restart).

    lam, mu, rho: float64 CUDA tensors of the grid's shape (n[::-1]); params: emg.Params
    (cycle_precision 32); sources: list of complex128 CUDA tensors of the solver's vector shape;
    receivers: int64 CUDA tensor of flat DOF indices; data: list of complex128 CUDA tensors (one
    value per receiver, per source)."""

    @staticmethod
    def forward(ctx, lam, mu, rho, params, sources, receivers, data, tol=1e-8, keep_fields=True, solver=None,
                stats=None, restart=20):
        # solver: an emg.Solver already built from this (lam, mu, rho), reused and left open;
        # stats: a list that receives each solve's statistics (forward, then adjoint)
        s = solver if solver is not None else emg.Solver(params, lam, mu, rho)
        fields, resid = [], []
        J = torch.zeros((), dtype=torch.float64, device=lam.device)
        for q, d in zip(sources, data):
            u = torch.zeros_like(q)
            st = s.solve(q, u, tol=tol, max_iter=4000, restart=restart)
            if not st["converged"]:
                raise RuntimeError("forward solve did not converge: %s" % st)
            if stats is not None:
                stats.append(dict(st, kind="forward"))
            r = u.reshape(-1)[receivers] - d
            J = J + 0.5 * torch.sum(r.real ** 2 + r.imag ** 2)
            fields.append(u if keep_fields else None)
            resid.append(r)
        ctx.solver, ctx.owned, ctx.stats = s, solver is None, stats
        ctx.fields, ctx.resid, ctx.sources = fields, resid, sources
        ctx.receivers, ctx.tol, ctx.restart = receivers, tol, restart
        return J

    @staticmethod
    def backward(ctx, gJ):
        s = ctx.solver
        out = tuple(torch.zeros(s.shape, dtype=torch.float64, device=gJ.device) for _ in range(3))
        for q, u, r in zip(ctx.sources, ctx.fields, ctx.resid):
            if u is None:  # recompute the forward field
                u = torch.zeros_like(q)
                st = s.solve(q, u, tol=ctx.tol, max_iter=4000, restart=ctx.restart)
                if not st["converged"]:
                    raise RuntimeError("recomputed forward solve did not converge: %s" % st)
            rhs = torch.zeros_like(q)
            rhs.reshape(-1).index_add_(0, ctx.receivers, r)
            a = torch.zeros_like(q)
            st = s.solve_adjoint(rhs, a, tol=ctx.tol, max_iter=4000, restart=ctx.restart)
            if not st["converged"]:
                raise RuntimeError("adjoint solve did not converge: %s" % st)
            if ctx.stats is not None:
                ctx.stats.append(dict(st, kind="adjoint"))
            s.material_gradient(u, a, out=out, accumulate=True)
        if ctx.owned:
            s.close()
        return (gJ * out[0], gJ * out[1], gJ * out[2]) + (None,) * 9


def misfit(lam, mu, rho, params, sources, receivers, data, tol=1e-8, keep_fields=True, solver=None, stats=None,
           restart=20):
    """J with autograd support for lam, mu, rho (see Misfit); restart: the FGMRES restart length
    of the forward and adjoint solves."""
    return Misfit.apply(lam, mu, rho, params, sources, receivers, data, tol, keep_fields, solver, stats, restart)
