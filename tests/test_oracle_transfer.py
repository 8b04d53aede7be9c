"""Pins of the oracle's restriction / prolongation and of the coarse-grid correction.

The expected values are the printed inter-grid stencils of Eq. (2.11)-(2.12) (golden
fixture), their Fourier symbols (Eq. 4.7 Ru1Symbol, read with its second line and the 1/8
factor), and the two-grid coarse-grid-correction symbol of Eq. (4.6) symbolTG with nu = 0.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle.discretization import Problem
from _paper_symbols import read_intergrid, operator_symbol, mode, dof_positions


def _homog(n, h=1.0, periodic=True, beta=2.0 / 3.0):
    shape = tuple(n[::-1])
    return Problem(n, h, 0.9, 0.05, beta, np.full(shape, 3.0), np.full(shape, 1.0),
                   np.full(shape, 1.0), periodic=periodic)


def _stencils(dim):
    """Per component: (R weights+offsets, P weights+offsets) in units of h, from the printed
    2D stencils; u1 is the rotated u2 stencil; 3D uses the tensor-product reading."""
    g = read_intergrid()

    def to_list(name, swap=False):
        w, x1, x2 = g[name]
        out = []
        for r, oy in enumerate(x2):
            for c, ox in enumerate(x1):
                if w[r, c] != 0:
                    out.append(((oy, ox) if swap else (ox, oy), w[r, c]))
        return out

    if dim == 2:
        R = [to_list("R_u2", swap=True), to_list("R_u2"), to_list("R_p")]
        P = [to_list("P_u2", swap=True), to_list("P_u2"), to_list("P_p")]
        return R, P
    # 3D: tensor products of the 1D factors read off the 2D stencils
    r_face = [(-1.0, 0.25), (0.0, 0.5), (1.0, 0.25)]
    r_cell = [(-0.5, 0.5), (0.5, 0.5)]
    p_face = [(-1.0, 0.5), (0.0, 1.0), (1.0, 0.5)]
    p_cell = [(-1.5, 0.25), (-0.5, 0.75), (0.5, 0.75), (1.5, 0.25)]
    R, P = [], []
    for comp in range(4):
        fr = [r_face if a == comp else r_cell for a in range(3)]
        fp = [p_face if a == comp else p_cell for a in range(3)]
        R.append([(tuple(o for o, _ in t), np.prod([w for _, w in t])) for t in itertools.product(*fr)])
        P.append([(tuple(o for o, _ in t), np.prod([w for _, w in t])) for t in itertools.product(*fp)])
    return R, P


def test_printed_stencils_are_consistent_with_their_description():
    g = read_intergrid()
    for name in ("R_p", "R_u2"):
        assert abs(g[name][0].sum() - 1.0) < 1e-15
    for name in ("P_p", "P_u2"):
        assert abs(g[name][0].sum() - 4.0) < 1e-15  # 2^d fine points per coarse point


def test_restriction_symbol_ru1_matches_eq_4_7():
    """R_u1 applied to a fine Fourier mode = R~_u1(theta) x coarse mode,
    R~_u1 = (1/8)[2cos(t1 + t2/2) + 2cos(t1 - t2/2) + 4cos(t2/2)] (Eq. 4.7, second line)."""
    n, h = (16, 16), 1.0
    fine = _homog(n, h)
    coarse = oracle.coarsen(fine)
    R = oracle.restriction(fine, coarse)
    N, Nc = fine.ncell, coarse.ncell
    for kidx in [(1, 2), (3, -2), (5, 7), (0, 4)]:
        th = [2 * np.pi * kidx[a] / n[a] for a in range(2)]
        k = [t / h for t in th]
        x = np.zeros(3 * N, complex)
        x[:N] = mode(n, h, 0, 2, k).ravel()
        y = R @ x
        t1, t2 = th
        rs = (2 * np.cos(t1 + t2 / 2) + 2 * np.cos(t1 - t2 / 2) + 4 * np.cos(t2 / 2)) / 8
        expect = rs * mode(coarse.n, coarse.h, 0, 2, k).ravel()
        np.testing.assert_allclose(y[:Nc], expect, atol=1e-13)
        assert np.abs(y[Nc:]).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_and_prolongation_match_printed_stencils(dim):
    """R and P act on Fourier modes exactly as the printed stencils say (every component)."""
    n = (8, 8) if dim == 2 else (4, 4, 4)
    h = 1.0
    fine = _homog(n, h)
    coarse = oracle.coarsen(fine)
    R = oracle.restriction(fine, coarse)
    P = oracle.prolongation(fine, coarse)
    N, Nc = fine.ncell, coarse.ncell
    Rst, Pst = _stencils(dim)
    rng = np.random.default_rng(3)
    for _ in range(4):
        kidx = rng.integers(0, 4, size=dim)
        k = [2 * np.pi * kidx[a] / (n[a] * h) for a in range(dim)]
        for comp in range(dim + 1):
            # restriction: (R v)(X) = sum_k r_k v(X + o_k)
            x = np.zeros((dim + 1) * N, complex)
            x[comp * N:(comp + 1) * N] = mode(n, h, comp, dim, k).ravel()
            y = R @ x
            rt = sum(w * np.exp(1j * sum(k[a] * o[a] * h for a in range(dim))) for o, w in Rst[comp])
            expect = rt * mode(coarse.n, coarse.h, comp, dim, k).ravel()
            np.testing.assert_allclose(y[comp * Nc:(comp + 1) * Nc], expect, atol=1e-13)
            # prolongation: fine(x) = sum over coarse X and stencil offsets o with X + o = x
            xc = np.zeros((dim + 1) * Nc, complex)
            cm = mode(coarse.n, coarse.h, comp, dim, k)
            xc[comp * Nc:(comp + 1) * Nc] = cm.ravel()
            z = (P @ xc)[comp * N:(comp + 1) * N].reshape(tuple(n[::-1]))
            fpos = dof_positions(n, h, comp, dim)
            cpos = dof_positions(coarse.n, coarse.h, comp, dim)
            ref = np.zeros(tuple(n[::-1]), complex)
            L = [n[a] * h for a in range(dim)]
            for o, w in Pst[comp]:
                # fine points that sit at X + o*h for a coarse point X (periodic wrap)
                tgt = [np.mod(cpos[a] + o[a] * h, L[a]) for a in range(dim)]
                idx = [np.rint((tgt[a] - fpos[a].flat[0]) / h).astype(int) % n[a] for a in range(dim)]
                np.add.at(ref, tuple(idx[::-1]), w * cm)
            np.testing.assert_allclose(z, ref, atol=1e-13)


def test_prolongation_reproduces_constants_and_linears_in_the_interior():
    n = (16, 16)
    fine = _homog(n, periodic=False)
    coarse = oracle.coarsen(fine)
    P = oracle.prolongation(fine, coarse)
    R = oracle.restriction(fine, coarse)
    N, Nc = fine.ncell, coarse.ncell
    for comp in range(3):
        for lin in (lambda x, y: 1.0 + 0 * x, lambda x, y: 2.0 * x - 0.5 * y + 3.0):
            cpos = dof_positions(coarse.n, coarse.h, comp, 2)
            fpos = dof_positions(n, fine.h, comp, 2)
            xc = np.zeros(3 * Nc)
            xc[comp * Nc:(comp + 1) * Nc] = lin(*cpos).ravel()
            xc = xc * oracle.active_mask(coarse)
            z = (P @ xc)[comp * N:(comp + 1) * N].reshape(n[::-1])
            want = lin(*fpos)
            inner = (slice(3, -3), slice(3, -3))
            np.testing.assert_allclose(z[inner], want[inner], atol=1e-12)
            xf = np.zeros(3 * N)
            xf[comp * N:(comp + 1) * N] = 1.0
            xf = xf * oracle.active_mask(fine)
            r = (R @ xf)[comp * Nc:(comp + 1) * Nc].reshape(coarse.n[::-1])
            np.testing.assert_allclose(r[2:-2, 2:-2], 1.0, atol=1e-14)


def _cgc_symbol(dim, th, h, beta, lam, mu, rho, omega, att, Rst, Pst, n, hc):
    """Eq. (4.6) with nu = 0: K~ = I - P~ A~_2h^{-1} R~ A~_h over the 2^d harmonics
    (ordering: component-major, harmonic-minor). Signs of the staggered coarse lattices are
    taken from the physical DOF positions (sigma, tau below)."""
    harm = list(itertools.product((0, 1), repeat=dim))
    nh = len(harm)
    nc = dim + 1
    ths = [np.array(th) + np.pi * np.array(kap) for kap in harm]
    Ah = np.zeros((nc * nh, nc * nh), complex)
    for a, t in enumerate(ths):
        A = operator_symbol(t / h, h, beta, lam, mu, rho, omega, att)
        for c in range(nc):
            for c2 in range(nc):
                Ah[c * nh + a, c2 * nh + a] = A[c, c2]
    A2h = operator_symbol(np.array(th) / h, hc, beta, lam, mu, rho, omega, att)
    Rt = np.zeros((nc, nc * nh), complex)
    Pt = np.zeros((nc * nh, nc), complex)
    for c in range(nc):
        y0 = [p.flat[0] for p in dof_positions(tuple(v // 2 for v in n), hc, c, dim)]
        for a, (t, kap) in enumerate(zip(ths, harm)):
            k = t / h
            sig = np.exp(1j * np.pi * sum(kap[b] * y0[b] / h for b in range(dim)))
            rt = sum(w * np.exp(1j * sum(k[b] * o[b] * h for b in range(dim))) for o, w in Rst[c])
            pt = sum(w * np.exp(-1j * sum(k[b] * o[b] * h for b in range(dim))) for o, w in Pst[c])
            Rt[c, c * nh + a] = rt * sig
            Pt[c * nh + a, c] = pt * np.conj(sig) / 2 ** dim
    return np.eye(nc * nh) - Pt @ np.linalg.solve(A2h, Rt @ Ah)


@pytest.mark.parametrize("dim,beta", [(2, 2.0 / 3.0), (2, 1.0), (3, 2.0 / 3.0)])
def test_coarse_grid_correction_matches_two_grid_symbol(dim, beta):
    """K = I - P A_2h^{-1} R A_h (re-discretised A_2h, exact coarse solve) restricted to the space
    of harmonics E(theta) equals the symbol matrix of Eq. (4.6) symbolTG with nu_1 = nu_2 = 0."""
    n = (16, 16) if dim == 2 else (8, 8, 8)
    h, shift = 1.0, 0.3
    fine = _homog(n, h, beta=beta)
    coarse = oracle.coarsen(fine)
    Ah = oracle.assemble(fine, shift)
    A2h = oracle.assemble(coarse, shift).toarray()
    R = oracle.restriction(fine, coarse)
    P = oracle.prolongation(fine, coarse)
    A2inv = sla.inv(A2h)
    Rst, Pst = _stencils(dim)
    N = fine.ncell
    nc = dim + 1
    harm = list(itertools.product((0, 1), repeat=dim))
    nh = len(harm)
    for kidx in ([1, 2] if dim == 2 else [1, 0, 2], [3, -1] if dim == 2 else [1, 1, 1]):
        th = np.array([2 * np.pi * kidx[a] / n[a] for a in range(dim)])
        Kt = _cgc_symbol(dim, th, h, beta, 3.0, 1.0, 1.0, 0.9, 0.05 + shift, Rst, Pst, n, 2 * h)
        basis = []
        for c in range(nc):
            for kap in harm:
                k = (th + np.pi * np.array(kap)) / h
                v = np.zeros(nc * N, complex)
                v[c * N:(c + 1) * N] = mode(n, h, c, dim, k).ravel()
                basis.append(v)
        B = np.array(basis).T
        KB = B - P @ (A2inv @ (R @ (Ah @ B)))
        coef = (B.conj().T @ KB) / N
        np.testing.assert_allclose(B @ coef, KB, atol=1e-10)     # K maps E(theta) into itself
        np.testing.assert_allclose(coef, Kt, atol=1e-10)
