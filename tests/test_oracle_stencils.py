"""Pins of the oracle's assembled operator against the paper's printed stencils and symbols.

CPU only. The expected values come from the paper (golden fixtures) or from closed-form
Fourier symbols written in tests/_paper_symbols.py -- never from the oracle itself.
"""
import numpy as np
import pytest

import oracle
from oracle.discretization import Problem
from _paper_symbols import read_singer_turkel, operator_symbol, mode


def _homog(n, h=1.0, beta=2.0 / 3.0, lam=3.0, mu=1.0, rho=1.0, omega=0.9, gamma=0.05, periodic=True):
    shape = tuple(n[::-1])
    return Problem(n, h, omega, gamma, beta, np.full(shape, lam), np.full(shape, mu),
                   np.full(shape, rho), periodic=periodic)


def _u_block_stencil(H, pb, comp, centre):
    """3x3 stencil (rows: x2 offset -1..1, cols: x1 offset -1..1) of the u_comp-u_comp block at a
    2D face, together with the total absolute mass of the row outside that 3x3 window."""
    N = pb.ncell
    nx, ny = pb.n
    i, j = centre
    row = comp * N + j * nx + i
    r = H.getrow(row).toarray().ravel()
    st = np.zeros((3, 3), dtype=complex)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            col = comp * N + ((j + dj) % ny) * nx + (i + di) % nx
            st[dj + 1, di + 1] = r[col]
            r[col] = 0.0
    other_u = np.abs(r[:2 * N]).sum()
    return st, other_u, r[2 * N:]


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_singer_turkel_reproduced_at_beta_two_thirds(h):
    """Eq. (3.1)-(3.3): at beta = 2/3 the u-block is the compact 4th-order acoustic stencil."""
    gold = read_singer_turkel()
    omega, gamma = 0.7 / h, 0.03
    pb = _homog((8, 8), h=h, omega=omega, gamma=gamma, mu=1.0, rho=1.0)
    H = oracle.assemble(pb, shift=0.0)
    expect = gold["LAP"] / h ** 2 - omega ** 2 * (1 - 1j * gamma) * gold["MASS"]
    for comp in (0, 1):
        st, other, prow = _u_block_stencil(H, pb, comp, (3, 4))
        np.testing.assert_allclose(st, expect, rtol=0, atol=1e-13 / h ** 2)
        assert other < 1e-14 / h ** 2, "u-block must be block diagonal and 9-point"
        # u-p coupling: the standard gradient (+1/h at the cell above, -1/h below), Eq. (4.4)
        nz = np.nonzero(np.abs(prow) > 0)[0]
        assert len(nz) == 2
        vals = sorted(prow[nz].real)
        np.testing.assert_allclose(vals, [-1.0 / h, 1.0 / h], rtol=1e-14)


@pytest.mark.parametrize("beta", [1.0, 0.8, 2.0 / 3.0, 0.5])
def test_laplacian_is_convex_combination_of_standard_and_skew(beta):
    """grad_h^T grad_h^beta = -Delta^beta (Section 3.1) with -Delta^beta of Eq. (3.2) LapHO."""
    h = 0.5
    pb = _homog((8, 8), h=h, beta=beta, omega=0.0, gamma=0.0)
    H = oracle.assemble(pb, shift=0.0)
    five = np.array([[0, -1, 0], [-1, 4, -1], [0, -1, 0]], float)
    skew = np.array([[-1, 0, -1], [0, 4, 0], [-1, 0, -1]], float)
    expect = beta * five / h ** 2 + (1 - beta) * skew / (2 * h ** 2)
    for comp in (0, 1):
        st, _, _ = _u_block_stencil(H, pb, comp, (4, 2))
        np.testing.assert_allclose(st.real, expect, atol=1e-12)
        assert np.abs(st.imag).max() == 0.0


def _check_symbol(n, h, kidx, beta, shift, dim):
    pb = _homog(n, h=h, beta=beta, lam=2.5, mu=1.3, rho=0.8, omega=1.1, gamma=0.02)
    H = oracle.assemble(pb, shift=shift)
    kvec = [2 * np.pi * kidx[a] / (n[a] * h) for a in range(dim)]
    A = operator_symbol(kvec, h, beta, 2.5, 1.3, 0.8, 1.1, 0.02 + shift)
    rng = np.random.default_rng(sum(kidx) + 17)
    uhat = rng.standard_normal(dim + 1) + 1j * rng.standard_normal(dim + 1)
    x = np.concatenate([uhat[c] * mode(n, h, c, dim, kvec).ravel() for c in range(dim + 1)])
    y = H @ x
    yhat = A @ uhat
    expect = np.concatenate([yhat[c] * mode(n, h, c, dim, kvec).ravel() for c in range(dim + 1)])
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("kidx", [(1, 0), (3, 5), (7, 2), (4, 4), (0, 6)])
@pytest.mark.parametrize("beta", [1.0, 2.0 / 3.0])
def test_operator_symbol_2d(kidx, beta):
    """Operator applied to a staggered Fourier mode = symbol of Eq. (4.4) times the mode."""
    _check_symbol((8, 8), 0.5, kidx, beta, 0.3, 2)


@pytest.mark.parametrize("kidx", [(1, 0, 0), (1, 2, 3), (3, 1, 2), (2, 2, 2)])
def test_operator_symbol_3d(kidx):
    """3D: Eq. dxSkew3D spread derivatives (with 1/h) and Eq. massHO3D, same block form."""
    _check_symbol((4, 4, 6), 1.0, kidx, 2.0 / 3.0, 0.1, 3)


def test_schur_complement_is_negated_elastic_operator():
    """Reading of the u-p coupling sign: eliminating p gives
    -(mu Lap + rho w^2 M + (lam+mu) grad div) in symbol form, consistent with Eq. (2.3)."""
    h, beta, lam, mu, rho, w, att = 1.0, 2.0 / 3.0, 4.0, 1.5, 1.2, 0.8, 0.0
    for kvec in ([0.3, 0.7], [1.1, -0.4], [2.0, 2.5]):
        # small-k agreement of -Schur with the continuous operator (second order in k h)
        kk = np.array(kvec) * 1e-3
        A2 = operator_symbol(kk, h, beta, lam, mu, rho, w, att)
        s2 = A2[:2, :2] - np.outer(A2[:2, 2], A2[2, :2]) / A2[2, 2]
        # continuous elastic operator symbol (Eq. 2.2): -mu |k|^2 - (lam+mu) k k^T + rho w^2
        c2 = -mu * (kk @ kk) * np.eye(2) - (lam + mu) * np.outer(kk, kk) + rho * w ** 2 * np.eye(2)
        np.testing.assert_allclose(-s2, c2, rtol=1e-5, atol=1e-10)


def test_homogeneous_dirichlet_boundary_faces_are_not_unknowns():
    pb = _homog((6, 4), periodic=False)
    H = oracle.assemble(pb, 0.2)
    act = oracle.active_mask(pb)
    assert act.sum() == 3 * 24 - 4 - 6
    dead = np.nonzero(~act)[0]
    assert abs(H[dead]).sum() == 0 and abs(H[:, dead]).sum() == 0
