"""Closed-form Fourier symbols and printed stencils used to pin the oracle.

Written from the paper's formulas only (Sections 3.1, 4.2, 5.3), independently of the
oracle's sparse assembly: a stencil's symbol is sum_k w_k exp(i k . offset_k), evaluated at
physical offsets, and the operator symbol is the 3x3 (2D) / 4x4 (3D) matrix of Eq. (4.4)
mixed-discretized-homogeneous with the homogeneous coefficients.
"""
from fractions import Fraction
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_singer_turkel():
    """LAP and MASS 3x3 stencils of Eq. (3.1), rows = x2 offset -1..1, cols = x1 offset -1..1."""
    out, cur = {}, None
    with open(os.path.join(GOLDEN, "singer_turkel_ho.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("LAP", "MASS"):
                cur = line
                out[cur] = []
                continue
            out[cur].append([float(Fraction(t)) for t in line.split()])
    return {k: np.array(v) for k, v in out.items()}


def read_intergrid():
    """{name: (weights[x2][x1], x1 offsets, x2 offsets)} in units of h."""
    out = {}
    with open(os.path.join(GOLDEN, "intergrid_stencils.txt")) as f:
        lines = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        name, den = lines[i].split()
        x1 = [float(t) for t in lines[i + 1].split(":")[1].split()]
        x2 = [float(t) for t in lines[i + 2].split(":")[1].split()]
        rows = [[float(t) for t in lines[i + 3 + r].split()] for r in range(len(x2))]
        out[name] = (np.array(rows) / float(den), np.array(x1), np.array(x2))
        i += 3 + len(x2)
    return out


def derivative_symbol(k, h):
    """Standard first derivative (1/h)[-1 * 1] on the half-shifted grid: 2i sin(k h / 2) / h."""
    return 2j * np.sin(k * h / 2.0) / h


def smooth_symbol(k, h):
    """[1 2 1]/4 along one axis: (1 + cos(k h)) / 2."""
    return 0.5 * (1.0 + np.cos(k * h))


def operator_symbol(kvec, h, beta, lam, mu, rho, omega, att):
    """Symbol of Eq. (4.4) for wavenumber vector kvec (radians per unit length).

    Rows/cols (u_1..u_d, p). Standard derivative s_a; beta-spread s_a^beta = s_a (beta +
    (1-beta) prod_{b != a} c_b) (Eq. 3.5 / dxSkew3D); Laplacian block sum_e conj(s_e) s_e^beta;
    mass beta + (1-beta)/(2d) sum_a 2 cos(k_a h) (Eq. 3.3 / massHO3D)."""
    d = len(kvec)
    s = np.array([derivative_symbol(kvec[a], h) for a in range(d)])
    c = np.array([smooth_symbol(kvec[a], h) for a in range(d)])
    sb = np.array([s[a] * (beta + (1 - beta) * np.prod([c[b] for b in range(d) if b != a]))
                   for a in range(d)])
    lap = mu * np.sum(np.conj(s) * sb)
    mass = beta + (1 - beta) / (2 * d) * np.sum(2 * np.cos(np.asarray(kvec) * h))
    m = rho * omega ** 2 * (1 - 1j * att)
    A = np.zeros((d + 1, d + 1), dtype=complex)
    for a in range(d):
        A[a, a] = lap - m * mass
        A[a, d] = s[a]
        A[d, a] = sb[a]
    A[d, d] = 1.0 / (lam + mu)
    return A


def dof_positions(n, h, comp, dim):
    """Physical positions (per axis) of the DOFs of one component on an n^dim grid, arrays
    shaped [z, y, x]. u_comp sits on the low face (x_comp = k h), p at cell centres."""
    grids = np.meshgrid(*[np.arange(v) for v in n[::-1]], indexing="ij")
    pos = []
    for a in range(dim):
        k = grids[dim - 1 - a].astype(float)
        pos.append(k * h if a == comp else (k + 0.5) * h)
    return pos


def mode(n, h, comp, dim, kvec):
    pos = dof_positions(n, h, comp, dim)
    phase = sum(kvec[a] * pos[a] for a in range(dim))
    return np.exp(1j * phase)
