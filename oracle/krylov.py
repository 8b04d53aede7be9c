"""Restarted flexible GMRES, right-preconditioned (oracle; test infrastructure only).

FGMRES(m) of Saad (1993), as used around the multigrid preconditioner in
Sections 3.2 and 5 (the paper's outer solver; FP64 outer vectors, Section 5.3):
Arnoldi with modified Gram-Schmidt on the vectors v_j, the preconditioned vectors
z_j = M^{-1} v_j are kept, Givens rotations reduce the Hessenberg matrix, and
x = x_0 + Z y at the end of every cycle of m steps. The true residual b - A x is
recomputed at every restart; the solve stops when ||b - A x|| / ||b|| <= tol
(zero initial guess by default, Section 5).
"""
from __future__ import annotations

import numpy as np


def fgmres(A, M, b, x0=None, tol=1e-6, max_iter=1000, restart=20, history=None):
    """Returns (x, iterations, relative true residual). A and M map flat vectors to flat vectors."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).ravel().copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b - A(x)
    beta = np.linalg.norm(r)
    its = 0
    if history is not None:
        history.append(beta / bnorm)
    while beta / bnorm > tol and its < max_iter:
        m = restart
        V = np.zeros((m + 1, b.size), dtype=np.complex128)
        Z = np.zeros((m, b.size), dtype=np.complex128)
        Hh = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A(Z[j])
            for i in range(j + 1):            # modified Gram-Schmidt
                Hh[i, j] = np.vdot(V[i], w)
                w = w - Hh[i, j] * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] != 0.0:
                V[j + 1] = w / Hh[j + 1, j]
            for i in range(j):                # previous rotations
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -np.conj(sn[i]) * Hh[i, j] + np.conj(cs[i]) * Hh[i + 1, j]
                Hh[i, j] = t
            a, bb = Hh[j, j], Hh[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j] = a / den
                sn[j] = bb / den
                cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
            Hh[j, j] = cs[j] * a + sn[j] * bb
            Hh[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or its >= max_iter or Hh[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(Hh[:k, :k]), g[:k])
        x = x + Z[:k].T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
    return x, its, beta / bnorm
