"""Pin of the oracle's cycle recursion (Algorithm 1 applied recursively, Sec. 2.2) against the
closed-form error propagator of multigrid theory (Hackbusch, Multi-Grid Methods and
Applications, 1985, Sec. 7.1; Trottenberg, Oosterlee and Schueller, Multigrid, 2001, Sec. 2.4).

For a linear cycle on level l with nu_1 pre- and nu_2 post-steps of a smoother whose error
propagator is S_l, and gamma recursive calls (the second starting from the first one's result),
the error propagator is

    M_l = S_l^{nu_2} (I - P_l (I - M_{l+1}^gamma) A_{l+1}^{-1} R_l A_l) S_l^{nu_1},

with M_{L-1} = 0 for an exact coarsest solve, and the cycle with a zero initial guess returns
x = (I - M_l) A_l^{-1} b. gamma = 1 is the V-cycle, gamma = 2 the W-cycle.

S_l is built column by column from the oracle's red-black sweep (itself pinned elsewhere:
single-cell exactness, fixed point, colour partition) and A_l, R_l, P_l are the assembled
operators (pinned by the symbols and printed stencils). The cycle is then checked against the
formula as a whole matrix, on the active DOFs of a tiny three-level hierarchy.

The reading "the coarsest level is solved once per visit" (the cycle on the level above the
coarsest makes a single call, also in a W-cycle) matters only when the coarsest solve is
inexact. With s red-black sweeps from a zero guess the coarsest "cycle" has the error propagator
M_c = S_c^s; under the reading the level above the coarsest uses (I - M_c), and a textbook
W-cycle that solved it twice would use (I - M_c^2). Both are computed below and the oracle
must match the first and differ from the second.
"""
import numpy as np
import pytest

import oracle
import oracle.multigrid as mg
from oracle.discretization import Problem
from oracle.smoother import red_black_sweep
from workloads import small_heterogeneous


def _hierarchy(cycle, coarse, nu=(1, 1), n=(16, 8)):
    w = small_heterogeneous(n, levels=3, abl_cells=2)
    pb = Problem(w.n, w.h, w.omega, w.gamma, w.beta, w.lam, w.mu, w.rho,
                 abl_length=w.abl_cells * w.h, abl_gamma_max=w.abl_gamma_max)
    kw = dict(coarse="dense") if coarse == "dense" else dict(coarse="smooth", coarse_sweeps=3, coarse_damping=0.8)
    return oracle.Hierarchy(pb, 3, [0.4, 0.6, 1.0], [0.6, 0.4, 0.8], nu_pre=nu[0], nu_post=nu[1], cycle=cycle, **kw)


def _sweep_matrix(hier, l, w):
    """Error propagator of one red-black sweep on level l (restricted to the active DOFs):
    column k is the sweep of the k-th unit error with a zero right-hand side."""
    act = oracle.active_mask(hier.pbs[l])
    ids = np.nonzero(act)[0]
    S = np.zeros((ids.size, ids.size), dtype=np.complex128)
    zero = np.zeros(act.size, dtype=np.complex128)
    for c, k in enumerate(ids):
        e = zero.copy()
        e[k] = 1.0
        S[:, c] = red_black_sweep(hier.H[l], hier.V[l], hier.idx[l], hier.colour[l], zero, e, w)[ids]
    return S, ids


def _level_mats(hier):
    mats = []
    for l in range(hier.levels):
        S, ids = _sweep_matrix(hier, l, hier.w[l])
        A = hier.H[l][ids][:, ids].toarray()
        mats.append({"S": S, "A": A, "ids": ids})
    for l in range(hier.levels - 1):
        fi, ci = mats[l]["ids"], mats[l + 1]["ids"]
        mats[l]["R"] = hier.R[l][ci][:, fi].toarray()
        mats[l]["P"] = hier.P[l][fi][:, ci].toarray()
    return mats


def _propagator(hier, mats, l, gamma, coarse_calls):
    """M_l from the closed form; coarse_calls = recursive calls made on the level above the
    coarsest (1 under the oracle's reading, gamma for a textbook W-cycle)."""
    last = hier.levels - 1
    I = np.eye(mats[l]["A"].shape[0])
    if l == last:
        if hier.coarse == "dense":
            return np.zeros_like(I, dtype=np.complex128)
        S = mats[l]["S"] if hier.coarse_damping == hier.w[l] else _sweep_matrix(hier, l, hier.coarse_damping)[0]
        return np.linalg.matrix_power(S, hier.coarse_sweeps)
    calls = coarse_calls if l + 1 == last else gamma
    Mc = _propagator(hier, mats, l + 1, gamma, coarse_calls)
    Ic = np.eye(Mc.shape[0])
    m = mats[l]
    cgc = I - m["P"] @ (Ic - np.linalg.matrix_power(Mc, calls)) @ np.linalg.solve(mats[l + 1]["A"], m["R"] @ m["A"])
    S1 = np.linalg.matrix_power(m["S"], hier.nu_pre)
    S2 = np.linalg.matrix_power(m["S"], hier.nu_post)
    return S2 @ cgc @ S1


def _cycle_matrix(hier, ids):
    """The oracle's cycle with a zero initial guess, column by column: x = N b."""
    n = hier.H[0].shape[0]
    N = np.zeros((ids.size, ids.size), dtype=np.complex128)
    for c, k in enumerate(ids):
        b = np.zeros(n, dtype=np.complex128)
        b[k] = 1.0
        N[:, c] = mg.vcycle(hier, b)[ids]
    return N


def _check(hier, gamma, coarse_calls):
    mats = _level_mats(hier)
    M = _propagator(hier, mats, 0, gamma, coarse_calls)
    A = mats[0]["A"]
    expect = (np.eye(A.shape[0]) - M) @ np.linalg.inv(A)
    got = _cycle_matrix(hier, mats[0]["ids"])
    return np.abs(got - expect).max() / np.abs(expect).max()


@pytest.mark.parametrize("nu", [(1, 1), (2, 1)])
def test_wcycle_equals_closed_form_error_propagator_with_exact_coarsest(nu):
    hier = _hierarchy("W", "dense", nu)
    assert _check(hier, 2, 2) <= 1e-12
    # the V-cycle formula (one call on level 1) is a different matrix
    assert _check(hier, 1, 1) > 1e-3


def test_vcycle_equals_closed_form_error_propagator():
    hier = _hierarchy("V", "dense")
    assert _check(hier, 1, 1) <= 1e-12
    assert _check(hier, 2, 2) > 1e-3


def test_wcycle_solves_an_inexact_coarsest_level_once_per_visit():
    """The reading: on the level above the coarsest the W-cycle makes one call of the inexact
    coarsest solve (s sweeps from zero), not two."""
    hier = _hierarchy("W", "smooth")
    assert _check(hier, 2, 1) <= 1e-12
    assert _check(hier, 2, 2) > 1e-4
