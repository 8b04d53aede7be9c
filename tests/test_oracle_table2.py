"""The oracle's solver in the paper's own 2D configuration (Table 2, Section 5.2: homogeneous
medium, W(1,1) cycles of red-black Vanka, exact coarsest solve, FGMRES(5)) against the printed
iteration counts, as context for the solver variants.

The counts depend on what the paper leaves unstated: the absorbing layer's profile and strength
and the source's component (readings: gamma_max (delta/L)^2 with gamma_max = 2, a unit force on
u_2 at the middle of the first unknown row). With those readings the oracle needs 0.35-0.55 times
the printed cycles; a weaker layer, gamma_max = 0.5, brings the two-level counts to 19 and 37
against the printed 22 and 39 (a source at mid-depth with gamma_max = 2: 20 and 37). What the table shows is reproduced and pinned: the
spread stencil beta = 2/3 needs clearly fewer cycles than the standard beta = 1 (printed ratio
0.56 with two levels, 0.66 with three), and three levels need several times the cycles of two.
The 1024 x 256 rows (printed 56 / 32; measured 29 / 17, the growth from 512 x 128 as printed,
x1.42 against x1.45) take minutes and are recorded, not run."""
import os

import numpy as np
import pytest

import oracle
from oracle.discretization import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_homogeneous.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            v = line.split()
            out.append((int(v[0]), int(v[1]), int(v[2]), float(v[3]), float(v[4]), int(v[5])))
    return out


def _cycles(nx, ny, levels, beta, alpha, gamma_max=2.0):
    h = 1.0
    shape = (ny, nx)
    pb = Problem((nx, ny), h, 2 * np.pi / (10 * h), 0.01, beta, np.full(shape, 20.0), np.ones(shape), np.ones(shape),
                 abl_length=20 * h, abl_gamma_max=gamma_max)
    w = {2: 0.55, 3: 0.35}[levels]
    hier = oracle.Hierarchy(pb, levels, alpha, w, nu_pre=1, nu_post=1, coarse="sparse", cycle="W")
    b = np.zeros(oracle.dof_shape(pb), dtype=complex)
    b[1, 1, nx // 2] = 1.0
    H = oracle.assemble(pb, 0.0)
    _, its, _ = oracle.fgmres(lambda v: H @ v, lambda v: oracle.vcycle(hier, v), b.ravel(), tol=1e-6, restart=5,
                              max_iter=400)
    return its


@pytest.fixture(scope="module")
def measured():
    return {r: _cycles(*r[:5]) for r in _rows() if r[0] == 512}


def test_spread_stencil_needs_fewer_cycles_as_in_table2(measured):
    by = {(r[2], r[3]): (its, r[5]) for r, its in measured.items()}
    for levels in (2, 3):
        (s_its, s_pr), (b_its, b_pr) = by[(levels, 2.0 / 3.0)], by[(levels, 1.0)]
        assert s_its < 0.75 * b_its, (levels, s_its, b_its)
        assert abs(s_its / b_its - s_pr / b_pr) <= 0.15, (levels, s_its / b_its, s_pr / b_pr)


def test_three_levels_need_several_times_the_cycles_of_two(measured):
    by = {(r[2], r[3]): its for r, its in measured.items()}
    for beta in (2.0 / 3.0, 1.0):
        assert by[(3, beta)] >= 2 * by[(2, beta)], by


def test_cycle_counts_are_within_the_stated_band_of_table2(measured):
    for r, its in measured.items():
        assert 0.3 * r[5] <= its <= 1.0 * r[5], (r, its)


def test_two_level_counts_match_table2_with_a_weaker_absorbing_layer():
    """With gamma_max = 0.5 the two-level 512 x 128 counts are within 20 % of the printed ones."""
    for r in _rows():
        if r[0] == 512 and r[2] == 2:
            its = _cycles(*r[:5], gamma_max=0.5)
            assert abs(its - r[5]) <= 0.2 * r[5], (r, its)
