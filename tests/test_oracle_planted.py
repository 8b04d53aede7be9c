"""Sensitivity of the oracle pins: a plausible mistake planted in the oracle (on the CPU,
by monkeypatching one of its building blocks) must make at least one pin fail."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.discretization as disc
import oracle.transfer as tr
import oracle.krylov as kr
import oracle.smoother as sm
import test_oracle_stencils as ts
import test_oracle_transfer as tt
import test_oracle_solver as tsol


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_planted_wrong_spread_weights_break_the_symbol_pin(monkeypatch):
    monkeypatch.setattr(disc, "_smooth121", lambda n, per: sp.csr_matrix(
        sp.diags([np.full(n - 1, 1 / 3), np.full(n, 1 / 3), np.full(n - 1, 1 / 3)], [-1, 0, 1])))
    _fails(ts._check_symbol, (8, 8), 0.5, (3, 5), 2.0 / 3.0, 0.3, 2)


def test_planted_gradient_sign_breaks_the_stencil_pin(monkeypatch):
    orig = disc._gradient_p
    monkeypatch.setattr(disc, "_gradient_p", lambda pb, c: -orig(pb, c))
    _fails(ts._check_symbol, (8, 8), 0.5, (1, 0), 1.0, 0.3, 2)


def test_planted_mass_spread_weight_breaks_singer_turkel(monkeypatch):
    orig = disc._mass_spread

    def wrong(pb):
        N = pb.ncell
        m = orig(pb)
        return m + (1 - pb.beta) * 0.05 * sp.identity(N)
    monkeypatch.setattr(disc, "_mass_spread", wrong)
    _fails(ts.test_singer_turkel_reproduced_at_beta_two_thirds, 1.0)


def test_planted_dropped_transverse_term_in_3d_breaks_the_3d_symbol(monkeypatch):
    orig = disc._derivative

    def wrong(pb, comp, e, spread):
        if not spread or pb.dim != 3:
            return orig(pb, comp, e, spread)
        return orig(pb, comp, e, False)  # spread silently dropped in 3D
    monkeypatch.setattr(disc, "_derivative", wrong)
    _fails(ts._check_symbol, (4, 4, 6), 1.0, (1, 2, 3), 2.0 / 3.0, 0.1, 3)


def test_planted_swapped_prolongation_weights_break_the_stencil_pin(monkeypatch):
    def wrong(nf, per):
        nc = nf // 2
        rows, cols, vals = [], [], []
        for K in range(nc):
            for off, w in ((-1, 0.75), (0, 0.25), (1, 0.25), (2, 0.75)):
                f = (2 * K + off) % nf
                rows.append(f); cols.append(K); vals.append(w)
        return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))
    monkeypatch.setattr(tr, "_p_cell", wrong)
    _fails(tt.test_restriction_and_prolongation_match_printed_stencils, 2)


def test_planted_restriction_weights_break_the_two_grid_symbol(monkeypatch):
    def wrong(nf, per):
        nc = nf // 2
        rows, cols, vals = [], [], []
        for K in range(nc):
            for off in (-1, 0, 1):
                rows.append(K); cols.append((2 * K + off) % nf); vals.append(1 / 3)
        return sp.csr_matrix((vals, (rows, cols)), shape=(nc, nf))
    monkeypatch.setattr(tr, "_r_face", wrong)
    _fails(tt.test_coarse_grid_correction_matches_two_grid_symbol, 2, 2.0 / 3.0)


def test_planted_transposed_vanka_block_breaks_cell_exactness(monkeypatch):
    orig = sm.cell_blocks
    monkeypatch.setattr(oracle, "cell_blocks", lambda H, idx: np.transpose(orig(H, idx), (0, 2, 1)))
    _fails(tsol.test_vanka_single_cell_with_unit_damping_zeroes_its_residuals, (8, 6))


def test_planted_conjugation_error_in_gram_schmidt_breaks_the_krylov_pin(monkeypatch):
    real_vdot = np.vdot

    class NP:
        def __getattr__(self, k):
            return getattr(np, k)

        @staticmethod
        def vdot(a, b):
            return real_vdot(b, a)
    monkeypatch.setattr(kr, "np", NP())
    _fails(tsol.test_fgmres_with_identity_preconditioner_matches_numpy_solve)


def test_material_coarsening_is_exact_for_linear_media():
    """Reading: coarse media are the mean of the 2^d children -- exact for linear fields."""
    n = (8, 4, 6)
    z, y, x = np.meshgrid(*[np.arange(v) + 0.5 for v in n[::-1]], indexing="ij")
    f = 1.0 + 0.3 * x - 0.2 * y + 0.7 * z
    pb = disc.Problem(n, 1.0, 1.0, 0.0, 2 / 3, f, f, f)
    c = oracle.coarsen(pb)
    zc, yc, xc = np.meshgrid(*[2 * (np.arange(v) + 0.5) for v in c.n[::-1]], indexing="ij")
    np.testing.assert_allclose(c.mu, 1.0 + 0.3 * xc - 0.2 * yc + 0.7 * zc, atol=1e-13)


# ---------------------------------------------------------------- adjoint-state gradient
import oracle.adjoint as adj
import test_oracle_adjoint as tadj


def test_planted_missing_absorbing_layer_in_the_mass_derivative_breaks_the_fd_pin(monkeypatch):
    monkeypatch.setattr(adj, "gamma_abl", lambda pb, comp: np.zeros(tuple(pb.n[::-1])))
    _fails(tadj.test_gradient_matches_central_differences_cell_by_cell, "rho")


def test_planted_two_cell_node_average_breaks_the_fd_pin(monkeypatch):
    orig = adj.average_matrix
    monkeypatch.setattr(adj, "average_matrix", lambda pb, axes, counts: orig(pb, axes[:1], counts))
    _fails(tadj.test_gradient_matches_central_differences_cell_by_cell, "mu")


def test_planted_unconjugated_adjoint_breaks_the_fd_pin(monkeypatch):
    orig = adj.material_derivative
    monkeypatch.setattr(adj, "material_derivative", lambda pb, u, a, shift=0.0: orig(pb, u, np.conj(a), shift))
    _fails(tadj.test_gradient_matches_central_differences_in_a_random_direction, (12, 10), 2, "mu")


# ---------------------------------------------------------------- LFA tool (pins against the oracle)
import paper_2307_03242_gb300.lfa as lfa
import test_lfa as tl


def test_planted_wrong_relaxation_order_breaks_the_lexicographic_symbol_pin(monkeypatch):
    """Cells of the same row relaxed after the cell counted as relaxed before it."""
    def wrong(s, theta):
        st = lfa.operator_stencil(s, s.h)
        L = np.zeros((theta.shape[0], 5, 5), dtype=np.complex128)
        for a, (ca, oa) in enumerate(lfa.CELL):
            for b, (cb, ob) in enumerate(lfa.CELL):
                for d, coef in st.get((ca, cb), {}).items():
                    e = (d[0] - ob[0] + oa[0], d[1] - ob[1] + oa[1])
                    if e[1] < 0 or (e[1] == 0 and e[0] != 0):
                        L[:, a, b] += coef * lfa._phase(theta, e)
        return L
    monkeypatch.setattr(lfa, "_earlier_coupling", wrong)
    _fails(tl.test_lexicographic_symbol_matches_oracle_sweep_away_from_the_start, "economic")


def test_planted_swapped_prolongation_weights_break_the_coarse_correction_pin(monkeypatch):
    orig = lfa._transfer_taps

    def wrong(comp, axis, kind):
        t = orig(comp, axis, kind)
        if kind == "P" and comp != axis:
            return {-1: 0.75, 0: 0.25, 1: 0.25, 2: 0.75}
        return t
    monkeypatch.setattr(lfa, "_transfer_taps", wrong)
    _fails(tl.test_coarse_correction_symbol_matches_oracle, 2.0 / 3.0, np.pi / 5, 0.15)


def test_planted_colour_sign_breaks_the_red_black_symbol_pin(monkeypatch):
    orig = lfa.red_black_symbol

    def wrong(s, theta):
        out = orig(s, theta)
        out[:, :3, 3:] *= -1.0  # the coupling between theta and theta + (pi, pi) with the wrong sign
        out[:, 3:, :3] *= -1.0
        return out
    monkeypatch.setattr(lfa, "red_black_symbol", wrong)
    _fails(tl.test_red_black_symbol_matches_oracle_sweep, "full", 2.0 / 3.0, np.pi / 5, 0.15)


def test_planted_second_recursive_call_from_zero_breaks_the_wcycle_pin(monkeypatch):
    """A W-cycle whose second recursive call starts from zero instead of from the first call's
    result computes the V-cycle's correction; the closed-form W propagator must catch it."""
    import oracle.multigrid as mg
    import test_oracle_wcycle as tw

    def wrong(hier, b, x=None, level=0):
        b = np.asarray(b, dtype=np.complex128).ravel()
        if level == hier.levels - 1:
            return hier.coarse_solve(b)
        x = np.zeros_like(b) if x is None else np.asarray(x, dtype=np.complex128).ravel().copy()
        x = hier.smooth(level, b, x, hier.nu_pre, hier.w[level])
        bc = hier.R[level] @ (b - hier.H[level] @ x)
        ec = wrong(hier, bc, None, level + 1)
        for _ in range(hier.gamma_cycle - 1):
            if level + 1 < hier.levels - 1:
                ec = wrong(hier, bc, None, level + 1)  # the mistake: restarts from zero
        x = x + hier.P[level] @ ec
        return hier.smooth(level, b, x, hier.nu_post, hier.w[level])
    monkeypatch.setattr(mg, "vcycle", wrong)
    _fails(tw.test_wcycle_equals_closed_form_error_propagator_with_exact_coarsest, (1, 1))


def test_planted_coarsest_solved_twice_breaks_the_once_per_visit_pin(monkeypatch):
    """A textbook W-cycle that also repeats the inexact coarsest solve on the level above it
    departs from the reading the pin fixes."""
    import oracle.multigrid as mg
    import test_oracle_wcycle as tw
    orig = mg.vcycle

    def wrong(hier, b, x=None, level=0):
        if level == hier.levels - 2 and hier.cycle == "W":
            b = np.asarray(b, dtype=np.complex128).ravel()
            x = np.zeros_like(b) if x is None else np.asarray(x, dtype=np.complex128).ravel().copy()
            x = hier.smooth(level, b, x, hier.nu_pre, hier.w[level])
            bc = hier.R[level] @ (b - hier.H[level] @ x)
            last = hier.levels - 1
            ec = hier.coarse_solve(bc)
            # the mistake: a second coarsest solve, continuing from the first one's result
            ec = hier.smooth(last, bc, ec, hier.coarse_sweeps, hier.coarse_damping)
            x = x + hier.P[level] @ ec
            return hier.smooth(level, b, x, hier.nu_post, hier.w[level])
        return orig(hier, b, x, level)
    monkeypatch.setattr(mg, "vcycle", wrong)
    _fails(tw.test_wcycle_solves_an_inexact_coarsest_level_once_per_visit)


# ---------------------------------------------------------------- hybrid Kaczmarz coarsest solve
import oracle.kaczmarz as kz
import test_oracle_kaczmarz as tk


def _planted_step(monkeypatch, tmp_path, old, new):
    """Builds oracle/kaczmarz.c with `old` replaced by `new` and makes it the step in use."""
    import os
    src = open(os.path.join(os.path.dirname(kz.__file__), "kaczmarz.c")).read()
    assert src.count(old) >= 1
    path = tmp_path / "planted.c"
    path.write_text(src.replace(old, new))
    monkeypatch.setattr(kz, "_STEP", kz.load_step(str(tmp_path / "planted.so"), str(path)))


def test_planted_missing_conjugate_breaks_the_projection_pin(monkeypatch, tmp_path):
    _planted_step(monkeypatch, tmp_path, "ai = -v[2 * q + 1]", "ai = v[2 * q + 1]")
    _fails(tk.test_projection_property_on_the_schur_rows, (10, 8))


def test_planted_average_over_all_subregions_breaks_the_fixed_point_pin(monkeypatch, tmp_path):
    _planted_step(monkeypatch, tmp_path, "acc[2 * j] / cnt[j]", "acc[2 * j] / nparts")
    _fails(tk.test_exact_solution_is_a_fixed_point, (10, 8), 2)


def test_planted_undamped_update_breaks_bjorck_elfving(monkeypatch, tmp_path):
    _planted_step(monkeypatch, tmp_path, "sr = w * rr / nn, si = w * ri / nn", "sr = rr / nn, si = ri / nn")
    _fails(tk.test_bjorck_elfving_sor_identity, 0.8)


def test_planted_shared_copy_across_subregions_breaks_the_hand_average(monkeypatch, tmp_path):
    # sub-regions start from the previous sub-region's copy instead of the common iterate
    _planted_step(monkeypatch, tmp_path, "work[2 * j] = x[2 * j];\n      work[2 * j + 1] = x[2 * j + 1];",
                  "if (p == 0) { work[2 * j] = x[2 * j];\n      work[2 * j + 1] = x[2 * j + 1]; }")
    _fails(tk.test_hand_examples_of_projection_and_component_average)


def test_planted_schur_sign_breaks_the_direct_solve_pin(monkeypatch):
    monkeypatch.setattr(kz, "_eliminate", lambda Huu, A_up, cinv, A_pu: (Huu + A_up @ sp.diags(cinv) @ A_pu).tocsr())
    _fails(tk.test_schur_reduction_reproduces_the_direct_solve, (10, 8))


def test_planted_narrow_reach_breaks_the_footprint_pin(monkeypatch):
    monkeypatch.setattr(kz, "reach_offsets", lambda d, c: ((1,) * d, (1,) * d))
    _fails(tk.test_reach_is_the_schur_stencil_footprint, (10, 8))


def test_planted_unorthogonalised_second_gcr_direction_breaks_the_least_squares_pin(monkeypatch):
    """K-cycle with the second search direction not orthogonalised against the first."""
    import oracle.multigrid as mg

    def kcycle_no_orth(hier, r, level):
        A = hier.H[level]
        z1 = mg.vcycle(hier, r, None, level)
        q1 = A @ z1
        a1 = np.vdot(q1, r) / np.vdot(q1, q1).real
        r2 = r - a1 * q1
        z2 = mg.vcycle(hier, r2, None, level)
        q2 = A @ z2
        a2 = np.vdot(q2, r2) / np.vdot(q2, q2).real
        return a1 * z1 + a2 * z2

    monkeypatch.setattr(mg, "kcycle_correction", kcycle_no_orth)
    _fails(tsol.test_kcycle_correction_is_the_least_squares_combination_of_its_two_cycles)
