"""Per-cell functions of the CUDA kernels, compiled for the host and looped over the cells
(libemg_hostcheck.so), against the FP64 oracle, on the CPU:
* the adjoint (csrc/adjoint.cuh): y = H^H x against the oracle's assembled conjugate transpose,
  the material derivative -Re a^H (dH/dm) u against oracle/adjoint.py;
* the 2D hot path: the red-black half-sweep (csrc/vanka2d_fast.cuh) and the residual and
  restriction (csrc/residual2d_fast.cuh), each with the kernel's per-cell choice among its
  general, interior and attenuation-free variants and the library's absorbing-layer tables,
  against the oracle's red-black sweep and R (b - H_s x), in FP64 and FP32.
These are the functions the GPU kernels run; the GPU tests check the launches."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.adjoint import material_derivative
from oracle.discretization import replace
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


# ---------------------------------------------------------------- forward 2D kernels, host build
from oracle.smoother import red_black_sweep
from _gpu_helpers import oracle_hierarchy, random_field

FWD = {"2d": ((72, 40), 3, 5), "2d_odd_coarse": ((36, 20), 3, 3)}


def _level_args(pb, hier, level, prec):
    pl = hier.pbs[level]
    n = np.array(list(pl.n) + [1], dtype=np.int32)
    mats = [np.ascontiguousarray(pl.mu.ravel()), np.ascontiguousarray(pl.rho.ravel()),
            np.ascontiguousarray((1.0 / (pl.lam + pl.mu)).ravel())]
    head = [prec, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pl.h), ctypes.c_double(pb.beta),
            ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma + hier.alphas[level]),
            ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max), ctypes.c_double(pb.domain[0]),
            ctypes.c_double(pb.domain[1])] + [m.ctypes.data_as(DP) for m in mats]
    return head, (n, mats)


@pytest.mark.parametrize("case", list(FWD))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("level", [0, 1])
@pytest.mark.parametrize("sweeps,zero_first", [(1, 0), (2, 0), (2, 1)])
def test_host_red_black_vanka_matches_the_oracle(hc, case, prec, level, sweeps, zero_first):
    """The 2D half-sweep's three variants (general, interior, interior without the absorbing
    layer), chosen per cell as the kernel chooses them, against the oracle's red-black sweep."""
    n, levels, abl = FWD[case]
    w = small_heterogeneous(n, seed=1, levels=levels, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    pl = hier.pbs[level]
    b, x = random_field(pl, 21), random_field(pl, 22)
    if zero_first:
        x = np.zeros_like(x)
    ref = x.ravel()
    for _ in range(sweeps):
        ref = red_black_sweep(hier.H[level], hier.V[level], hier.idx[level], hier.colour[level], b.ravel(), ref,
                              hier.w[level])
    got = np.ascontiguousarray(x.ravel()).copy()
    if zero_first:
        got[:] = np.nan  # a zero initial guess must not be read
    head, keep = _level_args(pb, hier, level, prec)
    bb = np.ascontiguousarray(b.ravel())
    assert hc.emg_hc_vanka2_sweeps(*head, _cvec(bb), _cvec(got), ctypes.c_double(hier.w[level]), sweeps,
                                   zero_first) == 0
    tol = 1e-12 if prec == 64 else 1e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("case", list(FWD))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("level", [0, 1])
def test_host_residual_restriction_matches_the_oracle(hc, case, prec, level):
    n, levels, abl = FWD[case]
    w = small_heterogeneous(n, seed=1, levels=levels, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    pl = hier.pbs[level]
    b, x = random_field(pl, 31), random_field(pl, 32)
    ref = hier.R[level] @ (b.ravel() - hier.H[level] @ x.ravel())
    bc = np.zeros(ref.size, dtype=np.complex128)
    head, keep = _level_args(pb, hier, level, prec)
    bb, xx = np.ascontiguousarray(b.ravel()), np.ascontiguousarray(x.ravel())
    assert hc.emg_hc_residual_restrict2(*head, _cvec(bb), _cvec(xx), _cvec(bc)) == 0
    tol = 1e-12 if prec == 64 else 2e-5
    assert np.abs(bc - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n,abl", [((20, 10, 6), 2), ((16, 8, 4), 0), ((18, 9, 7), 3)])
@pytest.mark.parametrize("sweeps,zero_first", [(1, 0), (2, 1)])
def test_host_3d_tile_sweep_matches_the_oracle(hc, prec, n, abl, sweeps, zero_first):
    """The 3D shared-memory tile half-sweep (csrc/vanka3d_tile.cuh: 16 x 8 x 4 cells per block,
    halo box, parity de-interleaved columns), its blocks run one after another with the library's
    ping-pong of the displacements, against the oracle's red-black sweep. The grids give ragged
    last tiles in every direction (20 x 10 x 6, 18 x 9 x 7) and a single tile (16 x 8 x 4)."""
    from oracle.smoother import cell_dofs, cell_blocks, cell_colour
    w = small_heterogeneous(n, seed=12, levels=1, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    alpha, wd = 0.4, 0.3
    H = oracle.assemble(pb, alpha)
    idx = cell_dofs(pb)
    V = cell_blocks(H, idx)
    b, x = random_field(pb, 91), random_field(pb, 92)
    if zero_first:
        x = np.zeros_like(x)
    ref = x.ravel()
    for _ in range(sweeps):
        ref = red_black_sweep(H, V, idx, cell_colour(pb), b.ravel(), ref, wd)
    got = np.ascontiguousarray(x.ravel()).copy()
    if zero_first:
        got[:] = np.nan  # a zero initial guess must not be read
    nn = np.array(n, dtype=np.int32)
    mats = [np.ascontiguousarray(pb.mu.ravel()), np.ascontiguousarray(pb.rho.ravel()),
            np.ascontiguousarray((1.0 / (pb.lam + pb.mu)).ravel())]
    bb = np.ascontiguousarray(b.ravel())
    assert hc.emg_hc_vanka3_tile_sweeps(prec, nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                                        ctypes.c_double(pb.beta), ctypes.c_double(pb.omega),
                                        ctypes.c_double(pb.gamma + alpha), ctypes.c_double(pb.abl_length),
                                        ctypes.c_double(pb.abl_gamma_max), *[ctypes.c_double(v) for v in pb.domain],
                                        *[m.ctypes.data_as(DP) for m in mats], _cvec(bb), _cvec(got),
                                        ctypes.c_double(wd), sweeps, zero_first) == 0
    tol = 1e-12 if prec == 64 else 2e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("n,abl", [((12, 10, 9), 2), ((16, 8, 8), 3)])
def test_host_3d_residual_matches_the_oracle(hc, prec, n, abl):
    """The 3D residual kernel's interior variants (the register cube with and without the
    absorbing layer) and its boundary rows, chosen per cell as the kernel chooses them."""
    w = small_heterogeneous(n, seed=6, levels=2, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    alpha = 0.4
    b, x = random_field(pb, 41), random_field(pb, 42)
    ref = b.ravel() - oracle.assemble(pb, alpha) @ x.ravel()
    nn = np.array(n, dtype=np.int32)
    mats = [np.ascontiguousarray(pb.mu.ravel()), np.ascontiguousarray(pb.rho.ravel()),
            np.ascontiguousarray((1.0 / (pb.lam + pb.mu)).ravel())]
    r = np.zeros_like(ref)
    bb, xx = np.ascontiguousarray(b.ravel()), np.ascontiguousarray(x.ravel())
    assert hc.emg_hc_residual3(prec, nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                               ctypes.c_double(pb.beta), ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma + alpha),
                               ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max),
                               *[ctypes.c_double(v) for v in pb.domain], *[m.ctypes.data_as(DP) for m in mats],
                               _cvec(bb), _cvec(xx), _cvec(r)) == 0
    act = oracle.active_mask(pb)
    tol = 1e-12 if prec == 64 else 2e-5
    assert np.abs((r - ref) * act).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shift", [0.0, 0.4])
@pytest.mark.parametrize("n,abl", [((12, 10, 9), 2), ((7, 6, 5), 1)])
def test_host_3d_float_float_apply_matches_the_oracle(hc, shift, n, abl):
    """The outer solve's 3D FP64 apply in double-FP32 arithmetic on the library's host-built
    coefficients: FP64 accuracy (about 48 significant bits) against the oracle's operator."""
    w = small_heterogeneous(n, seed=7, levels=2, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    x = random_field(pb, 51)
    ref = oracle.assemble(pb, shift) @ x.ravel()
    nn = np.array(n, dtype=np.int32)
    L = np.array(pb.domain, dtype=np.float64)
    mats = [np.ascontiguousarray(a.ravel()) for a in (pb.lam, pb.mu, pb.rho)]
    y = np.zeros_like(ref)
    xx = np.ascontiguousarray(x.ravel())
    assert hc.emg_hc_apply_ff3(nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                               ctypes.c_double(pb.beta), ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma),
                               ctypes.c_double(shift), ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max),
                               L.ctypes.data_as(DP), *[m.ctypes.data_as(DP) for m in mats], _cvec(xx), _cvec(y)) == 0
    act = oracle.active_mask(pb)
    assert np.abs((y - ref) * act).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,abl", [((12, 10, 9), 2), ((7, 6, 5), 1), ((6, 6, 6), 0)])
def test_host_3d_float_float_adjoint_apply_matches_the_oracle(hc, n, abl):
    """y = H^H x in double-FP32 arithmetic on the forward apply's coefficient arrays (the
    transpose of its 27-point expansion) against the oracle's conjugate transpose."""
    w = small_heterogeneous(n, seed=8, levels=2, abl_cells=max(abl, 1), sigma_cells=2.0)
    pb = oracle_problem(w)
    if abl == 0:
        pb = replace(pb, abl_length=0.0)
    x = random_field(pb, 61)
    ref = oracle.assemble(pb, 0.0).conj().T @ x.ravel()
    nn = np.array(n, dtype=np.int32)
    L = np.array(pb.domain, dtype=np.float64)
    mats = [np.ascontiguousarray(a.ravel()) for a in (pb.lam, pb.mu, pb.rho)]
    y = np.zeros_like(ref)
    xx = np.ascontiguousarray(x.ravel())
    assert hc.emg_hc_apply_adjoint_ff3(nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                                       ctypes.c_double(pb.beta), ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma),
                                       ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max),
                                       L.ctypes.data_as(DP), *[m.ctypes.data_as(DP) for m in mats], _cvec(xx),
                                       _cvec(y)) == 0
    act = oracle.active_mask(pb)
    assert np.abs((y - ref) * act).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------- one-pass tiled sweep, host build
TILED = {"72x40": ((72, 40), 3, 5), "200x64": ((200, 64), 2, 5), "124x36_layer": ((124, 36), 2, 12)}


@pytest.mark.parametrize("ty", [24, 8, 4])
@pytest.mark.parametrize("case", list(TILED))
@pytest.mark.parametrize("level", [0, 1])
@pytest.mark.parametrize("sweeps,zero_first", [(1, 0), (2, 1)])
def test_host_tiled_sweep_matches_the_oracle(hc, case, level, sweeps, zero_first, ty):
    """The one-pass tiled sweep (csrc/sweep2d_tile.cuh): tile decomposition, shared-region
    boundary handling, both colour phases and the lane mapping, against the oracle's red-black
    sweep in FP32. The 200 x 64 grid has tiles away from the boundary and the absorbing layer
    (the interior, attenuation-free variant); shared entries the kernel would read unwritten are
    NaN in the host build."""
    n, levels, abl = TILED[case]
    w = small_heterogeneous(n, seed=3, levels=levels, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    pl = hier.pbs[level]
    if pl.n[0] % 4:
        pytest.skip("the tiled kernel needs n_x divisible by 4")
    b, x = random_field(pl, 41), random_field(pl, 42)
    if zero_first:
        x = np.zeros_like(x)
    ref = x.ravel()
    for _ in range(sweeps):
        ref = red_black_sweep(hier.H[level], hier.V[level], hier.idx[level], hier.colour[level], b.ravel(), ref,
                              hier.w[level])
    got = np.ascontiguousarray(x.ravel()).copy()
    if zero_first:
        got[:] = np.nan  # a zero initial guess must not be read
    head, keep = _level_args(pb, hier, level, 32)
    bb = np.ascontiguousarray(b.ravel())
    interior = hc.emg_hc_sweep_tiled(*head[1:], _cvec(bb), _cvec(got), ctypes.c_double(hier.w[level]), sweeps,
                                     zero_first, ty)
    assert interior >= 0
    if case == "200x64" and level == 0:
        assert interior >= 2
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("ty", [24, 8, 4])
@pytest.mark.parametrize("case", ["72x40", "200x64"])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_host_tiled_sweep_with_prolongation_matches_the_oracle(hc, case, sweeps, ty):
    """The first post-sweep with the prolongation + correction fused into its tile loads:
    x + P e, then the sweeps, against the oracle's P and red-black sweep in FP32."""
    n, levels, abl = TILED[case]
    w = small_heterogeneous(n, seed=5, levels=levels, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    pl, pc = hier.pbs[0], hier.pbs[1]
    b, x, e = random_field(pl, 51), random_field(pl, 52), random_field(pc, 53)
    ref = x.ravel() + hier.P[0] @ e.ravel()
    for _ in range(sweeps):
        ref = red_black_sweep(hier.H[0], hier.V[0], hier.idx[0], hier.colour[0], b.ravel(), ref, hier.w[0])
    got = np.ascontiguousarray(x.ravel()).copy()
    head, keep = _level_args(pb, hier, 0, 32)
    bb, ee = np.ascontiguousarray(b.ravel()), np.ascontiguousarray(e.ravel())
    assert hc.emg_hc_prolong_sweep_tiled(*head[1:], _cvec(bb), _cvec(ee), _cvec(got), ctypes.c_double(hier.w[0]),
                                         sweeps, ty) == 0
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_float_float_split_and_join_are_exact_to_46_bits(hc):
    """df::split (integer and FP32 operations only) gives hi = x truncated to 24 significant bits
    and hi + lo within 2^-46 |x|; df::join / widen reassemble doubles exactly; non-finite values
    stay non-finite."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, -2.0, 2.0 ** -100, 3.0 * 2.0 ** 80, 1e-35, np.inf, -np.inf, np.nan]])
    n = x.size
    hi, lo = np.zeros(n, np.float32), np.zeros(n, np.float32)
    joined, widened = np.zeros(n), np.zeros(n)
    fp = ctypes.POINTER(ctypes.c_float)
    assert hc.emg_hc_split_join(x.ctypes.data_as(DP), n, hi.ctypes.data_as(fp), lo.ctypes.data_as(fp),
                                joined.ctypes.data_as(DP), widened.ctypes.data_as(DP)) == 0
    fin = np.isfinite(x) & (np.abs(x) > 1e-30)
    h64, l64 = hi.astype(np.float64), lo.astype(np.float64)
    assert np.all(np.abs(h64[fin]) <= np.abs(x[fin]))                                   # truncation
    assert np.all(np.abs(x[fin] - h64[fin]) < np.spacing(np.abs(hi[fin])).astype(np.float64))
    assert np.all(np.abs((h64 + l64 - x)[fin]) <= 2.0 ** -46 * np.abs(x[fin]))
    assert np.array_equal(joined[fin], (h64 + l64)[fin])
    assert np.array_equal(widened[np.isfinite(x)], h64[np.isfinite(x)])
    assert np.isnan(hi[-1]) and np.isinf(hi[-2]) and np.isinf(hi[-3]) and hi[-3] > 0 > hi[-2]
    assert hi[-10] == 0 and lo[-10] == 0


@pytest.mark.parametrize("bscale", [None, 0.125, 0.3])
@pytest.mark.parametrize("x32", [0, 1])
@pytest.mark.parametrize("n", [(14, 11), (9, 8, 7), (6, 6, 6)])
def test_host_float_float_residual_form_matches_the_oracle(hc, n, x32, bscale):
    """The outer apply's residual form y = bscale b - H x (the true residual at every restart):
    float-float throughout when bscale is a power of two (the split b is scaled exactly), FP64
    otherwise; x in FP64 or FP32; 2D and 3D; against the oracle's operator to 1e-12."""
    w = small_heterogeneous(n, seed=9, levels=2, abl_cells=2, sigma_cells=2.0)
    pb = oracle_problem(w)
    x = random_field(pb, 81).ravel()
    if x32:
        x = x.astype(np.complex64).astype(np.complex128)
    H = oracle.assemble(pb, 0.0)
    act = oracle.active_mask(pb)
    b = random_field(pb, 82).ravel() * 50.0
    ref = H @ x if bscale is None else (bscale * b - H @ x) * act
    nn = np.array(n + (1,) * (3 - len(n)), dtype=np.int32)
    L = np.array(tuple(pb.domain) + (1.0,) * (3 - len(n)), dtype=np.float64)
    mats = [np.ascontiguousarray(a.ravel()) for a in (pb.lam, pb.mu, pb.rho)]
    y = np.zeros_like(ref)
    xx, bb = np.ascontiguousarray(x), np.ascontiguousarray(b)
    assert hc.emg_hc_residual_ff(len(n), nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                                 ctypes.c_double(pb.beta), ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma),
                                 ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max), L.ctypes.data_as(DP),
                                 *[m.ctypes.data_as(DP) for m in mats], _cvec(xx),
                                 None if bscale is None else _cvec(bb), ctypes.c_double(bscale or 0.0), _cvec(y),
                                 x32) == 0
    scale = max(np.abs(H @ x).max(), np.abs(ref).max())
    assert np.abs((y - ref) * act).max() <= 1e-12 * scale
    assert np.all(y[~act.astype(bool)] == 0)


def test_float_float_join_is_within_one_ulp_of_the_exact_sum(hc):
    """df::join (TwoSum, then integer operations on the bits: no FP64 instruction) returns hi + lo
    truncated to a double: within one ulp of the exact sum (computed with fractions), exact where
    the sum fits in 53 bits. Pairs: normalised (|lo| <= ulp(hi)/2), opposite signs, powers of two
    with a lo of the other sign (the sum falls into the binade below), unnormalised pairs (lo as
    large as hi), subnormal parts, zeros and non-finite values."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    m = 4000
    hi = (rng.standard_normal(m) * 10.0 ** rng.uniform(-20, 20, m)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, m) * ulp).astype(np.float32)
    p2 = np.float32(2.0) ** rng.integers(-60, 60, 500).astype(np.float32)
    p2lo = (-np.sign(p2) * rng.uniform(0, 0.25, 500) * np.spacing(p2).astype(np.float64)).astype(np.float32)
    big = rng.standard_normal(500).astype(np.float32)
    biglo = (rng.standard_normal(500) * 10.0 ** rng.uniform(-9, 0, 500)).astype(np.float32)
    tiny = np.array([1e-45, -3e-42, 1.2e-38, 2.0 ** -126, 0.0, -0.0, 1.0, 1.0], np.float32)
    tinylo = np.array([0.0, 1e-45, -1e-45, -1e-45, 0.0, 0.0, -2.0 ** -25, 2.0 ** -40], np.float32)
    H = np.concatenate([hi, p2, -p2, big, tiny])
    L = np.concatenate([lo, p2lo, -p2lo, biglo, tinylo])
    out = np.zeros(H.size)
    fp = ctypes.POINTER(ctypes.c_float)
    assert hc.emg_hc_join(H.ctypes.data_as(fp), L.ctypes.data_as(fp), H.size, out.ctypes.data_as(DP)) == 0
    for h, l, o in zip(H, L, out):
        exact = Fraction(float(h)) + Fraction(float(l))
        err = abs(Fraction(float(o)) - exact)
        assert err < Fraction(np.spacing(abs(float(o)))) or err == 0, (h, l, o)
        if float(np.float64(h) + np.float64(l)) == exact:  # the sum fits in a double: exact
            assert float(o) == float(exact), (h, l, o)
    special = np.array([np.inf, -np.inf, np.nan, 3e38], np.float32)
    out4 = np.zeros(4)
    zero = np.zeros(4, np.float32)
    assert hc.emg_hc_join(special.ctypes.data_as(fp), zero.ctypes.data_as(fp), 4, out4.ctypes.data_as(DP)) == 0
    assert out4[0] == np.inf and out4[1] == -np.inf and np.isnan(out4[2]) and out4[3] == np.float64(np.float32(3e38))


@pytest.mark.parametrize("ty", [24, 8, 4])
@pytest.mark.parametrize("case", list(TILED))
@pytest.mark.parametrize("level", [0, 1])
def test_host_tiled_residual_restriction_matches_the_oracle(hc, case, level, ty):
    """The one-pass residual + restriction (csrc/residual2d_tile.cuh): the fine residual's
    displacement rows in shared memory, restricted there, the pressure rows formed on the fly,
    against the oracle's R (b - H_s x) in FP32; shared entries it would read unwritten are NaN."""
    n, levels, abl = TILED[case]
    w = small_heterogeneous(n, seed=6, levels=levels, abl_cells=abl, sigma_cells=2.0)
    pb = oracle_problem(w)
    hier = oracle_hierarchy(w, pb)
    pl = hier.pbs[level]
    if pl.n[0] % 4 or level + 1 >= levels:
        pytest.skip("needs n_x divisible by 4 and a coarser level")
    b, x = random_field(pl, 61), random_field(pl, 62)
    ref = hier.R[level] @ (b.ravel() - hier.H[level] @ x.ravel())
    bc = np.zeros(ref.size, dtype=np.complex128)
    head, keep = _level_args(pb, hier, level, 32)
    bb, xx = np.ascontiguousarray(b.ravel()), np.ascontiguousarray(x.ravel())
    assert hc.emg_hc_resid_restrict_tiled(*head[1:], _cvec(bb), _cvec(xx), _cvec(bc), ty) == 0
    assert np.all(np.isfinite(bc))
    assert np.abs(bc - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("n,abl,shift", [((40, 24), 4, 0.0), ((17, 11), 2, 0.3), ((12, 12), 0, 0.0)])
@pytest.mark.parametrize("x32", [0, 1])
def test_host_2d_float_float_apply_matches_the_oracle(hc, n, abl, shift, x32):
    """y = H x (or H_s x) in double-FP32 arithmetic, the rows factored into exact differences of
    the inputs weighted by mu and the spread weights (csrc/apply_ff2d.cuh), against the oracle's
    assembled operator in FP64: x in FP64, or rounded to FP32 as the cycle's output is."""
    w = small_heterogeneous(n, seed=9, levels=1, abl_cells=max(abl, 1), sigma_cells=2.0)
    pb = oracle_problem(w)
    if abl == 0:
        pb = replace(pb, abl_length=0.0)
    x = random_field(pb, 71).ravel()
    if x32:
        x = x.astype(np.complex64).astype(np.complex128)
    ref = oracle.assemble(pb, shift) @ x
    nn = np.array(n, dtype=np.int32)
    mats = [np.ascontiguousarray(a.ravel()) for a in (pb.lam, pb.mu, pb.rho)]
    y = np.zeros_like(ref)
    xx = np.ascontiguousarray(x)
    assert hc.emg_hc_apply_ff2(nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_double(pb.h),
                               ctypes.c_double(pb.beta), ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma),
                               ctypes.c_double(shift), ctypes.c_double(pb.abl_length),
                               ctypes.c_double(pb.abl_gamma_max), *[m.ctypes.data_as(DP) for m in mats], _cvec(xx),
                               _cvec(y), x32) == 0
    act = oracle.active_mask(pb)
    assert np.abs((y - ref) * act).max() <= 1e-12 * np.abs(ref).max()
