"""The hybrid Kaczmarz coarsest solve's host-callable parts (csrc/kaczmarz.cuh) against the
oracle (oracle/kaczmarz.py), on the CPU: the Schur rows formed by probing the level operator,
the slot layout of a stored row, and Kaczmarz steps run with the kernel's box geometry, region
index tables, row order and component average (lanes taken in turn); every region index is
checked to lie in its box's region and to map back to the entry's unknown."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import kaczmarz as kz
from workloads import small_heterogeneous
from _gpu_helpers import oracle_problem

DP = ctypes.POINTER(ctypes.c_double)
IP = ctypes.POINTER(ctypes.c_int)


@pytest.fixture(scope="module")
def hc():
    from paper_2307_03242_gb300.build import build_hostcheck
    lib = ctypes.CDLL(build_hostcheck())
    lib.emg_hc_kz_steps.restype = ctypes.c_long
    return lib


def _cvec(v):
    return v.view(np.float64).ctypes.data_as(DP)


def stored_rows(hc, sysm):
    """The oracle's S in the library's stored layout: dim N rows (component-major, boundary faces
    included as zero rows) x NE footprint entries."""
    pb = sysm.pb
    d, N = pb.dim, pb.ncell
    ne = 75 if d == 3 else 17
    rows = np.zeros((d * N, ne), dtype=np.complex128)
    S = sysm.S.tocoo()
    fr, fc = sysm.u_act[S.row], sysm.u_act[S.col]
    cr, kr = np.divmod(fr, N)
    cc, kc = np.divmod(fc, N)

    def coords(k):
        out = []
        for a in range(3):
            if a < d:
                out.append(k % pb.n[a])
                k = k // pb.n[a]
            else:
                out.append(np.zeros_like(k))
        return out

    pr, pc = coords(kr), coords(kc)
    for t in range(S.nnz):
        o = [int(pc[a][t] - pr[a][t]) for a in range(3)]
        slot = hc.emg_hc_kz_slot(d, int(cr[t]), int(cc[t]), *o)
        assert slot >= 0
        rows[fr[t], slot] = S.data[t]
    return rows


def _full(sysm, v):
    out = np.zeros(sysm.nu, dtype=np.complex128)
    out[sysm.u_act] = v
    return out


def _problem(n, seed, abl):
    w = small_heterogeneous(n, seed=seed, levels=1, abl_cells=abl, sigma_cells=2.0)
    return oracle_problem(w)


@pytest.mark.parametrize("n,abl", [((9, 7, 6), 2), ((8, 8, 8), 0), ((11, 9), 2)])
def test_probed_schur_rows_match_the_oracle(hc, n, abl):
    """Probing the level operator with the 4^d residue classes per component recovers every entry
    of S = A_uu - A_up C^-1 A_pu, and nothing else."""
    pb = _problem(n, 3, abl)
    alpha = 0.4
    sysm = kz.SchurSystem(pb, alpha)
    ref = stored_rows(hc, sysm)
    d = pb.dim
    nn = np.array(list(n) + [1] * (3 - d), dtype=np.int32)
    mats = [np.ascontiguousarray(pb.mu.ravel()), np.ascontiguousarray(pb.rho.ravel()),
            np.ascontiguousarray((1.0 / (pb.lam + pb.mu)).ravel())]
    got = np.zeros_like(ref)
    L = list(pb.domain) + [0.0] * (3 - d)
    assert hc.emg_hc_kz_probe(d, nn.ctypes.data_as(IP), ctypes.c_double(pb.h), ctypes.c_double(pb.beta),
                              ctypes.c_double(pb.omega), ctypes.c_double(pb.gamma + alpha),
                              ctypes.c_double(pb.abl_length), ctypes.c_double(pb.abl_gamma_max),
                              *[ctypes.c_double(v) for v in L], *[m.ctypes.data_as(DP) for m in mats],
                              _cvec(got)) == 0
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.count_nonzero(got) == np.count_nonzero(ref)


@pytest.mark.parametrize("n,box", [((9, 7, 6), (2, 2, 2)), ((8, 8, 8), (4, 2, 3)), ((10, 9, 5), (3, 3, 3)),
                                   ((11, 9), (2, 2)), ((16, 12), (4, 3)), ((6, 5, 4), (2, 2, 3)), ((7, 6, 9), (5, 6, 2)),
                                   ((6, 5, 4), (1, 1, 1)), ((9, 7), (1, 1))])
def test_kernel_kaczmarz_steps_match_the_oracle(hc, n, box):
    """Three steps with the kernel's geometry equal the oracle's component-averaged Kaczmarz steps
    over the same boxes (ragged boxes at the far ends included)."""
    pb = _problem(n, 5, 1)
    sysm = kz.SchurSystem(pb, 0.4)
    rows = stored_rows(hc, sysm)
    rng = np.random.default_rng(9)
    m = sysm.S.shape[0]
    rhs = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    x0 = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    ref = kz.kaczmarz_steps(sysm.S, kz.box_partition(sysm, box), rhs, x0, 3, 0.8)
    d = pb.dim
    nn = np.array(list(n) + [1] * (3 - d), dtype=np.int32)
    bb = np.array(list(box) + [1] * (3 - d), dtype=np.int32)
    rf = np.ascontiguousarray(_full(sysm, rhs))
    xf = np.ascontiguousarray(_full(sysm, x0))
    bad = hc.emg_hc_kz_steps(d, nn.ctypes.data_as(IP), bb.ctypes.data_as(IP), _cvec(np.ascontiguousarray(rows)),
                             _cvec(rf), _cvec(xf), 3, ctypes.c_double(0.8))
    assert bad == 0
    assert np.linalg.norm(xf[sysm.u_act] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(np.delete(xf, sysm.u_act)).max() == 0.0


def test_params_layout_matches_the_ctypes_mirror(hc):
    from paper_2307_03242_gb300 import emg
    out = (ctypes.c_long * 15)()
    assert hc.emg_hc_params_layout(out) == 0
    P = emg._Params
    names = ["dim", "n", "h", "damping", "coarse_solver", "level_alpha", "smoother", "sweep_path", "kaczmarz_box",
             "kaczmarz_steps", "kaczmarz_damping", "coarse_tol", "coarse_restart", "kaczmarz_max"]
    assert out[0] == ctypes.sizeof(P)
    for i, nm in enumerate(names):
        assert out[i + 1] == getattr(P, nm).offset, nm
