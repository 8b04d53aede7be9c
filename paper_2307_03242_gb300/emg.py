"""Thin ctypes binding of libemg.so (argument marshalling only).

Every entry point forwards to the C ABI declared in include/emg.h; torch tensors are passed as
raw device pointers and the handle runs on torch's current CUDA stream at creation time. There
is no CPU fallback: if libemg.so is missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libemg.so")
MAX_LEVELS = 10
COARSE_DENSE, COARSE_SMOOTH, COARSE_KACZMARZ = 0, 1, 2
CYCLE_V, CYCLE_W, CYCLE_K = 0, 1, 2
K_SMOOTH, K_RESTRICT, K_PROLONG, K_APPLY64, K_KRYLOV, K_COARSE = range(6)
VANKA_FULL, VANKA_ECONOMIC = 0, 1
SWEEP_AUTO, SWEEP_HALF, SWEEP_COOP, SWEEP_TILE24, SWEEP_TILE8, SWEEP_TILE4 = 0, 1, 2, 3, 4, 5
SWEEP_NAMES = {SWEEP_HALF: "half", SWEEP_COOP: "coop", SWEEP_TILE24: "tile24", SWEEP_TILE8: "tile8",
               SWEEP_TILE4: "tile4"}
K_ALL = 6

STATUS = {0: "EMG_OK", 1: "EMG_ERR_INVALID", 2: "EMG_ERR_NOMEM", 3: "EMG_ERR_CUDA", 4: "EMG_ERR_NONFINITE",
          5: "EMG_NOT_CONVERGED", 6: "EMG_ERR_TIMEOUT"}


class EmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("h", ctypes.c_double),
                ("omega", ctypes.c_double), ("gamma", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("abl_cells", ctypes.c_int32), ("abl_gamma_max", ctypes.c_double),
                ("levels", ctypes.c_int32), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("damping", ctypes.c_double * MAX_LEVELS), ("coarse_solver", ctypes.c_int32),
                ("coarse_sweeps", ctypes.c_int32), ("coarse_damping", ctypes.c_double),
                ("cycle_precision", ctypes.c_int32), ("cycle_type", ctypes.c_int32),
                ("level_alpha", ctypes.c_double * MAX_LEVELS), ("smoother", ctypes.c_int32),
                ("sweep_path", ctypes.c_int32), ("kaczmarz_box", ctypes.c_int32 * 3),
                ("kaczmarz_steps", ctypes.c_int32), ("kaczmarz_damping", ctypes.c_double),
                ("coarse_tol", ctypes.c_double), ("coarse_restart", ctypes.c_int32), ("kaczmarz_max", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_cap", ctypes.c_int32),
                ("history_len", ctypes.c_int32)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libemg.so not built (run __graft_entry__.build()): %s" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "emg_create": [ctypes.POINTER(_Params), vp, vp, vp, i32, vp, ctypes.POINTER(vp)],
        "emg_destroy": [vp],
        "emg_apply": [vp, i32, vp, vp],
        "emg_vcycle": [vp, vp, vp, i32],
        "emg_solve": [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(_Stats)],
        "emg_solve_host": [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(_Stats)],
        "emg_level_info": [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(dbl)],
        "emg_sweep_path": [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(dbl)],
        "emg_smooth": [vp, i32, vp, vp, i32],
        "emg_residual_restrict": [vp, i32, vp, vp, vp],
        "emg_prolong_correct": [vp, i32, vp, vp],
        "emg_coarse_solve": [vp, vp, vp],
        "emg_profile": [vp, i32],
        "emg_profile_read": [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(dbl)],
        "emg_smooth_noalloc": [ctypes.POINTER(_Params), vp, vp, vp, vp, vp, i32, vp],
        "emg_solve_batch": [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, i32, i32,
                            ctypes.POINTER(_Stats), i32, ctypes.POINTER(ctypes.c_int)],
        "emg_apply_adjoint": [vp, vp, vp],
        "emg_solve_adjoint": [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(_Stats)],
        "emg_material_gradient": [vp, vp, vp, vp, vp, vp, i32],
        "emg_coarse_stats": [vp, ctypes.POINTER(dbl)],
        "emg_coarse_schur_rows": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.emg_last_error.argtypes = []
    lib.emg_last_error.restype = ctypes.c_char_p
    return lib


LIB = _load()
EXPORTED = ["emg_create", "emg_destroy", "emg_last_error", "emg_apply", "emg_vcycle", "emg_solve", "emg_solve_host",
            "emg_level_info", "emg_smooth", "emg_residual_restrict", "emg_prolong_correct", "emg_coarse_solve",
            "emg_profile", "emg_profile_read", "emg_smooth_noalloc", "emg_solve_batch", "emg_apply_adjoint",
            "emg_solve_adjoint", "emg_material_gradient", "emg_sweep_path", "emg_coarse_stats",
            "emg_coarse_schur_rows"]
NOALLOC_MAX_CELLS = 262144


def _check(status, allow=(0,)):
    if status not in allow:
        raise EmgError(status, LIB.emg_last_error().decode())
    return status


@dataclass
class Params:
    n: tuple
    h: float = 1.0
    omega: float = 1.0
    gamma: float = 0.01
    alpha: float = 0.4
    beta: float = 2.0 / 3.0
    abl_cells: int = 0
    abl_gamma_max: float = 2.0
    levels: int = 2
    nu_pre: int = 2
    nu_post: int = 2
    damping: object = 0.0            # scalar or per-level list; 0 = default by depth
    coarse_solver: int = COARSE_DENSE
    coarse_sweeps: int = 0
    coarse_damping: float = 0.8
    cycle_precision: int = 32
    cycle_type: int = CYCLE_V
    level_alpha: object = None       # per-level shift list (entries <= 0 mean `alpha`)
    smoother: int = 0                # VANKA_FULL or VANKA_ECONOMIC
    sweep_path: int = 0              # SWEEP_AUTO (timed per level at creation) or a forced SWEEP_* path
    # COARSE_KACZMARZ (0: the paper's value -- 10 steps, damping 0.8, drop 0.1, FGMRES(5), at most
    # 250 Kaczmarz steps; boxes: the smallest cube of >= 2 cells the GPU can sweep all at once)
    kaczmarz_box: object = 0         # cells per axis: an int or one per axis
    kaczmarz_steps: int = 0
    kaczmarz_damping: float = 0.0
    coarse_tol: float = 0.0
    coarse_restart: int = 0
    kaczmarz_max: int = 0

    def to_c(self) -> _Params:
        p = _Params()
        p.dim = len(self.n)
        for a in range(3):
            p.n[a] = int(self.n[a]) if a < len(self.n) else 1
        p.h, p.omega, p.gamma, p.alpha, p.beta = self.h, self.omega, self.gamma, self.alpha, self.beta
        p.abl_cells, p.abl_gamma_max = int(self.abl_cells), float(self.abl_gamma_max)
        p.levels, p.nu_pre, p.nu_post = int(self.levels), int(self.nu_pre), int(self.nu_post)
        d = list(self.damping) if np.ndim(self.damping) else [float(self.damping)] * MAX_LEVELS
        for l in range(MAX_LEVELS):
            p.damping[l] = float(d[l]) if l < len(d) else 0.0
        p.coarse_solver, p.coarse_sweeps = int(self.coarse_solver), int(self.coarse_sweeps)
        p.coarse_damping, p.cycle_precision = float(self.coarse_damping), int(self.cycle_precision)
        p.cycle_type = int(self.cycle_type)
        la = list(self.level_alpha) if self.level_alpha is not None else []
        for l in range(MAX_LEVELS):
            p.level_alpha[l] = float(la[l]) if l < len(la) else 0.0
        p.smoother = int(self.smoother)
        p.sweep_path = int(self.sweep_path)
        kb = list(self.kaczmarz_box) if np.ndim(self.kaczmarz_box) else [int(self.kaczmarz_box)] * 3
        for a in range(3):
            p.kaczmarz_box[a] = int(kb[a]) if a < len(kb) else 0
        p.kaczmarz_steps, p.kaczmarz_damping = int(self.kaczmarz_steps), float(self.kaczmarz_damping)
        p.coarse_tol, p.coarse_restart, p.kaczmarz_max = float(self.coarse_tol), int(self.coarse_restart), int(self.kaczmarz_max)
        return p


def params_from_workload(w, cycle_precision=32, **over) -> Params:
    kw = dict(n=tuple(w.n), h=w.h, omega=w.omega, gamma=w.gamma, alpha=w.alpha, beta=w.beta,
              abl_cells=w.abl_cells, abl_gamma_max=w.abl_gamma_max, levels=w.levels, nu_pre=w.nu_pre,
              nu_post=w.nu_post, damping=w.damping,
              coarse_solver={"dense": COARSE_DENSE, "smooth": COARSE_SMOOTH, "kaczmarz": COARSE_KACZMARZ}[w.coarse],
              coarse_sweeps=w.coarse_sweeps, coarse_damping=w.coarse_damping, cycle_precision=cycle_precision,
              cycle_type={"V": CYCLE_V, "W": CYCLE_W, "K": CYCLE_K}[getattr(w, "cycle", "V")],
              level_alpha=w.level_alphas() if hasattr(w, "level_alphas") else None,
              smoother=VANKA_ECONOMIC if getattr(w, "smoother", "full") == "economic" else VANKA_FULL)
    kw.update(over)
    return Params(**kw)


def _ptr(t, dtype, numel, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (what, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def solve_batch(jobs, tol=1e-6, max_iter=1000, restart=20, workers=0, raise_errors=True):
    """emg_solve_batch: jobs is a list of (Solver, b, x) with complex128 CUDA tensors; the solves
    run concurrently, one host worker per distinct solver (give each solver its own stream).
    Returns one stats dict per job (with its own "status"); with raise_errors, raises on the first
    job error instead."""
    import torch
    count = len(jobs)
    hs = (ctypes.c_void_p * count)()
    bs = (ctypes.c_void_p * count)()
    xs = (ctypes.c_void_p * count)()
    for k, (s, b, x) in enumerate(jobs):
        n = s._n()
        hs[k] = s.h
        bs[k] = _ptr(b, torch.complex128, n, "b[%d]" % k)
        xs[k] = _ptr(x, torch.complex128, n, "x[%d]" % k)
    st = (_Stats * count)()
    status = (ctypes.c_int * count)()
    torch.cuda.current_stream().synchronize()  # b, x were produced on the caller's stream
    rc = LIB.emg_solve_batch(hs, count, bs, xs, tol, max_iter, restart, st, workers, status)
    if raise_errors:
        _check(rc, allow=(0, 5))
    out = []
    for k in range(count):
        d = Solver._stats(st[k], None, status[k])
        d["status"] = status[k]
        out.append(d)
    return out


def smooth_noalloc(params: Params, mu, rho, cp, b, x, sweeps, stream=None):
    """emg_smooth_noalloc: red-black Vanka sweeps on level 0 without a handle and without any
    allocation (see include/emg.h). mu, rho, cp: float32 CUDA tensors of n[0]*n[1] cells;
    b, x: complex64 CUDA tensors of 3*n[0]*n[1] entries."""
    import torch
    ncell = int(np.prod(params.n))
    if stream is None:
        stream = torch.cuda.current_stream()
    c = params.to_c()
    _check(LIB.emg_smooth_noalloc(ctypes.byref(c), _ptr(mu, torch.float32, ncell, "mu"),
                                  _ptr(rho, torch.float32, ncell, "rho"), _ptr(cp, torch.float32, ncell, "cp"),
                                  _ptr(b, torch.complex64, 3 * ncell, "b"), _ptr(x, torch.complex64, 3 * ncell, "x"),
                                  int(sweeps), ctypes.c_void_p(stream.cuda_stream)))
    return x


class Solver:
    """One multigrid hierarchy on the current CUDA device (see include/emg.h)."""

    def __init__(self, params: Params, lam, mu, rho, stream=None):
        import torch
        self.params = params
        self.dim = len(params.n)
        self.shape = tuple(int(v) for v in params.n[::-1])
        self.ncell = int(np.prod(self.shape))
        self.cdtype = torch.complex64 if params.cycle_precision == 32 else torch.complex128
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        mats = []
        on_dev = None
        for a in (lam, mu, rho):
            if isinstance(a, torch.Tensor):
                t = a.detach().to(torch.float64).contiguous()
                dev = 1 if t.is_cuda else 0
            else:
                t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
                dev = 0
            if t.numel() != self.ncell:
                raise ValueError("material has %d cells, expected %d" % (t.numel(), self.ncell))
            if on_dev is None:
                on_dev = dev
            elif on_dev != dev:
                raise ValueError("lam, mu, rho must all be on the host or all on the device")
            mats.append(t)
        self._mats = mats
        h = ctypes.c_void_p()
        self._p = params.to_c()
        _check(LIB.emg_create(ctypes.byref(self._p), ctypes.c_void_p(mats[0].data_ptr()),
                              ctypes.c_void_p(mats[1].data_ptr()), ctypes.c_void_p(mats[2].data_ptr()),
                              on_dev, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    # -- helpers
    def vec_shape(self, level=0):
        n = self.level_info(level)[0]
        return (self.dim + 1,) + tuple(n[:self.dim][::-1])

    def level_info(self, level):
        n = (ctypes.c_int32 * 3)()
        hh = ctypes.c_double()
        _check(LIB.emg_level_info(self.h, level, n, ctypes.byref(hh)))
        return tuple(n), hh.value

    def sweep_path(self, level):
        """(path, us): the sweep path of a level (SWEEP_*) and, if the autotuner chose it, the
        measured time of one smoothing call in microseconds (else 0)."""
        path = ctypes.c_int32()
        us = ctypes.c_double()
        _check(LIB.emg_sweep_path(self.h, level, ctypes.byref(path), ctypes.byref(us)))
        return path.value, us.value

    def _n(self, level=0):
        return int(np.prod(self.vec_shape(level)))

    def _in(self):
        """Order the handle's stream after the caller's current stream (the caller's tensors may
        still be in flight there)."""
        import torch
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def _out(self):
        """Order the caller's current stream after the handle's (its outputs)."""
        import torch
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    # -- entry points
    def apply(self, x, y, shifted=False):
        import torch
        n = self._n()
        self._in()
        _check(LIB.emg_apply(self.h, 1 if shifted else 0, _ptr(x, torch.complex128, n, "x"),
                             _ptr(y, torch.complex128, n, "y")))
        self._out()
        return y

    def vcycle(self, b, x, zero_guess=True):
        n = self._n()
        self._in()
        _check(LIB.emg_vcycle(self.h, _ptr(b, self.cdtype, n, "b"), _ptr(x, self.cdtype, n, "x"),
                              1 if zero_guess else 0))
        self._out()
        return x

    def smooth(self, level, b, x, sweeps):
        n = self._n(level)
        self._in()
        _check(LIB.emg_smooth(self.h, level, _ptr(b, self.cdtype, n, "b"), _ptr(x, self.cdtype, n, "x"), sweeps))
        self._out()
        return x

    def residual_restrict(self, level, b, x, bc):
        n, nc = self._n(level), self._n(level + 1)
        self._in()
        _check(LIB.emg_residual_restrict(self.h, level, _ptr(b, self.cdtype, n, "b"), _ptr(x, self.cdtype, n, "x"),
                                         _ptr(bc, self.cdtype, nc, "b_coarse")))
        self._out()
        return bc

    def prolong_correct(self, level, ec, x):
        n, nc = self._n(level), self._n(level + 1)
        self._in()
        _check(LIB.emg_prolong_correct(self.h, level, _ptr(ec, self.cdtype, nc, "e_coarse"),
                                       _ptr(x, self.cdtype, n, "x")))
        self._out()
        return x

    def coarse_solve(self, b, x):
        last = self.params.levels - 1
        n = self._n(last)
        self._in()
        _check(LIB.emg_coarse_solve(self.h, _ptr(b, self.cdtype, n, "b"), _ptr(x, self.cdtype, n, "x")))
        self._out()
        return x

    def coarse_stats(self):
        """Last coarsest solve of COARSE_KACZMARZ: (FGMRES iterations, relative Schur residual,
        Kaczmarz steps)."""
        out = (ctypes.c_double * 3)()
        _check(LIB.emg_coarse_stats(self.h, out))
        return int(out[0]), float(out[1]), int(out[2])

    def coarse_schur_rows(self):
        """The stored Schur rows of COARSE_KACZMARZ as a complex numpy array (dim N_c, 75 or 17),
        in the cycle precision (layout in include/emg.h)."""
        last = self.params.levels - 1
        cells = self._n(last) // (self.dim + 1)
        ne = 75 if self.dim == 3 else 17
        dt = np.complex64 if self.params.cycle_precision == 32 else np.complex128
        out = np.zeros((self.dim * cells, ne), dtype=dt)
        _check(LIB.emg_coarse_schur_rows(self.h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def solve(self, b, x, tol=1e-6, max_iter=1000, restart=20, history_cap=0):
        import torch
        n = self._n()
        st = _Stats()
        hist = None
        if history_cap:
            hist = (ctypes.c_double * history_cap)()
            st.history = hist
            st.history_cap = history_cap
        self._in()
        s = _check(LIB.emg_solve(self.h, _ptr(b, torch.complex128, n, "b"), _ptr(x, torch.complex128, n, "x"),
                                 tol, max_iter, restart, ctypes.byref(st)), allow=(0, 5))
        self._out()
        return self._stats(st, hist, s)

    def apply_adjoint(self, x, y):
        """y = H^H x (unshifted finest operator, conjugate-transposed), complex128."""
        import torch
        n = self._n()
        self._in()
        _check(LIB.emg_apply_adjoint(self.h, _ptr(x, torch.complex128, n, "x"), _ptr(y, torch.complex128, n, "y")))
        self._out()
        return y

    def solve_adjoint(self, b, x, tol=1e-6, max_iter=1000, restart=20, history_cap=0):
        """Solve H^H x = b (FGMRES preconditioned by the mapped cycle; FP32 cycle only)."""
        import torch
        n = self._n()
        st = _Stats()
        hist = None
        if history_cap:
            hist = (ctypes.c_double * history_cap)()
            st.history = hist
            st.history_cap = history_cap
        self._in()
        s = _check(LIB.emg_solve_adjoint(self.h, _ptr(b, torch.complex128, n, "b"),
                                         _ptr(x, torch.complex128, n, "x"), tol, max_iter, restart,
                                         ctypes.byref(st)), allow=(0, 5))
        self._out()
        return self._stats(st, hist, s)

    def material_gradient(self, u, a, out=None, accumulate=False):
        """-Re a^H (dH/dm) u per cell for m = lambda, mu, rho: a tuple of three float64 tensors of
        the grid's shape (written into `out` if given, added to it with accumulate=True)."""
        import torch
        n = self._n()
        if out is None:
            out = tuple(torch.zeros(self.shape, dtype=torch.float64, device=u.device) for _ in range(3))
        ptrs = [_ptr(g, torch.float64, self.ncell, nm) for g, nm in zip(out, ("g_lam", "g_mu", "g_rho"))]
        self._in()
        _check(LIB.emg_material_gradient(self.h, _ptr(u, torch.complex128, n, "u"), _ptr(a, torch.complex128, n, "a"),
                                         ptrs[0], ptrs[1], ptrs[2], 1 if accumulate else 0))
        self._out()
        return out

    def solve_host(self, b, x, tol=1e-6, max_iter=1000, restart=20, history_cap=0):
        """b, x: host numpy complex128 arrays (pinned or pageable); x is overwritten."""
        n = self._n()
        for a, nm in ((b, "b"), (x, "x")):
            if a.dtype != np.complex128 or a.size != n or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("%s must be a contiguous complex128 array of %d entries" % (nm, n))
        st = _Stats()
        hist = None
        if history_cap:
            hist = (ctypes.c_double * history_cap)()
            st.history = hist
            st.history_cap = history_cap
        s = _check(LIB.emg_solve_host(self.h, ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data),
                                      tol, max_iter, restart, ctypes.byref(st)), allow=(0, 5))
        return self._stats(st, hist, s)

    @staticmethod
    def _stats(st, hist, status):
        out = {"iterations": st.iterations, "restarts": st.restarts, "rel_residual": st.rel_residual,
               "converged": status == 0}
        if hist is not None:
            out["history"] = [hist[i] for i in range(st.history_len)]
        return out

    def profile(self, enable=True, coarse=False):
        """Per-class CUDA-event timing of the finest level's kernels; coarse=True also times every
        kernel of the coarser levels (class K_COARSE)."""
        _check(LIB.emg_profile(self.h, (2 if coarse else 1) if enable else 0))

    def profile_read(self, cls):
        ms, n, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(LIB.emg_profile_read(self.h, cls, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
        return {"ms": ms.value, "launches": n.value, "bytes": by.value}

    def close(self):
        if getattr(self, "h", None):
            _check(LIB.emg_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
