"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function that
include/emg.h declares; argument validation that needs no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "emg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emg_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    from paper_2307_03242_gb300.build import build_library
    lib = build_library()
    import ctypes
    so = ctypes.CDLL(lib)
    names = _declared()
    assert "emg_solve" in names and "emg_create" in names
    for n in names:
        assert hasattr(so, n), n
    from paper_2307_03242_gb300 import emg
    assert sorted(emg.EXPORTED) == names


def test_params_struct_layout_matches_header():
    """ctypes mirror of emg_params / emg_stats has the C layout (field offsets)."""
    import ctypes
    from paper_2307_03242_gb300 import emg
    P = emg._Params
    assert P.n.offset == 4 and P.h.offset == 16
    assert P.damping.offset % 8 == 0 and ctypes.sizeof(P) % 8 == 0
    S = emg._Stats
    assert S.history.offset == 16


def test_invalid_arguments_are_rejected_without_a_gpu():
    import numpy as np
    from paper_2307_03242_gb300 import emg
    p = emg.Params(n=(30, 16), levels=3)  # 30 not divisible by 4
    c = p.to_c()
    import ctypes
    h = ctypes.c_void_p()
    lam = np.ones(30 * 16)
    st = emg.LIB.emg_create(ctypes.byref(c), lam.ctypes.data, lam.ctypes.data, lam.ctypes.data, 0, None,
                            ctypes.byref(h))
    assert st == 1 and b"divisible" in emg.LIB.emg_last_error()
    assert emg.LIB.emg_solve(None, None, None, 1e-6, 10, 20, None) == 1
    assert emg.LIB.emg_destroy(None) == 0


def test_batch_arguments_are_rejected_without_a_gpu():
    import ctypes
    from paper_2307_03242_gb300 import emg
    vp = ctypes.c_void_p
    arr = (vp * 1)()
    assert emg.LIB.emg_solve_batch(arr, -1, arr, arr, 1e-6, 10, 5, None, 0, None) == 1
    assert emg.LIB.emg_solve_batch(None, 0, None, None, 1e-6, 10, 5, None, 0, None) == 0
    assert emg.LIB.emg_solve_batch(arr, 1, arr, arr, 1e-6, 10, 5, None, 0, None) == 1  # NULL handle
    assert b"NULL handle" in emg.LIB.emg_last_error()
    assert emg.LIB.emg_solve_batch(None, 1, arr, arr, 1e-6, 10, 5, None, 0, None) == 1


def test_invalid_material_is_rejected_before_any_device_work():
    import ctypes
    import numpy as np
    from paper_2307_03242_gb300 import emg
    c = emg.Params(n=(8, 8), levels=2).to_c()
    h = ctypes.c_void_p()
    good = np.ones(64)
    for bad_field in range(3):
        mats = [good.copy(), good.copy(), good.copy()]
        mats[bad_field][17] = np.nan if bad_field == 0 else -1.0
        st = emg.LIB.emg_create(ctypes.byref(c), mats[0].ctypes.data, mats[1].ctypes.data, mats[2].ctypes.data, 0,
                                None, ctypes.byref(h))
        assert st == 1 and b"material" in emg.LIB.emg_last_error() and b"cell 17" in emg.LIB.emg_last_error()
    c.smoother = 7
    st = emg.LIB.emg_create(ctypes.byref(c), good.ctypes.data, good.ctypes.data, good.ctypes.data, 0, None,
                            ctypes.byref(h))
    assert st == 1 and b"smoother" in emg.LIB.emg_last_error()


def test_sweep_path_range_is_checked_before_any_device_work():
    """EMG_SWEEP_TILE4 (5) is the last sweep path; 6 and -1 are rejected with a message, before the
    library touches a device."""
    import ctypes
    import numpy as np
    from paper_2307_03242_gb300 import emg
    assert (emg.SWEEP_AUTO, emg.SWEEP_HALF, emg.SWEEP_COOP, emg.SWEEP_TILE24, emg.SWEEP_TILE8, emg.SWEEP_TILE4) == \
        (0, 1, 2, 3, 4, 5)
    good = np.ones(64)
    h = ctypes.c_void_p()
    for bad in (6, -1):
        c = emg.Params(n=(8, 8), levels=2).to_c()
        c.sweep_path = bad
        st = emg.LIB.emg_create(ctypes.byref(c), good.ctypes.data, good.ctypes.data, good.ctypes.data, 0, None,
                                ctypes.byref(h))
        assert st == 1 and b"sweep_path" in emg.LIB.emg_last_error()
