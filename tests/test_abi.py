"""The C-ABI library loads and exports every entry point include/smol.h declares, and
its host-side argument checks work without a GPU (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smol.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(smol_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def smol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_16559_gb300 as m
    return m


def test_header_declares_the_interface():
    names = declared_functions()
    for must in ("smol_init_system", "smol_rhs", "smol_integrate", "smol_workspace_bytes", "smol_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(smol):
    lib = ctypes.CDLL(smol.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(smol.SIGNATURES)


def test_host_side_queries(smol):
    o = smol.default_opts()
    assert o.precision == 0 and o.euler_a == 0.1 and o.fac_max == 4.0 and o.chunk == 32
    assert smol.max_m(2) >= 2 ** 17 and smol.max_m(3, "fp32conv") >= 2 ** 17
    assert smol.max_m(0) == 0 and smol.max_m(smol.MAX_R + 1) == 0 and smol.max_m(smol.MAX_R) > 0
    assert smol.max_m_transforms(2) >= smol.max_m(2) and smol.max_m_transforms(2 * smol.MAX_R + 1) == 0
    lib = smol._lib
    assert lib.smol_workspace_bytes(2 ** 17, 2, None) > 0
    assert lib.smol_workspace_bytes(0, 2, None) == 0
    assert lib.smol_workspace_bytes(16, smol.MAX_R + 1, None) == 0
    assert smol.strerror(-3).startswith("non-finite")


def test_invalid_arguments_rejected_before_any_cuda_call(smol):
    lib = smol._lib
    h = ctypes.c_void_p()
    import numpy as np
    U = np.ones((8, 1))
    V = np.ones((1, 8))
    # NULL workspace, bad M, bad R, negative lambda: all EINVAL
    assert lib.smol_init_system(ctypes.byref(h), 8, 1, U.ctypes.data, V.ctypes.data, 0.0, None, None, 0) == -1
    assert lib.smol_init_system(ctypes.byref(h), 0, 1, U.ctypes.data, V.ctypes.data, 0.0, None, 256, 1 << 20) == -1
    assert lib.smol_init_system(ctypes.byref(h), 8, 0, U.ctypes.data, V.ctypes.data, 0.0, None, 256, 1 << 20) == -1
    assert lib.smol_init_system(ctypes.byref(h), 8, 1, U.ctypes.data, V.ctypes.data, -1.0, None, 256, 1 << 20) == -1
    # too small a workspace
    assert lib.smol_init_system(ctypes.byref(h), 8, 1, U.ctypes.data, V.ctypes.data, 0.0, None, 256, 16) == -7
    assert lib.smol_rhs(None, None, None) == -1
    assert lib.smol_integrate(None, None, 0.0, 1.0, 1e-8, 2, None) == -1
    lib.smol_destroy(None)


def test_malformed_schedule_options_rejected_before_any_cuda_call(smol):
    """The batch's per-size schedule tables (smol_opts.batch_lgn1 / batch_g) are checked
    like the single system's schedule: columns per CTA a power of two up to 64, log2 N1
    up to 30; a bad entry is SMOL_EINVAL before the library touches a device."""
    import numpy as np
    lib = smol._lib
    U = np.ones((1024, 1))
    V = np.ones((1, 1024))
    M = np.array([1024], dtype=np.int64)
    pU = (ctypes.c_void_p * 1)(U.ctypes.data)
    pV = (ctypes.c_void_p * 1)(V.ctypes.data)
    lam = np.array([0.01])
    pn = (ctypes.c_void_p * 1)(256)  # never dereferenced: the options are refused first
    h = ctypes.c_void_p()
    for field, k, bad in (("batch_g", 10, 3), ("batch_g", 10, -4), ("batch_lgn1", 10, 31), ("batch_lgn1", 5, -1)):
        o = smol.default_opts()
        getattr(o, field)[k] = bad
        assert lib.smol_batch_init(ctypes.byref(h), 1, M.ctypes.data, 1, pU, pV, lam.ctypes.data, ctypes.byref(o),
                                   256, 1 << 30) == -1, (field, k, bad)
        us = ctypes.c_double()
        assert lib.smol_batch_tune_schedules(1, M.ctypes.data, 1, pU, pV, lam.ctypes.data, pn, 1e-8, 2, 4,
                                             ctypes.byref(o), ctypes.byref(us)) == -1, (field, k, bad)
    o = smol.default_opts()
    o.fft_g = 6
    assert lib.smol_batch_init(ctypes.byref(h), 1, M.ctypes.data, 1, pU, pV, lam.ctypes.data, ctypes.byref(o),
                               256, 1 << 30) == -1
    assert smol.SIZE_CLASSES == len(o.batch_lgn1) == len(o.batch_g)
