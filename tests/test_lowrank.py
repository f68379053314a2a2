"""Low-rank factors of collision kernels without an exact low rank (the free-molecular
kernel of Sec. 3.1), from smol_lowrank_kernel (host code of the library; no GPU):
checked against the oracle's closed-form kernels, entry by entry."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def smol():
    import importlib.util
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("_b", os.path.join(root, "paper_2407_16559_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    try:
        b.build()
    except Exception as e:  # no compiler here: nothing to test
        pytest.skip(f"library not built: {e}")
    if root not in sys.path:
        sys.path.insert(0, root)
    import paper_2407_16559_gb300 as m
    return m


def test_free_molecular_closed_form_pins():
    """The oracle's free-molecular kernel: K_11 = (1 + 1)^2 sqrt(2), K_81 = (2 + 1)^2
    sqrt(1/8 + 1), symmetric, and homogeneous of degree 1/6 (2/3 from the square,
    -1/2 from the root): K(8i, 8j) = 2^{1/2} K(i, j)."""
    K = oracle.kernel_closed_form("free_molecular", 64)
    assert K[0, 0] == pytest.approx(4 * np.sqrt(2), rel=1e-15)
    assert K[7, 0] == pytest.approx(9 * np.sqrt(1.125), rel=1e-15)
    assert np.array_equal(K, K.T)
    i, j = np.arange(1, 9)[:, None], np.arange(1, 9)[None, :]
    assert np.allclose(K[8 * i - 1, 8 * j - 1], np.sqrt(2.0) * K[i - 1, j - 1], rtol=1e-14)


@pytest.mark.parametrize("kind,a,c,rank", [("const", 0.0, 0.0, 1), ("brownian", 0.3, 0.0, 2),
                                           ("brownian", 0.9, 2.0, 3), ("brownian", 1.0 / 3.0, 2.0, 3)])
def test_exact_rank_kernels_recovered(smol, kind, a, c, rank):
    """Kernels of exact low rank are recovered with their rank, to rounding."""
    M = 1500
    U, V, err = smol.lowrank_kernel(kind, M, tol=1e-13, a=a, c=c)
    K = oracle.kernel_closed_form("const" if kind == "const" else "brownian_const", M, a=a, c=c)
    assert U.shape == (M, rank) and V.shape == (rank, M)
    assert np.max(np.abs(U @ V - K) / K) < 1e-12
    assert err < 1e-12


@pytest.mark.parametrize("M,bound", [(1000, 1e-9), (4096, 2e-8)])
def test_free_molecular_approximation(smol, M, bound):
    """Rank 16 of the free-molecular kernel: every entry within `bound` (relative) of the
    closed form; the sampled estimate the call returns is no larger than the true
    maximum and within a factor 3 of it; V = diag(+-1) U^T, so the factors share their
    transforms."""
    U, V, est = smol.lowrank_kernel("free_molecular", M, tol=1e-14, max_rank=16)
    K = oracle.kernel_closed_form("free_molecular", M)
    true = np.max(np.abs(U @ V - K) / K)
    assert U.shape[1] == 16
    assert true < bound, true
    assert est <= true * (1 + 1e-4) and true <= 3 * est, (est, true)  # rounding of the tiny differences
    s = np.sign(V[:, 0] / U[0, :])
    assert set(np.unique(s)) <= {-1.0, 1.0}
    assert np.allclose(V, s[:, None] * U.T, rtol=1e-15, atol=0)


def test_tolerance_stops_early(smol):
    U, V, err = smol.lowrank_kernel("free_molecular", 2000, tol=1e-4, max_rank=16)
    assert U.shape[1] < 16
    K = oracle.kernel_closed_form("free_molecular", 2000)
    assert np.max(np.abs(U @ V - K) / K) < 1e-2


def test_bad_arguments(smol):
    lib = smol._lib
    import ctypes
    buf = np.zeros(100)
    r = ctypes.c_int32()
    assert lib.smol_lowrank_kernel(7, None, 10, 1e-8, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(r),
                                   None) == smol.EINVAL
    assert lib.smol_lowrank_kernel(2, None, 0, 1e-8, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(r),
                                   None) == smol.EINVAL
    assert lib.smol_lowrank_kernel(2, None, 10, 0.0, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(r),
                                   None) == smol.EINVAL
    assert lib.smol_lowrank_kernel(1, None, 10, 1e-8, 4, buf.ctypes.data, buf.ctypes.data, ctypes.byref(r),
                                   None) == smol.EINVAL  # the Brownian kernel needs its parameters
