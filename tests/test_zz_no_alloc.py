"""smol_rhs_static, the evaluation of S(n) that allocates nothing, against smol_rhs.

Callers that cannot allocate device memory (code running inside CUDA-graph capture,
hosts without a device allocator, plug-ins that do not own the process's memory) use
smol_rhs_static, whose scratch is a fixed device array inside the library. This test
calls it through the C interface twice in a row, with different sizes and inputs (the
array keeps the previous call's contents), and compares each result with the
workspace-based smol_rhs and with the FP64 oracle at the FP64 parity tolerance (1e-10
normwise). It is collected
last so that a failure here cannot stop the rest of a -x run, and it passes alone in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import kernel_factors, random_factors, random_state, sample_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smol():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_16559_gb300 as m
    return m


def _static(smol, U, V, lam, n):
    import torch
    dU = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    dV = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    dn = torch.from_numpy(n).cuda()
    out = torch.full_like(dn, np.nan)
    M, R = U.shape
    st = torch.cuda.current_stream()
    rc = smol._lib.smol_rhs_static(M, R, ctypes.c_void_p(dU.data_ptr()), ctypes.c_void_p(dV.data_ptr()),
                                   float(lam), ctypes.c_void_p(dn.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(st.cuda_stream))
    assert rc == 0, smol.strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _reference(smol, U, V, lam, n):
    import torch
    return smol.System(U, V, lam).rhs(torch.from_numpy(n).cuda()).cpu().numpy()


def _close(a, b, rtol=1e-10, scale=None):
    s = b if scale is None else scale
    assert np.linalg.norm(a - b) <= rtol * np.linalg.norm(s)
    assert np.max(np.abs(a - b)) <= rtol * np.max(np.abs(s))


def _oracle_close(S, U, V, lam, n):
    """S against the FP64 oracle (direct sums up to M = 2048, the low-rank FFT route
    above), normwise at 1e-10 on the scale |birth| + |loss| + |source|, as the other
    right-hand-side parity tests do."""
    d = oracle.rhs_terms_direct(n, U @ V, lam) if n.size <= 2048 else oracle.rhs_terms_lowrank(n, U, V, lam)
    scale = np.abs(d["birth"]) + np.abs(d["death"] + d["shatter_loss"])
    scale[0] += abs(d["monomer_source"][0])
    _close(S, d["total"], scale=scale)


def test_static_matches_workspace_entry_two_calls(smol):
    cases = [
        (kernel_factors("brownian_const", 65536, a=1.0 / 3.0), 0.1, sample_state(65536, 0.1, seed=3)),
        (random_factors(1000, 2, seed=9), 0.02, random_state(1000, seed=4)),
    ]
    for (U, V), lam, n in cases:
        S = _static(smol, U, V, lam, n)
        _close(S, _reference(smol, U, V, lam, n))
        _oracle_close(S, U, V, lam, n)


def test_static_after_a_smaller_system(smol):
    """A workspace system of small M created after the first static call must not lower
    the shared-memory limits that a static call at the largest M launches with (the
    limits only rise), and the static call must not lower a live system's either."""
    import torch
    U, V = kernel_factors("brownian", 65536, a=0.9)
    n = sample_state(65536, 0.005, seed=5)
    S1 = _static(smol, U, V, 0.005, n)
    Us, Vs = kernel_factors("brownian", 64, a=0.9)
    small = smol.System(Us, Vs, 0.005)
    small.rhs(torch.from_numpy(sample_state(64, 0.005)).cuda())
    S2 = _static(smol, U, V, 0.005, n)
    assert np.array_equal(S1, S2)  # same call, same inputs: bit-identical
    _close(S2, _reference(smol, U, V, 0.005, n))


@pytest.mark.parametrize("M", [1, 3, 4, 4097])
@pytest.mark.parametrize("R", [1, 3])
def test_static_small_and_ragged_sizes(smol, M, R):
    """M < 4 (padded to 4), an odd log2 of the FFT size (4097 -> 8192) and the smallest
    and largest rank, against the workspace entry point and the oracle."""
    U, V = random_factors(M, R, seed=11 + M + R)
    n = random_state(M, seed=M)
    S = _static(smol, U, V, 0.03, n)
    _close(S, _reference(smol, U, V, 0.03, n))
    _oracle_close(S, U, V, 0.03, n)


def test_static_rejects_sizes_beyond_its_array(smol):
    lib = smol._lib
    big = smol.STATIC_MAX_M + 1
    assert lib.smol_rhs_static(big, 2, 16, 16, 0.0, 16, 16, None) == smol.EUNSUPPORTED
    assert lib.smol_rhs_static(100, smol.STATIC_MAX_R + 1, 16, 16, 0.0, 16, 16, None) == smol.EUNSUPPORTED
    assert lib.smol_rhs_static(100, 2, None, 16, 0.0, 16, 16, None) == smol.EINVAL
