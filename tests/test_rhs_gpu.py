"""Parity of the CUDA right-hand side of Eq. (4) with the FP64 oracle.

Tolerances are normwise: an FFT's rounding error is bounded relative to the norm of
the convolution, not entrywise, so the small tail entries carry an absolute error of
order eps * ||birth||. Each term is checked as
    ||x - x_ref||_2 <= rtol ||x_ref||_2  and  ||x - x_ref||_inf <= rtol ||x_ref||_inf,
and the total S, whose terms cancel near a steady state, against the scale
|| |birth| + |loss| + |source| ||. rtol = 1e-10 for FP64, 1e-4 for the FP32
convolution form (FP32 FFT error ~ 1e-7 log2(M) relative).
"""
import numpy as np
import pytest

import oracle
from synth import kernel_factors, random_factors, random_state, sample_state

pytestmark = pytest.mark.gpu

RTOL = {"fp64": 1e-10, "fp32conv": 1e-4, "df64": 1e-10}


@pytest.fixture(scope="module")
def smol():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_16559_gb300 as m
    return m


def _ref_terms(n, U, V, lam, route):
    if route == "direct":
        d = oracle.rhs_terms_direct(n, U @ V, lam)
    else:
        d = oracle.rhs_terms_lowrank(n, U, V, lam)
    loss = d["death"] + d["shatter_loss"]
    return d["birth"], loss, float(d["monomer_source"][0]), d["total"]


def _close(x, ref, rtol, scale=None, what=""):
    x = np.asarray(x)
    ref = np.asarray(ref)
    s2 = np.linalg.norm(ref) if scale is None else np.linalg.norm(scale)
    si = np.max(np.abs(ref)) if scale is None else np.max(np.abs(scale))
    e2 = np.linalg.norm(x - ref)
    ei = np.max(np.abs(x - ref)) if x.size else 0.0
    assert e2 <= rtol * s2 + 1e-300, f"{what}: l2 {e2:.3e} > {rtol:.0e} * {s2:.3e}"
    assert ei <= rtol * si + 1e-300, f"{what}: linf {ei:.3e} > {rtol:.0e} * {si:.3e}"


def check_rhs(smol, n, U, V, lam, precision="fp64", route=None, **opts):
    import torch
    M = n.size
    if route is None:
        route = "direct" if M <= 2048 else "lowrank"
    sysm = smol.System(U, V, lam, precision=precision, **opts)
    dn = torch.from_numpy(n).cuda()
    S = sysm.rhs(dn).cpu().numpy()
    b, l, src = (t.cpu().numpy() for t in sysm.rhs_terms(dn))
    rb, rl, rsrc, rS = _ref_terms(n, U, V, lam, route)
    rtol = RTOL[precision]
    _close(b, rb, rtol, what="birth")
    _close(l, rl, rtol, what="loss")
    assert abs(src[0] - rsrc) <= rtol * (abs(rsrc) + np.max(np.abs(rl)) * 1e-3 + 1e-300), (src[0], rsrc)
    scale = np.abs(rb) + np.abs(rl)
    scale[0] += abs(rsrc)
    _close(S, rS, rtol, scale=scale, what="total")
    return sysm


KERNELS = [("const", 0.0), ("brownian", 0.3), ("brownian", 0.9), ("brownian_const", 1.0 / 3.0)]


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 8, 17, 64, 100, 257, 1000, 1024, 2048])
@pytest.mark.parametrize("kind,a", KERNELS)
def test_rhs_small_sizes(smol, M, kind, a):
    """Several tiles and ragged tails; M not a power of two is zero-padded to Mp."""
    U, V = kernel_factors(kind, M, a=a)
    n = random_state(M, seed=M + 3)
    check_rhs(smol, n, U, V, 0.01)


@pytest.mark.parametrize("lam", [0.0, 0.005, 0.1, 1.0])
def test_rhs_lambda(smol, lam):
    M = 777
    U, V = kernel_factors("brownian", M, a=0.9)
    check_rhs(smol, sample_state(M, lam), U, V, lam)


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
@pytest.mark.parametrize("M,R", [(50, 1), (300, 3), (1500, 4), (4096, 8)])
def test_rhs_random_nonsymmetric_factors(smol, M, R, precision):
    """Non-symmetric factors with no shared transforms (T = 2R, up to 16: beyond the
    column kernels' weight prefetch of 4): a transposed U / V or a wrong pairing in the
    spectral product fails the loss or source term."""
    U, V = random_factors(M, R, seed=5 * M + R)
    n = random_state(M, seed=M)
    s = check_rhs(smol, n, U, V, 0.2, precision=precision)
    assert s.num_transforms == 2 * R


def test_transform_sharing(smol):
    M = 128
    for kind, a, T in (("const", 0.0, 1), ("brownian", 0.5, 2), ("brownian_const", 1 / 3, 3)):
        U, V = kernel_factors(kind, M, a=a)
        assert smol.System(U, V, 0.0).num_transforms == T


@pytest.mark.parametrize("M", [4096, 8192, 16384, 65536, 65537, 131072])
@pytest.mark.parametrize("kind,a", [("brownian", 0.9), ("brownian_const", 1.0 / 3.0)])
def test_rhs_large_vs_lowrank_oracle(smol, M, kind, a):
    """Up to the bench size M = 2^17: against the oracle's numpy-FFT route (itself
    pinned to the direct sums)."""
    U, V = kernel_factors(kind, M, a=a)
    check_rhs(smol, sample_state(M, 0.005, seed=M), U, V, 0.005)


def test_rhs_full_size_sampled_direct_entries(smol):
    """M = 2^17, the size the bench times: sampled outputs against the direct O(M)
    per-entry sums of Eq. (4), including the first and last sizes."""
    import torch
    M, a, lam = 131072, 0.9, 0.005
    U, V = kernel_factors("brownian", M, a=a)
    n = sample_state(M, lam, seed=11)
    sysm = smol.System(U, V, lam)
    S = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    b, l, _ = (t.cpu().numpy() for t in sysm.rhs_terms(torch.from_numpy(n).cuda()))
    rng = np.random.default_rng(0)
    sizes = sorted(set([2, 3, M // 2, M - 1, M] + list(rng.integers(2, M + 1, 40))))
    ref = oracle.rhs_entries_direct(n, lambda i, j: (i / j) ** a + (j / i) ** a, lam, sizes)
    got = S[np.array(sizes) - 1]
    scale = np.max(np.abs(b)) + np.abs(l[np.array(sizes) - 1])
    assert np.all(np.abs(got - ref) <= 1e-10 * scale), np.max(np.abs(got - ref) / scale)


@pytest.mark.parametrize("M", [64, 1000, 4096, 65536, 131072])
@pytest.mark.parametrize("kind,a", [("brownian", 0.9), ("brownian_const", 1.0 / 3.0)])
def test_rhs_fp32conv(smol, M, kind, a):
    U, V = kernel_factors(kind, M, a=a)
    check_rhs(smol, sample_state(M, 0.1, seed=M), U, V, 0.1, precision="fp32conv")


def test_rhs_fp32conv_scaled_states(smol):
    """Per-transform power-of-two scaling keeps the FP32 spectra (products of two
    transforms) in range for dilute (1e-12) and dense (1e+12) states; the FP32 form
    needs S itself to be representable in FP32."""
    M = 4096
    U, V = kernel_factors("brownian", M, a=0.6)
    for mag in (1e-12, 1e12):
        check_rhs(smol, sample_state(M, 0.01) * mag, U, V, 0.01, precision="fp32conv")


def test_rhs_zero_state_and_repeat(smol):
    import torch
    M = 300
    U, V = kernel_factors("brownian", M, a=0.4)
    sysm = smol.System(U, V, 0.01)
    z = sysm.rhs(torch.zeros(M, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(z == 0.0)
    n = torch.from_numpy(random_state(M, seed=1)).cuda()
    a1 = sysm.rhs(n).cpu().numpy()
    a2 = sysm.rhs(n).cpu().numpy()
    assert np.array_equal(a1, a2)  # deterministic reductions


def _rule(M):
    """The FFT schedule rule: log2 Mp, log2 N1 (column length) and columns per CTA."""
    lgmp = max(2, int(M - 1).bit_length())
    lg1 = (lgmp + 1) // 2
    return lgmp, lg1, max(1, 256 >> lg1)


@pytest.mark.parametrize("M", [9, 1000, 4096, 65537])
@pytest.mark.parametrize("dl,gm", [(-1, 1), (1, 1), (0, 2), (1, 2), (-2, 4)])
def test_rhs_fft_schedules(smol, M, dl, gm):
    """Every schedule the autotuner may pick (another split Mp = N1 N2, more columns per
    CTA) computes the same S: the split changes only the rounding order."""
    lgmp, lg1, _ = _rule(M)
    lg = lg1 + dl
    if not 1 <= lg < lgmp:
        pytest.skip("split outside the valid range for this size")
    g = min(max(1, 256 >> lg) * gm, 1 << (lgmp - lg), 64)
    U, V = kernel_factors("brownian_const", M, a=0.45)
    try:
        check_rhs(smol, sample_state(M, 0.02, seed=M + 7), U, V, 0.02, fft_lgn1=lg, fft_g=g)
    except smol.SmolError as e:
        # long rows whose T transforms exceed the shared memory of a CTA (the tuner
        # skips these candidates too)
        assert e.code == smol.EUNSUPPORTED and (1 << (lgmp - lg)) >= 1024
        pytest.skip("shape beyond the shared-memory limit")


@pytest.mark.parametrize("dl", [-1, 1])
def test_rhs_fft_schedules_fp32conv(smol, dl):
    M = 65536
    lgmp, lg1, g = _rule(M)
    U, V = kernel_factors("brownian", M, a=0.8)
    check_rhs(smol, sample_state(M, 0.02, seed=3), U, V, 0.02, precision="fp32conv", fft_lgn1=lg1 + dl, fft_g=g)


def test_rhs_bad_schedule_rejected(smol):
    U, V = kernel_factors("brownian", 64, a=0.5)
    with pytest.raises(smol.SmolError):
        smol.System(U, V, 0.0, fft_g=3)


@pytest.mark.parametrize("M", [1, 2, 3, 17, 100, 1000, 4096, 65537, 131072])
@pytest.mark.parametrize("kind,a", [("const", 0.0), ("brownian", 0.9), ("brownian_const", 1.0 / 3.0)])
def test_rhs_df64(smol, M, kind, a):
    """The double-float form meets the FP64 tolerance at every size."""
    U, V = kernel_factors(kind, M, a=a)
    check_rhs(smol, sample_state(M, 0.01, seed=M + 1), U, V, 0.01, precision="df64")


def test_rhs_df64_scaled_states_and_random_factors(smol):
    """Per-transform power-of-two scaling keeps the double-float spectra in FP32's
    exponent range for dilute and dense states; non-symmetric factors (T = 2R)."""
    M = 4096
    U, V = kernel_factors("brownian", M, a=0.6)
    for mag in (1e-12, 1e12):
        check_rhs(smol, sample_state(M, 0.01) * mag, U, V, 0.01, precision="df64")
    U, V = random_factors(1500, 4, seed=9)
    check_rhs(smol, random_state(1500, seed=4), U, V, 0.2, precision="df64")


def test_rhs_df64_full_size_sampled_direct_entries(smol):
    """M = 2^17 in the double-float form: sampled outputs against the direct O(M)
    per-entry sums of Eq. (4) at the FP64 tolerance."""
    import torch
    M, a, lam = 131072, 0.9, 0.005
    U, V = kernel_factors("brownian", M, a=a)
    n = sample_state(M, lam, seed=11)
    sysm = smol.System(U, V, lam, precision="df64")
    S = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    b, l, _ = (t.cpu().numpy() for t in sysm.rhs_terms(torch.from_numpy(n).cuda()))
    rng = np.random.default_rng(0)
    sizes = sorted(set([2, 3, M // 2, M - 1, M] + list(rng.integers(2, M + 1, 40))))
    ref = oracle.rhs_entries_direct(n, lambda i, j: (i / j) ** a + (j / i) ** a, lam, sizes)
    got = S[np.array(sizes) - 1]
    scale = np.max(np.abs(b)) + np.abs(l[np.array(sizes) - 1])
    assert np.all(np.abs(got - ref) <= 1e-10 * scale), np.max(np.abs(got - ref) / scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_rhs_at_maximum_size(smol, precision):
    """The largest M the kernels take for the Brownian kernel, whose rank-2 factors share
    their transforms (T = 2; smol_max_m_transforms: the tiles' shared memory sets it):
    parity with the oracle's FFT route there, and the next size is refused with
    SMOL_EUNSUPPORTED. Without shared transforms (random factors, T = 2R = 4) the limit
    is smol_max_m(2)."""
    M = smol.max_m_transforms(2, precision)
    U, V = kernel_factors("brownian", M, a=0.7)
    assert smol.System(U, V, 0.002, precision=precision).num_transforms == 2
    check_rhs(smol, sample_state(M, 0.002, seed=5), U, V, 0.002, precision=precision, route="lowrank")
    U1, V1 = kernel_factors("brownian", M + 1, a=0.7)
    with pytest.raises(smol.SmolError) as e:
        smol.System(U1, V1, 0.002, precision=precision)
    assert e.value.code == smol.EUNSUPPORTED
    M4 = smol.max_m(2, precision)
    U4, V4 = random_factors(M4 + 1, 2, seed=3)
    with pytest.raises(smol.SmolError) as e:
        smol.System(U4, V4, 0.002, precision=precision)
    assert e.value.code == smol.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_small_system_after_large_keeps_large_working(smol, precision):
    """The kernels' shared-memory limit is one setting per kernel shared by every live
    system: creating a small system after a large one must not lower it below what the
    large one launches with. The large system still evaluates and integrates afterwards."""
    import torch
    M = 1 << 17
    U, V = kernel_factors("brownian", M, a=0.9)
    n = sample_state(M, 0.005)
    big = smol.System(U, V, 0.005, precision=precision)
    S0 = big.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    Us, Vs = kernel_factors("brownian", 1024, a=0.9)
    small = smol.System(Us, Vs, 0.005, precision=precision)
    small.rhs(torch.from_numpy(sample_state(1024, 0.005)).cuda())
    S1 = big.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    assert np.array_equal(S0, S1)
    _, st = big.integrate(torch.from_numpy(n).cuda(), 0.0, 1e-3, 1e-8, scheme="rkf45")
    assert st["status"] == 0 and st["accepted"] >= 1, st
