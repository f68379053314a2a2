"""The right-hand side and integration with the free-molecular kernel of Sec. 3.1, which
has no exact low rank: the CUDA path runs on the factors of smol_lowrank_kernel (rank 16,
V = diag(+-1) U^T, so T = 16 shared transforms) and is compared with the oracle's direct
route on the dense closed-form kernel (not on the factors). The bar is the factors'
approximation error (their largest relative entry error, which bounds the relative error
of every birth and loss entry, since all terms are positive) plus the FP64 one."""
import numpy as np
import pytest

import oracle
from synth import monodisperse, sample_state

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


def fm(i, j):
    return (np.cbrt(i) + np.cbrt(j)) ** 2 * np.sqrt(1.0 / i + 1.0 / j)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("M,lam", [(700, 0.01), (2048, 0.1)])
def test_free_molecular_rhs_vs_dense_closed_form(smol, precision, M, lam):
    import torch
    U, V, _ = smol.lowrank_kernel("free_molecular", M, tol=1e-14)
    K = oracle.kernel_closed_form("free_molecular", M)
    eps = float(np.max(np.abs(U @ V - K) / K))
    n = sample_state(M, lam, seed=M)
    sysm = smol.System(U, V, lam, precision=precision)
    assert sysm.num_transforms == U.shape[1] == 16
    S = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    d = oracle.rhs_terms_direct(n, K, lam)
    scale = np.abs(d["birth"]) + np.abs(d["death"] + d["shatter_loss"])
    scale[0] += abs(d["monomer_source"][0])
    # the factors' error is relative entry by entry; the transforms' rounding is
    # relative to the largest entries (normwise), which dominates in the near-empty tail
    err = np.abs(S - d["total"])
    assert np.all(err <= eps * scale + 1e-10 * np.max(scale)), np.max(err / (eps * scale + 1e-10 * np.max(scale)))


def test_free_molecular_full_size_sampled_entries(smol):
    """M = 32768 (the size of the paper's sources experiments, the largest FP64 size for
    16 transforms): sampled entries against the direct per-entry sums of Eq. (4) with the
    closed-form kernel."""
    import torch
    M, lam = 32768, 0.01
    assert smol.max_m_transforms(16, "fp64") >= M
    U, V, est = smol.lowrank_kernel("free_molecular", M, tol=1e-14)
    n = sample_state(M, lam, seed=4)
    sysm = smol.System(U, V, lam)
    S = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    b, l, _ = (t.cpu().numpy() for t in sysm.rhs_terms(torch.from_numpy(n).cuda()))
    rng = np.random.default_rng(1)
    sizes = sorted(set([2, 3, 100, M // 2, M - 1, M] + list(rng.integers(2, M + 1, 30))))
    ref = oracle.rhs_entries_direct(n, fm, lam, sizes)
    idx = np.array(sizes) - 1
    scale = np.abs(b[idx]) + np.abs(l[idx])
    lim = 3 * est * scale + 1e-10 * (np.max(np.abs(b)) + np.abs(l[idx]))
    assert np.all(np.abs(S[idx] - ref) <= lim), np.max(np.abs(S[idx] - ref) / lim)


def test_free_molecular_sources_integration_vs_dense_oracle(smol):
    """Sec. 3.1's setting with the free-molecular kernel: aggregation with the sources
    P_1 = 1, P_100 = 0.01 (Eq. (3), lambda = 0), M = 1024, RKF45 tol 1e-8 over t <= 20;
    the GPU on the rank-16 factors against the oracle's direct route on the dense
    closed-form kernel."""
    import torch
    M = 1024
    U, V, _ = smol.lowrank_kernel("free_molecular", M, tol=1e-14)
    src = {1: 1.0, 100: 0.01}
    sysm = smol.System(U, V, 0.0, tau0=1e-3)
    sysm.set_sources(src)
    n, st = sysm.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 20.0, 1e-8)
    osys = oracle.System(M, 0.0, K=oracle.kernel_closed_form("free_molecular", M), route="direct", sources=src)
    m, ost, _ = oracle.integrate(osys, monodisperse(M), 0.0, 20.0, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-3))
    assert st["status"] == 0 and ost["status"] == 0
    x = n.cpu().numpy()
    assert np.linalg.norm(x - m) <= (10 * 1e-8 / np.linalg.norm(m) + 1e-8) * np.linalg.norm(m)
    # the factors differ from the kernel by ~1e-10 relative, which moves decisions taken
    # near the tolerance: counts within 5%
    assert abs(st["accepted"] - ost["accepted"]) <= max(2, 0.05 * ost["accepted"])
