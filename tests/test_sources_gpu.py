"""Aggregation with constant point sources, Eq. (3) (Sec. 3.1 injects P_1 = 1 and
P_100 = p): the CUDA path against the oracle, and the constant-kernel closed form."""
import math

import numpy as np
import pytest

import oracle
from synth import kernel_factors, monodisperse, random_state

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


def _close(x, ref, rtol, scale):
    assert np.linalg.norm(x - ref) <= rtol * np.linalg.norm(scale), np.linalg.norm(x - ref) / np.linalg.norm(scale)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32conv", 1e-4)])
@pytest.mark.parametrize("M,P,lam", [(300, {1: 1.0, 100: 0.05}, 0.0), (300, {300: 0.3, 2: -0.1}, 0.02),
                                     (1, {1: 2.0}, 0.0), (5000, {1: 1.0, 100: 0.01}, 0.0)])
def test_rhs_with_sources(smol, precision, rtol, M, P, lam):
    import torch
    U, V = kernel_factors("brownian", M, a=0.3)
    n = random_state(M, seed=M, decay=M / 10 + 2)
    sysm = smol.System(U, V, lam, precision=precision)
    sysm.set_sources(P)
    S = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    route = "direct" if M <= 2048 else "lowrank"
    d = oracle.System(M, lam, U=U, V=V, route=route, sources=P).rhs_terms(n)
    scale = np.abs(d["birth"]) + np.abs(d["death"]) + np.abs(d["shatter_loss"]) + np.abs(d["sources"])
    scale[0] += abs(d["monomer_source"][0])
    _close(S, d["total"], rtol, scale)
    sysm.set_sources({})  # removed again
    S0 = sysm.rhs(torch.from_numpy(n).cuda()).cpu().numpy()
    _close(S0, d["total"] - d["sources"], rtol, scale)


def test_integrate_with_two_sources_matches_oracle(smol):
    """The Tables 1-2 set-up at a small size: two sources, monodisperse start."""
    import torch
    M, P = 256, {1: 1.0, 100: 0.01}
    U, V = kernel_factors("brownian", M, a=1.0 / 3.0)
    sysm = smol.System(U, V, 0.0, tau0=1e-3)
    sysm.set_sources(P)
    n, st = sysm.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 2.0, 1e-8)
    o = oracle.System(M, 0.0, U=U, V=V, route="direct", sources=P)
    m, ost, _ = oracle.integrate(o, monodisperse(M), 0.0, 2.0, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-3))
    assert st["status"] == ost["status"] == 0
    assert (st["accepted"], st["rejected"]) == (ost["accepted"], ost["rejected"])
    n = n.cpu().numpy()
    assert np.linalg.norm(n - m) <= 1e-9 * np.linalg.norm(m)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32conv", 2e-5)])
def test_constant_kernel_with_monomer_source_closed_form(smol, precision, tol):
    """K = 1, P_1 = J, empty start: N(t) = sqrt(2J) tanh(t sqrt(J/2)), mass J t."""
    import torch
    M, J = 64, 1.0
    U, V = kernel_factors("const", M)
    sysm = smol.System(U, V, 0.0, precision=precision, tau0=1e-3)
    sysm.set_sources({1: J})
    n, st = sysm.integrate(torch.zeros(M, dtype=torch.float64, device="cuda"), 0.0, 3.0, 1e-11)
    assert st["status"] == 0
    n = n.cpu().numpy()
    assert abs(n.sum() - math.sqrt(2 * J) * math.tanh(3.0 * math.sqrt(J / 2))) <= tol
    assert abs(np.dot(np.arange(1, M + 1), n) - 3.0 * J) <= 10 * tol


def test_batch_sources_per_system(smol):
    """Sources set on one system of a batch act on that system only, as in a single
    system run."""
    import torch
    specs = [(200, 0.3), (300, 0.5), (128, 0.2)]
    Us, Vs, n0 = [], [], []
    for M, a in specs:
        U, V = kernel_factors("brownian", M, a=a)
        Us.append(U)
        Vs.append(V)
        n0.append(torch.from_numpy(monodisperse(M)))
    b = smol.Batch(Us, Vs, [0.0, 0.0, 0.0], tau0=1e-3)
    b.set_sources(1, {1: 1.0, 100: 0.02})
    ns, sts = b.integrate(n0, 0.0, 0.5, 1e-8)
    for q, (M, a) in enumerate(specs):
        s = smol.System(Us[q], Vs[q], 0.0, tau0=1e-3)
        if q == 1:
            s.set_sources({1: 1.0, 100: 0.02})
        m, st = s.integrate(n0[q], 0.0, 0.5, 1e-8)
        assert (sts[q]["accepted"], sts[q]["rejected"]) == (st["accepted"], st["rejected"])
        assert torch.linalg.norm(ns[q].cpu() - m.cpu()) <= 1e-12 * torch.linalg.norm(m.cpu())


def test_sources_rejected_arguments(smol):
    U, V = kernel_factors("brownian", 50, a=0.3)
    s = smol.System(U, V, 0.0)
    for bad in ({51: 1.0}, {0: 1.0}, {1: float("nan")}, {k: 1.0 for k in range(1, 10)}):
        with pytest.raises(smol.SmolError):
            s.set_sources(bad)


def test_sources_changed_between_integrations(smol):
    """Sources may be set after an integration: the next one uses them (the captured
    graph is rebuilt), and equals a system created with them from the start."""
    import torch
    M = 200
    U, V = kernel_factors("brownian", M, a=0.3)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    s = smol.System(U, V, 0.0, tau0=0.01)
    s.integrate(n0, 0.0, 1.0, 1e-8)
    s.set_sources({1: 1.0, 100: 0.01})
    a, sa = s.integrate(n0, 0.0, 1.0, 1e-8)
    fresh = smol.System(U, V, 0.0, tau0=0.01)
    fresh.set_sources({1: 1.0, 100: 0.01})
    b, sb = fresh.integrate(n0, 0.0, 1.0, 1e-8)
    assert sa["status"] == 0 and sa["accepted"] == sb["accepted"]
    assert torch.equal(a, b)
