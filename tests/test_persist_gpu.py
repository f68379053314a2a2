"""The persistent attempt kernel (SMOL_FLAG_PERSISTENT): a chunk of RKF45 attempts of one
system in one cooperative launch whose CTAs run the phases back to back between grid
barriers. It runs the graph path's device functions on the same element-to-unit maps,
so its integrations must take the same decisions and give the same states."""
import numpy as np
import pytest

import oracle
from synth import kernel_factors, monodisperse, sample_state

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


def _run(smol, U, V, lam, n0, t1, tol, precision, flags, **opts):
    import torch
    s = smol.System(U, V, lam, precision=precision, flags=flags, **opts)
    n, st = s.integrate(torch.from_numpy(n0).cuda(), 0.0, t1, tol, scheme="rkf45")
    return n, st


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
@pytest.mark.parametrize("M,kind,a,lam,t1", [(1 << 17, "brownian", 0.9, 0.005, 0.02), (5000, "brownian_const", 1 / 3, 0.1, 2.0),
                                            (300, "brownian", 0.5, 0.01, 5.0), (2048, "brownian", 0.95, 0.01, 3.0)])
def test_persistent_equals_graph(smol, precision, M, kind, a, lam, t1):
    """Same accepted / rejected counts (rejections included, where the step starts at the
    stability bound: a retry reuses its first stage) and the same state as the graph
    path, across several chunks."""
    import torch
    U, V = kernel_factors(kind, M, a=a)
    n0 = monodisperse(M)
    ng, sg = _run(smol, U, V, lam, n0, t1, 1e-8, precision, 0, tau0=1e-4, chunk=16)
    npst, sp = _run(smol, U, V, lam, n0, t1, 1e-8, precision, smol.FLAG_PERSISTENT, tau0=1e-4, chunk=16)
    assert sg["status"] == 0 and sp["status"] == 0, (sg, sp)
    for k in ("accepted", "rejected", "rhs_evals", "attempts"):
        assert sp[k] == sg[k], (k, sp[k], sg[k])
    assert torch.allclose(npst, ng, rtol=0, atol=1e-13 * float(ng.abs().max()))
    assert sp["t"] == sg["t"] and sp["tau_next"] == pytest.approx(sg["tau_next"], rel=1e-12)


def test_persistent_vs_oracle(smol):
    """Against the oracle (FP64, direct sums): counts within 2% and the state within the
    tolerance's reach."""
    import torch
    M = 512
    U, V = kernel_factors("brownian", M, a=0.5)
    s = smol.System(U, V, 0.01, flags=smol.FLAG_PERSISTENT, tau0=1e-3)
    n, st = s.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 20.0, 1e-8, scheme="rkf45")
    osys = oracle.System(M, 0.01, U=U, V=V, route="direct")
    m, ost, _ = oracle.integrate(osys, monodisperse(M), 0.0, 20.0, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-3))
    assert st["status"] == 0 and ost["status"] == 0
    assert abs(st["accepted"] - ost["accepted"]) <= max(2, 0.02 * ost["accepted"])
    assert np.linalg.norm(n.cpu().numpy() - m) <= 1e-7 * np.linalg.norm(m)


def test_persistent_steady_stop_equals_graph(smol):
    """The steady stop (||S(n)|| / ||n|| below steady_rtol, tested on each attempt's first
    stage) ends the persistent run at the same attempt as the graph run."""
    import torch
    M = 2048
    U, V = kernel_factors("brownian_const", M, a=1 / 3)
    r = []
    for fl in (0, smol.FLAG_PERSISTENT):
        s = smol.System(U, V, 0.1, flags=fl, steady_rtol=1e-6, tau0=1e-3)
        r.append(s.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 1e4, 1e-8, scheme="rkf45"))
    (ng, sg), (npst, sp) = r
    assert sg["status"] == 1 and sp["status"] == 1  # SMOL_STEADY
    assert sp["t"] == sg["t"] and sp["accepted"] == sg["accepted"] and sp["rejected"] == sg["rejected"]
    assert torch.allclose(npst, ng, rtol=0, atol=1e-13 * float(ng.abs().max()))


def test_persistent_flag_ignored_where_it_does_not_apply(smol):
    """Batches, step doubling and constant steps keep the graph path: same results with
    and without the flag."""
    import torch
    M = 400
    U, V = kernel_factors("brownian", M, a=0.4)
    for scheme, extra in (("rk4", {}), ("rkf45", {"fixed_tau": 0.01})):
        r = []
        for fl in (0, smol.FLAG_PERSISTENT):
            s = smol.System(U, V, 0.02, flags=fl, tau0=1e-3, **extra)
            n, st = s.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 0.5, 1e-8, scheme=scheme)
            r.append((n, st))
        assert torch.equal(r[0][0], r[1][0]) and r[0][1]["accepted"] == r[1][1]["accepted"]
    fs = [kernel_factors("brownian", m, a=0.5) for m in (100, 300)]
    out = []
    for fl in (0, smol.FLAG_PERSISTENT):
        b = smol.Batch([f[0] for f in fs], [f[1] for f in fs], [0.01, 0.02], flags=fl, tau0=1e-3)
        ns, st = b.integrate([torch.from_numpy(monodisperse(m)).cuda() for m in (100, 300)], 0.0, 1.0, 1e-8)
        out.append(ns)
    for x, y in zip(*out):
        assert torch.equal(x, y)


def test_persistent_resume_and_rhs_unchanged(smol):
    """start / advance / finish with the persistent kernel, a resumed run, and the
    standalone evaluation of the same system object."""
    import torch
    M = 2048
    U, V = kernel_factors("brownian", M, a=0.7)
    s = smol.System(U, V, 0.01, flags=smol.FLAG_PERSISTENT, tau0=1e-3, chunk=8)
    g = smol.System(U, V, 0.01, tau0=1e-3, chunk=8)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    a, sa = s.integrate(n0, 0.0, 1.0, 1e-8)
    b, sb = g.integrate(n0, 0.0, 1.0, 1e-8)
    assert sa["accepted"] == sb["accepted"]
    s.set_tau0(sa["tau_next"])
    g.set_tau0(sb["tau_next"])
    a2, _ = s.integrate(a, 1.0, 2.0, 1e-8)
    b2, _ = g.integrate(b, 1.0, 2.0, 1e-8)
    assert torch.allclose(a2, b2, rtol=0, atol=1e-13 * float(b2.abs().max()))
    x = torch.from_numpy(sample_state(M, 0.01)).cuda()
    assert torch.equal(s.rhs(x), g.rhs(x))
