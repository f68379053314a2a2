"""The batched integrator (smol_batch_*): independent systems of uneven size, kernel
exponent and shattering rate advanced together, each with its own adaptive step.

Each system of a batch must follow the same trajectory as when it is integrated alone
(same kernels, same arithmetic; only the CTA sizes of a launch, and so the order of
the block reductions, may differ) and must match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from synth import batch_recipe, kernel_factors, monodisperse, sample_state

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


def _systems(specs):
    Us, Vs, lams, n0s = [], [], [], []
    for M, a, lam in specs:
        U, V = kernel_factors("brownian", M, a=a)
        Us.append(U)
        Vs.append(V)
        lams.append(lam)
        n0s.append(monodisperse(M))
    return Us, Vs, lams, n0s


SPECS = [(1000, 0.3, 0.01), (4096, 0.7, 0.05), (513, 0.5, 0.1), (16384, 0.9, 0.005), (64, 0.2, 0.02)]


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_batch_equals_single_systems(smol, precision):
    import torch
    Us, Vs, lams, n0s = _systems(SPECS)
    b = smol.Batch(Us, Vs, lams, precision=precision, tau0=1e-3)
    ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, 0.5, 1e-8, scheme="rkf45")
    for q, (U, V, lam, n0) in enumerate(zip(Us, Vs, lams, n0s)):
        s = smol.System(U, V, lam, precision=precision, tau0=1e-3)
        m, st = s.integrate(torch.from_numpy(n0), 0.0, 0.5, 1e-8, scheme="rkf45")
        assert sts[q]["status"] == st["status"] == 0
        assert (sts[q]["accepted"], sts[q]["rejected"]) == (st["accepted"], st["rejected"]), (q, sts[q], st)
        assert sts[q]["rhs_evals"] == st["rhs_evals"]
        assert torch.allclose(ns[q], m, rtol=0, atol=1e-12 * float(m.abs().max()))


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_batch_retries_keep_first_stage(smol, precision):
    """A large initial step makes every system reject its first attempts, each on its
    own schedule (here one rejection for the first system, two for the others), so one
    launch holds systems whose first-stage kernels return at once (a retry keeps
    S(n^k); Sec. 2 repeats the step from n^k) beside systems that evaluate. Each system
    takes the oracle's decisions and makes its number of evaluations."""
    import torch
    specs = [(300, 0.3, 0.01), (1000, 0.4, 0.05), (77, 0.5, 0.2)]
    Us, Vs, lams, n0s = _systems(specs)
    b = smol.Batch(Us, Vs, lams, precision=precision, tau0=0.3)
    ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, 3.0, 1e-8, scheme="rkf45")
    for q, (U, V, lam, n0) in enumerate(zip(Us, Vs, lams, n0s)):
        osys = oracle.System(len(n0), lam, U=U, V=V, route="lowrank")
        m, ost, olog = oracle.integrate(osys, n0, 0.0, 3.0, 1e-8,
                                        oracle.Options(scheme="rkf45", tau0=0.3, log=True))
        assert sum(1 for prev in olog[:-1] if not prev[3]) >= 1
        assert (sts[q]["accepted"], sts[q]["rejected"]) == (ost["accepted"], ost["rejected"])
        assert sts[q]["rhs_evals"] == ost["rhs_evals"] < ost["rhs_evals_paper"]
        assert np.linalg.norm(ns[q].cpu().numpy() - m) <= 1e-9 * np.linalg.norm(m)


def test_batch_fp64_vs_oracle(smol):
    """Non-stiff parameters: with a steep kernel (a = 0.8, M = 1000) the tail modes are
    stiff and the rounding noise of any FFT route excites them, so the number of rejected
    attempts depends on the FFT's rounding (the oracle's own numpy-FFT and direct routes
    disagree there: 39 and 0 rejections); accepted / rejected counts are compared where
    the step control is not at its stability limit."""
    import torch
    specs = [(300, 0.3, 0.01), (1000, 0.4, 0.05), (77, 0.5, 0.2)]
    Us, Vs, lams, n0s = _systems(specs)
    b = smol.Batch(Us, Vs, lams, tau0=1e-2)
    ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, 3.0, 1e-8, scheme="rkf45")
    for q, (U, V, lam, n0) in enumerate(zip(Us, Vs, lams, n0s)):
        osys = oracle.System(len(n0), lam, U=U, V=V, route="lowrank")
        m, ost, _ = oracle.integrate(osys, n0, 0.0, 3.0, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-2))
        assert (sts[q]["accepted"], sts[q]["rejected"]) == (ost["accepted"], ost["rejected"])
        x = ns[q].cpu().numpy()
        assert np.linalg.norm(x - m) <= 1e-9 * np.linalg.norm(m)
        s = np.arange(1, len(m) + 1)
        assert abs(sts[q]["mass"] - float(np.dot(s, m))) <= 1e-12 * float(np.dot(s, m))


def test_batch_recipe_sample_fp32conv(smol):
    """A sample of the 256-system workload (M log-uniform in [2^10, 2^16], exponent in
    [0.2, 0.9], lambda log-uniform in [0.005, 0.1]), FP32 convolutions with FP64 control,
    against the FP64 oracle at the reduced-precision bar 1e-4. Without the exponential
    tilt of the transform inputs the FP32 rounding (1e-7 of the largest values) would land
    in every size bin, the near-empty tail included, and reach n_1 through the monomers'
    collisions with large clusters (K_1j ~ j^a): up to 1.2e-4 after t = 2. Systems up to
    M = 8192 run to t = 2, the larger ones to t = 0.3 (the oracle's numpy FFT is slow
    there)."""
    import torch
    rec = batch_recipe(256)[:8]
    for t1, keep in ((2.0, lambda M: M <= 8192), (0.3, lambda M: M > 8192)):
        specs = [(r["M"], r["a"], r["lam"]) for r in rec if keep(r["M"])]
        Us, Vs, lams, n0s = _systems(specs)
        b = smol.Batch(Us, Vs, lams, precision="fp32conv", tau0=1e-3)
        ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, t1, 1e-8, scheme="rkf45")
        for q, (U, V, lam, n0) in enumerate(zip(Us, Vs, lams, n0s)):
            assert sts[q]["status"] == 0 and sts[q]["t"] == t1
            osys = oracle.System(len(n0), lam, U=U, V=V, route="lowrank")
            m, ost, _ = oracle.integrate(osys, n0, 0.0, t1, 1e-8, oracle.Options(scheme="rkf45", tau0=1e-3))
            x = ns[q].cpu().numpy()
            rel = np.linalg.norm(x - m) / np.linalg.norm(m)
            assert rel <= 1e-4, (len(n0), t1, rel)


@pytest.mark.parametrize("scheme", ["rk2", "rk4"])
def test_batch_step_doubling_vs_single(smol, scheme):
    import torch
    Us, Vs, lams, n0s = _systems(SPECS[:3])
    b = smol.Batch(Us, Vs, lams, tau0=1e-2, ctrl="formula")
    ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, 1.0, 1e-8, scheme=scheme)
    for q, (U, V, lam, n0) in enumerate(zip(Us, Vs, lams, n0s)):
        s = smol.System(U, V, lam, tau0=1e-2, ctrl="formula")
        m, st = s.integrate(torch.from_numpy(n0), 0.0, 1.0, 1e-8, scheme=scheme)
        assert (sts[q]["accepted"], sts[q]["rejected"]) == (st["accepted"], st["rejected"])
        assert torch.allclose(ns[q], m, rtol=0, atol=1e-12 * float(m.abs().max()))


def test_batch_systems_stop_independently(smol):
    """One system hits its attempt limit, another a non-finite state; the rest finish."""
    import torch
    Us, Vs, lams, n0s = _systems(SPECS[:3])
    n0s[1] = n0s[1].copy()
    n0s[1][5] = np.nan
    b = smol.Batch(Us, Vs, lams, tau0=1e-2)
    ns, sts = b.integrate([torch.from_numpy(n) for n in n0s], 0.0, 1.0, 1e-8, scheme="rkf45")
    assert sts[1]["status"] == smol.ENONFINITE
    assert sts[0]["status"] == 0 and sts[2]["status"] == 0 and sts[0]["t"] == 1.0


def test_batch_tune_keeps_results(smol):
    """smol_batch_tune keeps the fastest launch mode; the batch's trajectories do not
    depend on it (bit-identical, or equal to rounding if it unfused the column passes)."""
    import torch
    Us, Vs, lams, n0s = _systems(SPECS)
    st0 = [torch.from_numpy(n) for n in n0s]
    a = smol.Batch(Us, Vs, lams, tau0=1e-3)
    ra, sa = a.integrate(st0, 0.0, 0.3, 1e-8)
    b = smol.Batch(Us, Vs, lams, tau0=1e-3)
    fl, us = b.tune(st0, 1e-8, attempts=4)
    assert fl in (0, smol.FLAG_NO_PDL, smol.FLAG_NO_PDL_FWD_COLS, smol.FLAG_NO_FUSE,
                  smol.FLAG_NO_FUSE | smol.FLAG_NO_PDL) and us > 0.0
    rb, sb = b.integrate(st0, 0.0, 0.3, 1e-8)
    for x, y, p, q in zip(ra, rb, sa, sb):
        assert p["accepted"] == q["accepted"]
        if fl & smol.FLAG_NO_FUSE:  # another order of the final block sums: equal to rounding
            assert torch.linalg.norm(x - y) <= 1e-12 * torch.linalg.norm(x)
        else:
            assert torch.equal(x, y)


def test_batch_tune_schedules_keeps_results(smol):
    """smol_batch_tune_schedules picks a schedule per size class among its candidates
    (log2 N1 from two below the rule to one above, 1, 2, 4 or 8 times the rule's columns
    per CTA); classes
    the batch does not hold keep the rule. A batch built with the tables follows the
    rule's trajectories: another split Mp = N1 N2 changes only the rounding of the
    transforms. Where a step's error sits at the accept bound that rounding can decide it
    the other way, and the step sequences part from there: the counts stay within 2%,
    and the states within the global bound of two runs whose decisions part, 2 A tol
    (A accepted steps, tol per accepted step; at least 10 tol)."""
    import torch
    Us, Vs, lams, n0s = _systems(SPECS)
    st0 = [torch.from_numpy(n) for n in n0s]
    tables, us = smol.batch_tune_schedules(Us, Vs, lams, st0, 1e-8, attempts=4, tau0=1e-3)
    assert us > 0.0
    held = {int(np.ceil(np.log2(max(M, 4)))) for M, _, _ in SPECS}
    for k in range(smol.SIZE_CLASSES):
        lg, g = tables["batch_lgn1"][k], tables["batch_g"][k]
        if k not in held:
            assert lg == 0 and g == 0, (k, lg, g)
            continue
        assert lg == 0 or 1 <= lg < k, (k, lg)
        assert g == 0 or (g & (g - 1)) == 0 and g <= 64, (k, g)
    a = smol.Batch(Us, Vs, lams, tau0=1e-3)
    ra, sa = a.integrate(st0, 0.0, 0.3, 1e-8)
    b = smol.Batch(Us, Vs, lams, tau0=1e-3, **tables)
    rb, sb = b.integrate(st0, 0.0, 0.3, 1e-8)
    tol = 1e-8
    for x, y, p, q in zip(ra, rb, sa, sb):
        assert p["status"] == 0 and q["status"] == 0
        assert abs(p["accepted"] - q["accepted"]) <= max(2, 0.02 * p["accepted"]), (p["accepted"], q["accepted"])
        assert float(torch.linalg.norm(x - y)) <= max(10 * tol, 2 * p["accepted"] * tol)
    with pytest.raises(smol.SmolError):
        smol.Batch(Us, Vs, lams, batch_g=[3] * smol.SIZE_CLASSES)

