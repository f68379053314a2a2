"""Parity of the device-resident adaptive integrators (Sec. 2) with the FP64 oracle.

Modes:
  * constant steps (fixed_tau): the same arithmetic step by step, so the states agree
    to the RHS tolerance times the number of steps;
  * free-running adaptive runs on the relaxation problem: both sides take the same
    accept / reject decisions (counts equal) and the states agree far below tol;
  * the closed-form constant-kernel solution;
  * error statuses (non-finite state, step underflow, attempt limit) and the steady stop.
The error estimate is compared at 1e-5 relative and the step sizes at 1e-3: the oracle
forms err = ||n_RK5 - n^{k+1}|| from two separately rounded O(1) states (about 1e-8
relative noise when err ~ tol), the device from the weight differences, and each step
factor (tol/err)^(1/p) carries that noise into every later step.
"""
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


def run_both(smol, M, kind, a, lam, t1, tol, scheme, n0=None, route="lowrank", **opts):
    import torch
    U, V = kernel_factors(kind, M, a=a)
    n0 = monodisperse(M) if n0 is None else n0
    gopts = {k: v for k, v in opts.items() if k not in ("log",)}
    sysm = smol.System(U, V, lam, log_capacity=4096, **gopts)
    n, st = sysm.integrate(torch.from_numpy(n0).cuda(), 0.0, t1, tol, scheme=scheme)
    osys = oracle.System(M, lam, U=U, V=V, route=route)
    oo = oracle.Options(scheme=scheme, log=True, **{k: v for k, v in opts.items() if k in oracle.Options.__dataclass_fields__})
    m, ost, olog = oracle.integrate(osys, n0, 0.0, t1, tol, oo)
    return n.cpu().numpy(), st, m, ost, olog, sysm


@pytest.mark.parametrize("scheme", ["rk2", "rk4", "rkf45"])
def test_fixed_step_parity(smol, scheme):
    M = 512
    n, st, m, ost, _, _ = run_both(smol, M, "brownian", 0.3, 0.01, 5.0, 1e-8, scheme, fixed_tau=0.01)
    assert st["status"] == 0 and ost["status"] == 0
    assert st["accepted"] == ost["accepted"] and st["accepted"] in (500, 501)
    assert st["rhs_evals_paper"] == ost["rhs_evals_paper"]
    assert np.linalg.norm(n - m) <= 1e-11 * np.linalg.norm(m) * 500 ** 0.5


@pytest.mark.parametrize("scheme,ctrl", [("rk2", "double_halve"), ("rk2", "formula"), ("rk4", "double_halve"),
                                         ("rk4", "formula"), ("rkf45", "double_halve")])
def test_adaptive_parity_relaxation(smol, scheme, ctrl):
    """The shattering workload at M = 512 (kernel (i/j)^0.3 + (j/i)^0.3, lambda = 0.01,
    monodisperse start) on t in [0, 20]."""
    M = 512
    n, st, m, ost, olog, sysm = run_both(smol, M, "brownian", 0.3, 0.01, 20.0, 1e-8, scheme, ctrl=ctrl, tau0=0.01)
    assert st["status"] == ost["status"] == 0
    assert st["t"] == ost["t"] == 20.0
    assert (st["accepted"], st["rejected"]) == (ost["accepted"], ost["rejected"]), (st, ost)
    assert st["rhs_evals"] == ost["rhs_evals"] and st["rhs_evals_paper"] == ost["rhs_evals_paper"]
    assert np.linalg.norm(n - m) <= 1e-9 * np.linalg.norm(m), np.linalg.norm(n - m) / np.linalg.norm(m)
    # step log: same decisions and step sizes
    t, h, e, acc, cnt = sysm.get_log()
    assert cnt == len(olog)
    k = len(t)
    oh = np.array([x[1] for x in olog])[-k:]
    oe = np.array([x[2] for x in olog])[-k:]
    oa = np.array([x[3] for x in olog])[-k:]
    assert np.array_equal(acc, oa)
    # where err approaches the oracle's rounding floor its relative noise is large and
    # (tol/err)^(1/p) carries it into the next step; decisions and states agree above
    assert np.allclose(h, oh, rtol=1e-3, atol=0)
    # before err first nears the rounding floor the step sizes agree far more closely
    # (the oracle's err itself carries ~1e-8 relative noise: two O(1) states subtracted)
    assert np.allclose(h[:10], oh[:10], rtol=1e-6, atol=0)
    # atol: the oracle forms err from O(1) states, so below ~1e-14 it is rounding noise
    assert np.allclose(e, oe, rtol=1e-5, atol=1e-14)


def test_euler_initial_step(smol):
    """No tau0: the Euler criterion tau0 = a / max_i sum_j K_ij n_j (a = 1/10)."""
    M = 256
    n, st, m, ost, olog, sysm = run_both(smol, M, "brownian", 0.3, 0.01, 1.0, 1e-8, "rkf45")
    t, h, *_ = sysm.get_log()
    assert abs(h[0] - olog[0][1]) <= 1e-14 * olog[0][1]
    assert (st["accepted"], st["rejected"]) == (ost["accepted"], ost["rejected"])


@pytest.mark.parametrize("scheme,tol", [("rk2", 1e-9), ("rk4", 1e-10), ("rkf45", 1e-10)])
def test_closed_form_constant_kernel(smol, scheme, tol):
    import torch
    M, t1 = 128, 3.0
    U, V = kernel_factors("const", M)
    sysm = smol.System(U, V, 0.0)
    n, st = sysm.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, t1, tol, scheme=scheme)
    s = np.arange(1, M + 1, dtype=np.float64)
    ref = (t1 / 2) ** (s - 1) / (1 + t1 / 2) ** (s + 1)
    assert st["status"] == 0
    assert np.linalg.norm(n.cpu().numpy() - ref) <= 200 * tol * max(1, st["accepted"]) ** 0.5


def test_statuses(smol):
    import torch
    M = 64
    U, V = kernel_factors("brownian", M, a=0.3)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    s = smol.System(U, V, 0.01)
    _, st = s.integrate(n0, 0.0, 10.0, 1e-300, scheme="rkf45")
    assert st["status"] == smol.ESTEP_UNDERFLOW
    s = smol.System(U, V, 0.01, max_attempts=3)
    _, st = s.integrate(n0, 0.0, 10.0, 1e-8, scheme="rkf45")
    assert st["status"] == smol.EMAXATTEMPTS and st["attempts"] == 3
    bad = monodisperse(M)
    bad[3] = np.nan
    s = smol.System(U, V, 0.01, tau0=0.01)
    _, st = s.integrate(torch.from_numpy(bad).cuda(), 0.0, 10.0, 1e-8, scheme="rk2")
    assert st["status"] == smol.ENONFINITE
    # t1 == t0: nothing to do
    n, st = s.integrate(n0, 1.0, 1.0, 1e-8)
    assert st["status"] == 0 and st["attempts"] == 0 and torch.equal(n, n0)


def test_steady_stop(smol):
    M, lam = 64, 1.0
    n, st, m, ost, _, _ = run_both(smol, M, "const", 0.0, lam, 1e4, 1e-9, "rkf45", steady_rtol=1e-8, tau0=0.01)
    assert st["status"] == ost["status"] == smol.STEADY
    assert abs(st["t"] - ost["t"]) <= 1e-6 * ost["t"]
    assert np.linalg.norm(n - m) <= 1e-7 * np.linalg.norm(m)


def test_resume_equals_single_run(smol):
    """Checkpoint / resume: a run split at t = 1 with tau0 = tau_next continues the
    same step sequence."""
    import torch
    M = 256
    U, V = kernel_factors("brownian", M, a=0.3)
    s = smol.System(U, V, 0.01, tau0=0.01)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    full, st = s.integrate(n0, 0.0, 2.0, 1e-8)
    half, st1 = s.integrate(n0, 0.0, 1.0, 1e-8)
    s2 = smol.System(U, V, 0.01, tau0=st1["tau_next"])
    rest, st2 = s2.integrate(half, st1["t"], 2.0, 1e-8)
    assert st2["status"] == 0
    assert torch.allclose(rest, full, rtol=0, atol=1e-8 * float(full.norm()))


def test_resume_with_set_tau0(smol):
    """smol_set_tau0 resumes the same system object from a checkpoint: a run split at
    t = 1 takes exactly the steps of a new system created with tau0 = tau_next
    (bit-identical state) and stays within the tolerance of the unsplit run; a batch
    resumes each system with its own tau_next."""
    import torch
    M = 256
    U, V = kernel_factors("brownian", M, a=0.3)
    s = smol.System(U, V, 0.01, tau0=0.01)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    full, st = s.integrate(n0, 0.0, 2.0, 1e-8)
    half, st1 = s.integrate(n0, 0.0, 1.0, 1e-8)
    s.set_tau0(st1["tau_next"])
    rest, st2 = s.integrate(half, st1["t"], 2.0, 1e-8)
    s2 = smol.System(U, V, 0.01, tau0=st1["tau_next"])
    rest2, _ = s2.integrate(half, st1["t"], 2.0, 1e-8)
    assert st2["status"] == 0
    assert torch.equal(rest, rest2)
    assert torch.allclose(rest, full, rtol=0, atol=1e-8 * float(full.norm()))
    s.set_tau0(0.0)  # back to the tau0 option
    again, st3 = s.integrate(n0, 0.0, 2.0, 1e-8)
    assert torch.equal(again, full) and st3["accepted"] == st["accepted"]
    Ms = [100, 300]
    fs = [kernel_factors("brownian", m, a=0.5) for m in Ms]
    b = smol.Batch([f[0] for f in fs], [f[1] for f in fs], [0.01, 0.02], tau0=0.01)
    n0s = [torch.from_numpy(monodisperse(m)).cuda() for m in Ms]
    bf, sf = b.integrate(n0s, 0.0, 2.0, 1e-8)
    bh, sh = b.integrate(n0s, 0.0, 1.0, 1e-8)
    b.set_tau0([x["tau_next"] for x in sh])
    br, sr = b.integrate(bh, 1.0, 2.0, 1e-8)
    for q in range(2):
        sq = smol.System(fs[q][0], fs[q][1], [0.01, 0.02][q], tau0=sh[q]["tau_next"])
        rq, _ = sq.integrate(bh[q], 1.0, 2.0, 1e-8)
        assert torch.allclose(br[q], rq, rtol=0, atol=1e-12 * float(rq.abs().max())), q
        assert torch.allclose(br[q], bf[q], rtol=0, atol=1e-6 * float(bf[q].norm())), q


def test_fp32conv_integrate_accuracy(smol):
    """FP32 convolutions with FP64 control on the relaxation workload: the state stays
    within the reduced-precision tolerance 1e-4 (relative, normwise) of the FP64 oracle."""
    M = 4096
    n, st, m, ost, _, _ = run_both(smol, M, "brownian_const", 1 / 3, 0.1, 10.0, 1e-8, "rkf45",
                                   precision="fp32conv", tau0=0.01)
    assert st["status"] == 0 and ost["status"] == 0
    assert np.linalg.norm(n - m) <= 1e-4 * np.linalg.norm(m)


@pytest.mark.parametrize("precision", ["fp64", "fp32conv"])
@pytest.mark.parametrize("scheme", ["rkf45", "rk4", "rk2"])
def test_launch_modes_do_not_change_results(smol, precision, scheme):
    """Programmatic dependent launch only changes when CTAs are scheduled: every launch
    mode gives bit-identical trajectories. Fusing the column passes changes only the
    order of the final kernel's block sums (column CTAs instead of finish CTAs): the
    fused and unfused trajectories agree to rounding, with the same decisions."""
    import torch
    M = 8192
    U, V = kernel_factors("brownian", M, a=0.6)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    runs = {}
    for flags in (0, smol.FLAG_NO_PDL, smol.FLAG_NO_PDL_FWD_COLS, smol.FLAG_NO_PDL_ROWS | smol.FLAG_NO_PDL_STEP,
                  smol.FLAG_NO_FUSE, smol.FLAG_NO_FUSE | smol.FLAG_NO_PDL):
        n, st = smol.System(U, V, 0.01, precision=precision, tau0=1e-3, flags=flags).integrate(
            n0, 0.0, 2.0, 1e-8, scheme=scheme)
        assert st["status"] == 0
        runs[flags] = (n.cpu().numpy(), st["accepted"], st["rejected"])
    for flags, got in runs.items():
        ref = runs[flags & smol.FLAG_NO_FUSE]
        assert np.array_equal(got[0], ref[0]) and got[1:] == ref[1:], flags
    a, b = runs[0], runs[smol.FLAG_NO_FUSE]
    assert a[1:] == b[1:]
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.linalg.norm(a[0] - b[0]) <= tol * np.linalg.norm(b[0])


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_wide_column_ctas_match_default(smol, precision):
    """SMOL_FLAG_WIDE_COLS (512-thread column CTAs on a schedule with 512 element pairs a
    tile, ragged M) only changes the order of block sums: the right-hand side and the
    trajectory agree with the default launch to rounding, with the same decisions (the
    FP32 form ignores the flag)."""
    import torch
    M = 100000
    U, V = kernel_factors("brownian", M, a=0.9)
    n0 = torch.from_numpy(sample_state(M, 0.01)).cuda()
    sched = dict(fft_lgn1=8, fft_g=4)
    out = {}
    for flags in (0, smol.FLAG_WIDE_COLS, smol.FLAG_WIDE_COLS | smol.FLAG_NO_FUSE):
        s = smol.System(U, V, 0.005, precision=precision, tau0=1e-5, flags=flags, **sched)
        r = s.rhs(n0).cpu().numpy()
        n, st = s.integrate(n0, 0.0, 2e-3, 1e-8, scheme="rkf45")
        assert st["status"] == 0
        out[flags] = (r, n.cpu().numpy(), st["accepted"], st["rejected"])
    tol = {"fp64": 1e-12, "df64": 1e-12, "fp32conv": 1e-6}[precision]
    base = out[0]
    for flags, got in out.items():
        assert got[2:] == base[2:], (flags, got[2:], base[2:])
        assert np.linalg.norm(got[0] - base[0]) <= tol * np.linalg.norm(base[0]), flags
        assert np.linalg.norm(got[1] - base[1]) <= tol * np.linalg.norm(base[1]), flags


def test_tune_picks_a_valid_schedule(smol):
    """smol_tune returns one of its candidates, and the tuned system follows the
    default one's constant-step trajectory to rounding."""
    import torch
    M = 4096
    U, V = kernel_factors("brownian", M, a=0.5)
    n0 = torch.from_numpy(sample_state(M, 0.01)).cuda()
    sched, us = smol.tune(U, V, 0.01, n0, 1e-8, attempts=8)
    assert us > 0.0
    assert sched["fft_lgn1"] in (4, 5, 6, 7) and sched["fft_g"] in (2, 4, 8, 16, 32, 64)
    assert sched["flags"] in (0, smol.FLAG_NO_PDL, smol.FLAG_NO_PDL_FWD_COLS, smol.FLAG_NO_FUSE,
                              smol.FLAG_NO_FUSE | smol.FLAG_NO_PDL, smol.FLAG_PERSISTENT,
                              smol.FLAG_WIDE_COLS | smol.FLAG_NO_PDL, smol.FLAG_WIDE_COLS | smol.FLAG_NO_PDL_FWD_COLS)
    a, _ = smol.System(U, V, 0.01, fixed_tau=0.01, **sched).integrate(n0, 0.0, 1.0, 1e-8)
    b, _ = smol.System(U, V, 0.01, fixed_tau=0.01).integrate(n0, 0.0, 1.0, 1e-8)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32conv"])
def test_fused_kernels_at_full_size(smol, precision):
    """M = 2^17 (the bench size: column tiles beyond the default 48 KB of dynamic shared
    memory): fused and unfused column passes give the same RKF45 trajectory to rounding
    over constant steps; adaptive runs from the stiff monodisperse start both reach t1
    (their thousands of accept / reject decisions near err = tol may differ in a few
    places, since the two sum the error norm in different orders)."""
    import torch
    M = 131072
    U, V = kernel_factors("brownian", M, a=0.9)
    n0 = torch.from_numpy(monodisperse(M)).cuda()
    out = []
    for flags in (0, smol.FLAG_NO_FUSE):
        # 2e-6 is below the Euler bound 0.1 / max_s D_s(n0) = 0.1 / (M^0.9 + M^-0.9)
        n, st = smol.System(U, V, 0.005, precision=precision, fixed_tau=2e-6, flags=flags).integrate(
            n0, 0.0, 1e-4, 1e-8)
        assert st["status"] == 0 and st["accepted"] in (50, 51)
        out.append(n.cpu().numpy())
        n, st = smol.System(U, V, 0.005, precision=precision, tau0=1e-3, flags=flags).integrate(n0, 0.0, 0.05, 1e-8)
        assert st["status"] == 0 and abs(st["t"] - 0.05) < 1e-12
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.linalg.norm(out[0] - out[1]) <= tol * np.linalg.norm(out[1])


@pytest.mark.parametrize("scheme", ["rkf45", "rk4"])
def test_df64_adaptive_parity(smol, scheme):
    """The double-float form takes the oracle's accept / reject decisions and ends on
    its state at the FP64 parity bar."""
    n, st, m, ost, _, _ = run_both(smol, 512, "brownian", 0.3, 0.01, 20.0, 1e-8, scheme, precision="df64",
                                   tau0=0.01)
    assert st["status"] == ost["status"] == 0
    assert (st["accepted"], st["rejected"]) == (ost["accepted"], ost["rejected"])
    assert np.linalg.norm(n - m) <= 1e-9 * np.linalg.norm(m)


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_finish_then_advance_continues(smol, precision):
    """smol_integrate_finish leaves the state in the caller's vector and the run able to
    continue: start, two chunks, finish, one more chunk, finish equals start, three
    chunks, finish (bit for bit; the reduced-precision forms also carry their shadow
    of the state across)."""
    import torch
    M = 4096
    U, V = kernel_factors("brownian", M, a=0.5)
    outs = []
    for split in (True, False):
        s = smol.System(U, V, 0.02, precision=precision, tau0=1e-3, chunk=3)
        n = s.start(torch.from_numpy(monodisperse(M)).cuda(), 0.0, 50.0, 1e-8)
        s.advance()
        s.advance()
        if split:
            n, st = s.finish()
            assert st["attempts"] == 6
        s.advance()
        n, st = s.finish()
        outs.append((n.cpu().numpy(), st["attempts"], st["accepted"]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1:] == outs[1][1:]


@pytest.mark.parametrize("precision", ["fp64", "fp32conv", "df64"])
def test_mass_statistic_and_conservation(smol, precision):
    """stats.mass is sum_s s n_s of the returned state (FP64 in every form); with the
    distribution far from M the truncation flux is negligible and shattering conserves
    mass, so it stays 1 to the integration error."""
    import torch
    M = 8192
    U, V = kernel_factors("brownian", M, a=0.4)
    n, st = smol.System(U, V, 0.05, precision=precision, tau0=1e-3).integrate(
        torch.from_numpy(monodisperse(M)).cuda(), 0.0, 3.0, 1e-9)
    assert st["status"] == 0
    s = np.arange(1, M + 1, dtype=np.float64)
    m = float(np.dot(s, n.cpu().numpy()))
    assert abs(st["mass"] - m) <= 1e-13 * m
    assert abs(m - 1.0) <= (1e-7 if precision != "fp32conv" else 1e-4)


@pytest.mark.parametrize("fuse", [True, False])
@pytest.mark.parametrize("scheme", ["rkf45", "rk4", "rk2"])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_retry_keeps_first_stage(smol, precision, scheme, fuse):
    """A rejected attempt is repeated from the same n^k (Sec. 2): the retry keeps the
    rejected attempt's S(n^k), rescaled to the new step, where the oracle keeps its
    S(n). A large initial step forces a run of rejections; the decisions, the number of
    evaluations made and the final state match the oracle, in the fused and the
    unfused launch sequence."""
    M = 512
    flags = 0 if fuse else smol.FLAG_NO_FUSE
    n, st, m, ost, olog, sysm = run_both(smol, M, "brownian", 0.3, 0.01, 5.0, 1e-8, scheme, precision=precision,
                                         tau0=2.0, flags=flags)
    assert st["status"] == ost["status"] == 0
    retries = sum(1 for prev in olog[:-1] if not prev[3])
    assert retries >= 3
    assert (st["accepted"], st["rejected"]) == (ost["accepted"], ost["rejected"])
    assert st["rhs_evals"] == ost["rhs_evals"] and st["rhs_evals_paper"] == ost["rhs_evals_paper"]
    per = 6 if scheme == "rkf45" else 3 * oracle.STAGES[scheme] - 1
    assert st["rhs_evals"] == per * len(olog) - retries
    assert np.linalg.norm(n - m) <= 1e-9 * np.linalg.norm(m)
    _, h, _, acc, cnt = sysm.get_log()
    oh = np.array([x[1] for x in olog])
    assert cnt == len(olog) and np.array_equal(acc, [x[3] for x in olog])
    lead = next(i for i, x in enumerate(olog) if x[3])  # the first run of rejections
    assert lead >= 2 and np.allclose(h[:lead + 1], oh[:lead + 1], rtol=1e-6, atol=0)
