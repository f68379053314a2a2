"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself:
  * the closed-form solution of the constant-kernel problem (Sec. 1 cites it as an
    exactly solvable case): n_s(t) = (t/2)^{s-1} / (1 + t/2)^{s+1};
  * the mass balance of Eq. (4): shattering moves mass to monomers without loss, so
    sum_s s S_s(n) equals the truncation flux exactly;
  * a brute-force pure-Python restatement of Eq. (4) on tiny M (explicit loops);
  * the direct O(M^2) route against the low-rank FFT route (Sec. 1, Sec. 2) on
    non-symmetric random factors, so a transposed U/V fails the death term;
  * the stability polynomials of the Sec. 2 schemes on y' = z y (tests/golden);
  * the worked examples of the RKF45 step rule (Sec. 2, last paragraph; tests/golden);
  * observed convergence orders 2 / 4 / 4 on a smooth ODE;
  * conservation of the linear invariant sum_s s n_s + F by every explicit RK step.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import kernel_factors, monodisperse, random_factors, random_state, sample_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def closed_form(M, t):
    s = np.arange(1, M + 1, dtype=np.float64)
    h = t / 2.0
    return h ** (s - 1) / (1.0 + h) ** (s + 1)


def closed_form_dt(M, t):
    """d/dt of the closed form, differentiated by hand:
    n_s = h^{s-1} (1+h)^{-(s+1)}, h = t/2, dh/dt = 1/2 ->
    dn_s/dt = 1/2 [ (s-1) h^{s-2} (1+h)^{-(s+1)} - (s+1) h^{s-1} (1+h)^{-(s+2)} ]."""
    s = np.arange(1, M + 1, dtype=np.float64)
    h = t / 2.0
    a = np.where(s > 1, (s - 1) * h ** np.maximum(s - 2, 0) / (1.0 + h) ** (s + 1), 0.0)
    b = (s + 1) * h ** (s - 1) / (1.0 + h) ** (s + 2)
    return 0.5 * (a - b)


def brute_force_rhs(n, kfun, lam):
    """Eq. (4) written with explicit loops over 1-based sizes (tiny M only)."""
    M = len(n)
    N = {s: n[s - 1] for s in range(1, M + 1)}
    out = []
    for s in range(1, M + 1):
        loss = N[s] * sum(kfun(s, i) * N[i] for i in range(1, M + 1))
        if s == 1:
            src = 0.0
            for i in range(2, M + 1):
                for j in range(2, M + 1):
                    src += 0.5 * lam * (i + j) * kfun(i, j) * N[i] * N[j]
            src += lam * N[1] * sum(j * kfun(1, j) * N[j] for j in range(2, M + 1))
            out.append(-loss + src)
        else:
            birth = 0.5 * sum(kfun(i, s - i) * N[i] * N[s - i] for i in range(1, s))
            out.append(birth - loss - lam * loss)
    return np.array(out)


# ---------------------------------------------------------------------------
# Right-hand side
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("t", [0.5, 2.0, 5.0])
def test_rhs_matches_closed_form_derivative(t):
    """K = 1, lambda = 0 on the closed-form state: S(n) = dn/dt up to the death sum's
    truncation n_s sum_{i>M} n_i, which is below 1e-20 at M = 256 for t <= 5."""
    M = 256
    n = closed_form(M, t)
    U, V = kernel_factors("const", M)
    for terms in (oracle.rhs_terms_direct(n, U @ V, 0.0), oracle.rhs_terms_lowrank(n, U, V, 0.0)):
        S = terms["total"]
        ref = closed_form_dt(M, t)
        assert np.max(np.abs(S - ref)) <= 1e-14 * np.max(np.abs(ref)) + 1e-20


@pytest.mark.parametrize("kind,a", [("const", 0.0), ("brownian", 0.3), ("brownian", 0.9), ("brownian_const", 1 / 3)])
@pytest.mark.parametrize("lam", [0.0, 0.01, 0.5])
def test_mass_flux_identity(kind, a, lam):
    """Eq. (4) with a symmetric kernel: sum_s s S_s(n) = -1/2 sum_{i+j>M} (i+j) K_ij n_i n_j.
    Fails if the n_1 factor of the monomer source, the (i+j) weight, or the shattering
    loss is dropped or mis-signed."""
    M = 40
    n = random_state(M, seed=7, decay=12.0)
    U, V = kernel_factors(kind, M, a=a)
    K = oracle.kernel_closed_form(kind, M, a=a)
    s = np.arange(1, M + 1, dtype=np.float64)
    flux = oracle.mass_flux_direct(n, K)
    for S in (oracle.rhs_terms_direct(n, K, lam)["total"], oracle.rhs_terms_lowrank(n, U, V, lam)["total"]):
        lhs = float(np.dot(s, S))
        scale = float(np.dot(s, np.abs(S))) + abs(flux)
        assert abs(lhs - flux) <= 1e-13 * scale


def test_mass_identity_fails_without_n1_factor():
    """The reading of the monomer equation matters: the literal printed term
    lambda sum_{j>=2} j K_{1j} n_j (no n_1) breaks the mass balance."""
    M, lam = 30, 0.3
    n = random_state(M, seed=3, decay=8.0)
    K = oracle.kernel_closed_form("brownian", M, a=0.4)
    s = np.arange(1, M + 1, dtype=np.float64)
    S = oracle.rhs_terms_direct(n, K, lam)["total"].copy()
    w = lam * np.sum(s[1:] * K[0, 1:] * n[1:])
    S[0] += w - n[0] * w          # swap lambda n_1 sum(...) for the literal lambda sum(...)
    flux = oracle.mass_flux_direct(n, K)
    assert abs(float(np.dot(s, S)) - flux) > 1e-6


@pytest.mark.parametrize("M", [1, 2, 3, 7])
@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_brute_force_tiny(M, lam):
    """Vectorised direct route and low-rank FFT route vs explicit loops, with a
    non-symmetric rank-2 kernel."""
    U, V = random_factors(M, 2, seed=11)
    K = U @ V
    n = random_state(M, seed=5, decay=2.0)
    ref = brute_force_rhs(n, lambda i, j: K[i - 1, j - 1], lam)
    d = oracle.rhs_terms_direct(n, K, lam)["total"]
    f = oracle.rhs_terms_lowrank(n, U, V, lam)["total"]
    scale = np.max(np.abs(ref)) + 1e-300
    assert np.max(np.abs(d - ref)) <= 1e-14 * scale
    assert np.max(np.abs(f - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("M,R", [(64, 1), (257, 3), (1024, 2), (4096, 4)])
def test_direct_vs_lowrank_random_factors(M, R):
    """Sec. 1 / Sec. 2: the O(M R log M) route equals the O(M^2) definition; factors
    are non-symmetric, so swapping U and V changes the death and source terms."""
    U, V = random_factors(M, R, seed=M + R)
    n = random_state(M, seed=M)
    d = oracle.rhs_terms_direct(n, U @ V, 0.05)
    f = oracle.rhs_terms_lowrank(n, U, V, 0.05)
    for key in ("birth", "death", "shatter_loss", "monomer_source"):
        ref = d[key]
        nrm = np.linalg.norm(ref) + 1e-300
        assert np.linalg.norm(f[key] - ref) <= 1e-12 * nrm, key
    swapped = oracle.rhs_terms_lowrank(n, V.T.copy(), U.T.copy(), 0.05)
    assert np.linalg.norm(swapped["death"] - d["death"]) > 1e-6 * np.linalg.norm(d["death"])


def test_kernel_factors_reproduce_closed_forms():
    M = 300
    for kind, a in (("const", 0.0), ("brownian", 0.3), ("brownian", 0.9), ("brownian_const", 1 / 3)):
        U, V = kernel_factors(kind, M, a=a)
        K = oracle.kernel_closed_form(kind, M, a=a)
        assert np.max(np.abs(U @ V - K) / K) <= 1e-14


def test_entries_direct_matches_full_direct():
    M, lam = 200, 0.01
    n = sample_state(M, lam)
    K = oracle.kernel_closed_form("brownian", M, a=0.9)
    full = oracle.rhs_terms_direct(n, K, lam)["total"]
    sizes = [2, 3, 50, 199, 200]
    got = oracle.rhs_entries_direct(n, lambda i, j: (i / j) ** 0.9 + (j / i) ** 0.9, lam, sizes)
    ref = full[np.array(sizes) - 1]
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12


# ---------------------------------------------------------------------------
# Runge-Kutta tableaux
# ---------------------------------------------------------------------------
def _poly(coefs, z):
    return sum(float(Fraction(num, den)) * z ** k for k, (num, den) in enumerate(coefs))


@pytest.mark.parametrize("z", [-0.3, 0.7, -1.9, 1.3 - 0.4j, -2.2 + 1.1j])
def test_stability_polynomials(z):
    g = json.load(open(os.path.join(GOLDEN, "rk_stability.json")))["polys"]
    S = lambda y: z * y  # noqa: E731
    y0 = np.array([1.0 + 0j])
    assert abs(oracle.rk2_step(S, y0, 1.0)[0] - _poly(g["rk2"], z)) <= 1e-14
    assert abs(oracle.rk4_step(S, y0, 1.0)[0] - _poly(g["rk4"], z)) <= 1e-14
    n4, n5 = oracle.rkf45_step(S, y0, 1.0)
    assert abs(n4[0] - _poly(g["rkf45_n4"], z)) <= 1e-13
    assert abs(n5[0] - _poly(g["rkf45_n5"], z)) <= 1e-13


def test_observed_orders():
    """y' = -y^2 + cos t style smooth scalar ODE; errors at t=1 shrink as tau^p."""
    def S(y, t=[0.0]):
        return -y * y
    y0 = np.array([1.0])
    exact = 1.0 / (1.0 + 1.0)  # y = 1/(1+t) at t = 1
    def run(step, N, pick=0):
        y = y0.copy()
        for _ in range(N):
            r = step(S, y, 1.0 / N)
            y = r[pick] if isinstance(r, tuple) else r
        return abs(y[0] - exact)
    for step, p, pick in ((oracle.rk2_step, 2, 0), (oracle.rk4_step, 4, 0), (oracle.rkf45_step, 4, 0),
                          (oracle.rkf45_step, 5, 1)):
        e1, e2 = run(step, 8, pick), run(step, 16, pick)
        rate = math.log2(e1 / e2)
        assert rate > p - 0.35, (step.__name__, p, rate)
        if pick == 0:                     # the propagated solutions have exactly order p
            assert rate < p + 0.35, (step.__name__, p, rate)


@pytest.mark.parametrize("scheme", ["rk2", "rk4", "rkf45"])
def test_linear_invariant_mass_plus_flux(scheme):
    """Explicit RK preserves linear invariants: augmenting Eq. (4) with F' = -flux(n),
    sum_s s n_s + F is the same before and after a step, to rounding."""
    M, lam = 48, 0.05
    K = oracle.kernel_closed_form("brownian", M, a=0.6)
    s = np.arange(1, M + 1, dtype=np.float64)

    def S_aug(v):
        n = v[:M]
        return np.concatenate([oracle.rhs_terms_direct(n, K, lam)["total"], [-oracle.mass_flux_direct(n, K)]])

    n = sample_state(M, lam)
    v = np.concatenate([n, [0.0]])
    step = {"rk2": oracle.rk2_step, "rk4": oracle.rk4_step, "rkf45": oracle.rkf45_step}[scheme]
    r = step(S_aug, v, 0.7)
    w = r[0] if isinstance(r, tuple) else r
    inv0 = float(np.dot(s, v[:M]) + v[M])
    inv1 = float(np.dot(s, w[:M]) + w[M])
    assert abs(inv1 - inv0) <= 1e-14 * abs(inv0)
    assert abs(float(np.dot(s, w[:M])) - float(np.dot(s, v[:M]))) > 1e-8  # flux actually acts


# ---------------------------------------------------------------------------
# Step-size controllers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("route", ["direct", "lowrank"])
def test_euler_initial_step_closed_forms(route):
    """Sec. 1's criterion tau0 = a / max_i sum_j K_ij n_j on a monodisperse state
    (n_1 = 1): the rate is K_i1, so tau0 = a for K = 1 and a / (M^a' + M^-a') for the
    Brownian kernel (i/j)^a' + (j/i)^a', whose K_i1 = i^a' + i^-a' grows with i."""
    M = 200
    n = monodisperse(M)
    U, V = kernel_factors("const", M)
    sysm = oracle.System(M, 0.0, U=U, V=V, route=route)
    assert oracle.euler_tau0(sysm, n, 0.1) == pytest.approx(0.1, rel=1e-15)
    for a in (0.3, 0.9):
        U, V = kernel_factors("brownian", M, a=a)
        sysm = oracle.System(M, 0.01, U=U, V=V, route=route)
        assert oracle.euler_tau0(sysm, n, 0.1) == pytest.approx(0.1 / (M ** a + M ** -a), rel=1e-13)
    # a spread state: the rate of K = 1 is the number density N = sum_j n_j at every i
    n2 = sample_state(M, 0.01)
    U, V = kernel_factors("const", M)
    sysm = oracle.System(M, 0.0, U=U, V=V, route=route)
    assert oracle.euler_tau0(sysm, n2, 0.2) == pytest.approx(0.2 / float(np.sum(n2)), rel=1e-13)


def test_rkf45_controller_worked_examples():
    g = json.load(open(os.path.join(GOLDEN, "rkf45_controller.json")))
    tol, tau = 1e-8, 0.37
    for case in g["cases"]:
        acc, tau_new = oracle.ctrl_rkf45(tau, case["err_over_tol"] * tol, tol)
        assert acc == case["accept"]
        assert abs(tau_new / tau - case["factor"]) <= case["abs_tol"]


def test_double_halve_and_formula_controllers():
    assert oracle.ctrl_double_halve(0.2, 2e-8, 1e-8) == (False, 0.1)
    assert oracle.ctrl_double_halve(0.2, 1e-8, 1e-8) == (True, 0.4)
    acc, tn = oracle.ctrl_formula(1.0, 1e-8 / 16.0, 1e-8, p=4)
    assert acc and abs(tn - 0.25 * 2.0) < 1e-15        # s (tol/err)^(1/p) = 1/4 * 16^(1/4)
    acc, tn = oracle.ctrl_formula(1.0, 4e-8, 1e-8, p=2)
    assert (not acc) and abs(tn - 0.125) < 1e-15         # 1/4 * (1/4)^(1/2)


def _stability(scheme, z):
    """R(z) of a scheme on y' = lambda y, z = tau lambda, from tests/golden/rk_stability.json."""
    g = json.load(open(os.path.join(GOLDEN, "rk_stability.json")))["polys"]
    return _poly(g[scheme], z)


def test_rkf45_loop_on_linear_equation():
    """The RKF45 integrator on y' = -y against a replay built from the embedded pair's
    stability polynomials: the error is |R5(-tau) - R4(-tau)| |y|, the fourth-order value
    is propagated, tau <- 0.9 tau (tol/err)^(1/5) clamped to [0.1, 4] on every attempt,
    and the last step is shortened to t1."""
    tol, t1, tau0 = 1e-9, 4.0, 1.5
    y, st, log = oracle.integrate(lambda n: -n, np.array([1.0]), 0.0, t1, tol,
                                  oracle.Options(scheme="rkf45", tau0=tau0, log=True))
    assert st["status"] == oracle.OK
    t, yy, tau, rows = 0.0, 1.0, tau0, []
    while t < t1:
        clamped = tau >= t1 - t
        h = t1 - t if clamped else tau
        n4 = _stability("rkf45_n4", -h) * yy
        err = abs(_stability("rkf45_n5", -h) * yy - n4)
        acc = err <= tol
        new = h * min(max(0.9 * (tol / err) ** 0.2, 0.1), 4.0)
        rows.append((t, h, err, acc))
        if acc:
            yy, t = n4, (t1 if clamped else t + h)
            if not clamped:
                tau = new
        else:
            tau = new
    assert [r[3] for r in log] == [r[3] for r in rows] and st["rejected"] >= 1
    np.testing.assert_allclose([r[1] for r in log], [r[1] for r in rows], rtol=1e-5, atol=0)
    np.testing.assert_allclose([r[2] for r in log], [r[2] for r in rows], rtol=1e-5, atol=1e-18)
    assert abs(y[0] - yy) <= 1e-12


@pytest.mark.parametrize("scheme", ["rk2", "rk4"])
@pytest.mark.parametrize("ctrl", ["double_halve", "formula"])
def test_step_doubling_loop_on_linear_equation(scheme, ctrl):
    """The step-doubling integrator on y' = -y against a replay built from the schemes'
    stability polynomials alone: a full step multiplies y by R(-tau), two half steps by
    R(-tau/2)^2, the error is their difference, the half steps are propagated, and the
    step follows the rule of Sec. 2 (halve / double, or Eq. (6) with s = 1/4 and the
    factor clamped to [0.1, 4])."""
    p = 2 if scheme == "rk2" else 4
    tol, t1, tau0 = 1e-7, 3.0, 0.3
    y, st, log = oracle.integrate(lambda n: -n, np.array([1.0]), 0.0, t1, tol,
                                  oracle.Options(scheme=scheme, ctrl=ctrl, tau0=tau0, log=True))
    assert st["status"] == oracle.OK
    t, yy, tau, rows = 0.0, 1.0, tau0, []
    while t < t1:
        clamped = tau >= t1 - t
        h = t1 - t if clamped else tau
        full = _stability(scheme, -h) * yy
        half = _stability(scheme, -h / 2) ** 2 * yy
        err = abs(half - full)
        acc = err <= tol
        if ctrl == "double_halve":
            new = 2 * h if acc else h / 2
        else:
            new = h * min(max(0.25 * (tol / err) ** (1.0 / p), 0.1), 4.0)
        rows.append((t, h, err, acc))
        if acc:
            yy, t = half, (t1 if clamped else t + h)
            if not clamped:
                tau = new
        else:
            tau = new
    assert [r[3] for r in log] == [r[3] for r in rows]
    # err is a difference of two O(y) values (relative rounding ~1e-9 at err ~ tol);
    # Eq. (6) carries it into every later step, multiplicatively
    rt = 1e-12 if ctrl == "double_halve" else 1e-5
    np.testing.assert_allclose([r[1] for r in log], [r[1] for r in rows], rtol=rt, atol=0)
    np.testing.assert_allclose([r[2] for r in log], [r[2] for r in rows], rtol=1e-5, atol=1e-18)
    assert abs(y[0] - yy) <= 1e-12 and st["rejected"] >= 1


# ---------------------------------------------------------------------------
# Whole trajectories
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scheme,tol", [("rk2", 1e-9), ("rk4", 1e-10), ("rkf45", 1e-10)])
def test_integrate_constant_kernel_closed_form(scheme, tol):
    """K = 1, lambda = 0, monodisperse start: the adaptive integrator tracks the exact
    solution; M = 128 keeps the truncation below 1e-19 up to t = 3."""
    M, t1 = 128, 3.0
    U, V = kernel_factors("const", M)
    sysm = oracle.System(M, 0.0, U=U, V=V, route="lowrank")
    n, st, _ = oracle.integrate(sysm, monodisperse(M), 0.0, t1, tol, oracle.Options(scheme=scheme))
    assert st["status"] == oracle.OK and st["t"] == t1
    ref = closed_form(M, t1)
    err = np.linalg.norm(n - ref)
    assert err <= 200 * tol * max(1.0, st["accepted"]) ** 0.5, (err, st)
    assert st["rhs_evals_paper"] % oracle.STAGES[scheme] == 0


def test_integrate_stats_conventions():
    M = 64
    U, V = kernel_factors("brownian", M, a=0.3)
    sysm = oracle.System(M, 0.01, U=U, V=V, route="direct")
    n, st, log = oracle.integrate(sysm, monodisperse(M), 0.0, 2.0, 1e-8,
                                  oracle.Options(scheme="rkf45", log=True))
    assert st["status"] == oracle.OK and st["t"] == 2.0
    assert st["accepted"] + st["rejected"] == len(log)
    assert st["rhs_evals_paper"] == 6 * len(log)
    # an attempt after a rejection starts from the same n and keeps its S(n)
    retries = sum(1 for prev in log[:-1] if not prev[3])
    assert st["rhs_evals"] == 6 * len(log) - retries
    # a fixed-step replay of the accepted steps reproduces the trajectory bit for bit
    taus = [h for (_, h, _, acc) in log if acc]
    m = monodisperse(M)
    for h in taus:
        m, _ = oracle.rkf45_step(sysm, m, h)
    assert np.array_equal(m, n)


@pytest.mark.parametrize("scheme,opts", [("rk2", {}), ("rk4", {}), ("rkf45", {}), ("rk4", {"fixed_tau": 0.05})])
def test_rhs_eval_counts_match_calls(scheme, opts):
    """rhs_evals counts the calls of S actually made (step doubling shares S(n^k));
    rhs_evals_paper counts stages x RK steps evaluated, the tables' convention."""
    M = 32
    U, V = kernel_factors("brownian", M, a=0.3)
    sysm = oracle.System(M, 0.01, U=U, V=V)
    _, st, log = oracle.integrate(sysm, monodisperse(M), 0.0, 1.0, 1e-8,
                                  oracle.Options(scheme=scheme, tau0=0.05, log=True, **opts))
    assert st["rhs_evals"] == sysm.evals
    per = oracle.STAGES[scheme] * (1 if (scheme == "rkf45" or opts) else 3)
    assert st["rhs_evals_paper"] == per * len(log)


@pytest.mark.parametrize("scheme", ["rk2", "rk4", "rkf45"])
def test_retry_keeps_first_stage(scheme):
    """A rejected attempt is repeated from the same n^k (Sec. 2), so the retry's first
    stage S(n^k) is not evaluated again: the actual count is the paper's count less one
    per retry, and equals the number of calls of S. A large initial step forces
    rejections."""
    M = 32
    U, V = kernel_factors("brownian", M, a=0.3)
    sysm = oracle.System(M, 0.01, U=U, V=V)
    _, st, log = oracle.integrate(sysm, monodisperse(M), 0.0, 1.0, 1e-8,
                                  oracle.Options(scheme=scheme, tau0=2.0, log=True))
    retries = sum(1 for prev in log[:-1] if not prev[3])
    assert st["rejected"] >= 2 and retries == st["rejected"]
    assert st["rhs_evals"] == sysm.evals
    p = oracle.STAGES[scheme]
    assert st["rhs_evals"] == len(log) * (p if scheme == "rkf45" else 3 * p - 1) - retries


def test_integrate_status_codes():
    M = 32
    U, V = kernel_factors("brownian", M, a=0.3)
    sysm = oracle.System(M, 0.01, U=U, V=V)
    n0 = monodisperse(M)
    _, st, _ = oracle.integrate(sysm, n0, 0.0, 10.0, 1e-300, oracle.Options(scheme="rkf45"))
    assert st["status"] == oracle.ESTEP_UNDERFLOW
    _, st, _ = oracle.integrate(sysm, n0, 0.0, 10.0, 1e-8, oracle.Options(scheme="rkf45", max_attempts=3))
    assert st["status"] == oracle.EMAXATTEMPTS and st["accepted"] + st["rejected"] == 3
    bad = n0.copy()
    bad[3] = np.nan
    _, st, _ = oracle.integrate(sysm, bad, 0.0, 10.0, 1e-8, oracle.Options(scheme="rk2", tau0=0.01))
    assert st["status"] == oracle.ENONFINITE


def test_steady_tail_constant_kernel_shattering():
    """Sec. 3.2: with K = 1 and shattering, the stationary distribution decays like
    k^{-3/2} exp(-lambda^2 k). With lambda = 1 and M = 64 the truncation flux is small,
    so the run must stop on the residual test ||S(n)||_2 / ||n||_2 < 1e-8 before t = 1e4
    with mass sum_s s n_s still within 1e-4 of 1."""
    M, lam = 64, 1.0
    U, V = kernel_factors("const", M)
    sysm = oracle.System(M, lam, U=U, V=V, route="lowrank")
    n, st, _ = oracle.integrate(sysm, monodisperse(M), 0.0, 1e4, 1e-9,
                                oracle.Options(scheme="rkf45", steady_rtol=1e-8))
    assert st["status"] == oracle.STEADY and st["t"] < 1e4
    S = sysm.rhs(n)
    assert np.linalg.norm(S) / np.linalg.norm(n) < 1e-8
    assert abs(oracle.total_mass(n) - 1.0) < 1e-4


# ---------------------------------------------------------------------------
# Aggregation with constant sources, Eq. (3) (Sec. 3.1: P_1 = 1, P_100 = p)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("route", ["direct", "lowrank"])
def test_sources_mass_identity(route):
    """Eq. (3): sum_s s S_s(n) = sum_s s P_s minus the truncation flux, exactly (for any
    n): injection adds sum_s s P_s of mass per unit time and coagulation conserves
    mass up to the pairs lost above M. Fails if a source enters at the wrong size
    (off by one) or with the wrong sign."""
    M = 150
    n = random_state(M, seed=11, decay=30.0)
    U, V = kernel_factors("brownian", M, a=0.3)
    K = oracle.kernel_closed_form("brownian", M, a=0.3)
    P = {1: 1.0, 100: 0.05}
    sysm = oracle.System(M, 0.0, K=K, U=U, V=V, route=route, sources=P)
    S = sysm.rhs(n)
    s = np.arange(1, M + 1, dtype=np.float64)
    inj = 1.0 * 1 + 0.05 * 100
    lhs = float(np.dot(s, S))
    rhs = inj + oracle.mass_flux_direct(n, K)
    assert abs(lhs - rhs) <= 1e-12 * (float(np.dot(s, np.abs(S))) + inj)
    d = sysm.rhs_terms(n)
    assert d["sources"][0] == 1.0 and d["sources"][99] == 0.05 and np.count_nonzero(d["sources"]) == 2


def test_sources_constant_kernel_total_density_closed_form():
    """K = 1, monomer source J, empty start: N = sum_s n_s obeys dN/dt = J - N^2 / 2 (the
    pairs above M are negligible here), so N(t) = sqrt(2J) tanh(t sqrt(J/2)); and the
    mass is J t. Pins Eq. (3)'s source and birth/death balance through an integration."""
    M, J = 64, 1.0
    sysm = oracle.System(M, 0.0, K=np.ones((M, M)), sources={1: J})
    n, st, _ = oracle.integrate(sysm, np.zeros(M), 0.0, 3.0, 1e-11, oracle.Options(scheme="rkf45", tau0=1e-3))
    assert st["status"] == 0
    N_exact = math.sqrt(2 * J) * math.tanh(3.0 * math.sqrt(J / 2))
    assert abs(oracle.number_density(n) - N_exact) <= 1e-8
    assert abs(oracle.total_mass(n) - 3.0 * J) <= 1e-7


def test_sources_rejects_size_outside_range():
    with pytest.raises(ValueError):
        oracle.System(10, 0.0, K=np.ones((10, 10)), sources={11: 1.0})
