"""Plain FP64 restatement of the paper's method. TEST INFRASTRUCTURE ONLY.

Notation follows the paper: sizes s = 1..M (stored 0-based, n[s-1] = n_s), kernel
K_{i,j}, shattering rate lambda, tolerance tol, step tau, RK stage vectors k_i.

Readings of the paper taken here (each is also listed with its reason in the design
notes of the repository):
  * Eq. (4), monomer equation: the term lambda * sum_{j>=2} j K_{1,j} n_j is read with
    the factor n_1 (lambda n_1 sum_{j>=2} j K_{1,j} n_j): every collision term is
    quadratic in n, and only with n_1 does shattering conserve mass.
  * Truncation (Eq. (2) and (4)): births above M are dropped, death sums run to M.
  * Step doubling for RK2/RK4 (Sec. 2): the two half steps are propagated; the error
    is ||n_hat - n||_2 (absolute by default; 'rel' divides by ||n^k||_2).
  * Controllers: 'double_halve' (halve on reject, double on accept) and 'formula'
    (Eq. (6), s = 1/4, accept iff err <= tol); RKF45: repeat while err > tol,
    tau <- 0.9 tau (tol/err)^(1/5) on every attempt. Step factors are clamped to
    [fac_min, fac_max] = [0.1, 4] (the paper gives no bounds; err = 0 needs one).
  * Initial step: the Euler criterion of Sec. 1 with a = 1/10,
    tau0 = a / max_i sum_j K_ij n_j(0), unless the caller gives tau0.
  * Last step is clamped to t1 - t; an accepted clamped step keeps the proposed tau.

No parity pin exists for the RK2/RK4 controllers beyond their stated formulas (the
paper prints no worked example for them): parity unpinned for those two rules.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "kernel_closed_form", "kernel_from_factors", "System",
    "rhs_terms_direct", "rhs_terms_lowrank", "rhs_entries_direct", "mass_flux_direct",
    "total_mass", "number_density",
    "rk2_step", "rk4_step", "rkf45_step", "STAGES",
    "ctrl_rkf45", "ctrl_formula", "ctrl_double_halve",
    "Options", "integrate", "euler_tau0",
    "OK", "STEADY", "EINVAL", "ENONFINITE", "ESTEP_UNDERFLOW", "EMAXATTEMPTS",
]

# Status codes shared in meaning (not in code) with the C interface.
OK, STEADY = 0, 1
EINVAL, ENONFINITE, ESTEP_UNDERFLOW, EMAXATTEMPTS = -1, -3, -4, -5


# ---------------------------------------------------------------------------
# Kernels K_{i,j} (Sec. 1 example; Sec. 3.1 list; Sec. 3.2 non-local kernel)
# ---------------------------------------------------------------------------
def kernel_closed_form(kind: str, M: int, a: float = 0.0, c: float = 2.0) -> np.ndarray:
    """K_{i,j} for i, j = 1..M evaluated from its closed form (the kernels listed in
    Sec. 3.1: constant, generalized Brownian (+ c), free-molecular)."""
    i = np.arange(1, M + 1, dtype=np.float64)[:, None]
    j = np.arange(1, M + 1, dtype=np.float64)[None, :]
    if kind == "const":
        return np.ones((M, M))
    if kind == "brownian":
        return (i / j) ** a + (j / i) ** a
    if kind == "brownian_const":
        return (i / j) ** a + (j / i) ** a + c
    if kind == "free_molecular":
        # Sec. 3.1: (i^{1/3} + j^{1/3})^2 sqrt(1/i + 1/j); no exact low rank
        return (np.cbrt(i) + np.cbrt(j)) ** 2 * np.sqrt(1.0 / i + 1.0 / j)
    raise ValueError(kind)


def kernel_from_factors(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """K = U V, i.e. K_{i,j} = sum_alpha U_{i,alpha} V_{alpha,j} (Sec. 1)."""
    return U @ V


# ---------------------------------------------------------------------------
# Right-hand side of Eq. (4), by the direct sums that define it (O(M^2))
# ---------------------------------------------------------------------------
def rhs_terms_direct(n: np.ndarray, K: np.ndarray, lam: float, _cache: dict | None = None) -> dict:
    """Terms of Eq. (4) for state n and dense kernel matrix K (K[i-1, j-1] = K_{i,j}).

    Returns birth, death (n_s sum_i K_{s,i} n_i for every s), shatter_loss
    (lambda n_s sum_i K_{s,i} n_i for s >= 2), monomer_source (new monomers from
    shattering; nonzero only at s = 1) and total = birth - death - shatter_loss +
    monomer_source.
    """
    n = np.asarray(n, dtype=np.float64)
    M = n.size
    if _cache is not None and _cache.get("M") == M:
        antidiag, ipj = _cache["antidiag"], _cache["ipj"]
    else:
        idx = np.arange(M)
        antidiag = np.add.outer(idx, idx).ravel()          # (i-1)+(j-1) = i+j-2
        ipj = np.add.outer(idx + 1.0, idx + 1.0)            # i + j
        if _cache is not None:
            _cache.update(M=M, antidiag=antidiag, ipj=ipj)
    A = K * np.outer(n, n)                                   # K_ij n_i n_j
    # birth_s = 1/2 sum_{i+j=s} K_ij n_i n_j, s = 2..M  (0-based anti-diagonal s-2)
    diag = np.bincount(antidiag, weights=A.ravel(), minlength=2 * M - 1)
    birth = np.zeros(M)
    birth[1:] = 0.5 * diag[: M - 1]
    # death_s = n_s sum_{i=1}^{M} K_{s,i} n_i
    death = n * (K @ n)
    # shattering into monomers, s = 2..M: lambda n_s sum_i K_{s,i} n_i
    shatter_loss = np.zeros(M)
    shatter_loss[1:] = lam * death[1:]
    # new monomers: lambda/2 sum_{i>=2} sum_{j>=2} (i+j) K_ij n_i n_j
    #             + lambda n_1 sum_{j>=2} j K_{1,j} n_j
    s = np.arange(1, M + 1, dtype=np.float64)
    src = 0.5 * lam * np.sum(ipj[1:, 1:] * A[1:, 1:])
    src += lam * n[0] * np.sum(s[1:] * K[0, 1:] * n[1:])
    monomer_source = np.zeros(M)
    monomer_source[0] = src
    total = birth - death - shatter_loss + monomer_source
    return dict(birth=birth, death=death, shatter_loss=shatter_loss,
                monomer_source=monomer_source, total=total)


def mass_flux_direct(n: np.ndarray, K: np.ndarray) -> float:
    """Rate of mass lost by truncation: -1/2 sum_{i,j<=M, i+j>M} (i+j) K_ij n_i n_j.

    Shattering moves mass into monomers without loss, so for Eq. (4) the exact identity
    sum_s s S_s(n) = mass_flux_direct(n, K) holds."""
    M = n.size
    s = np.arange(1, M + 1, dtype=np.float64)
    ipj = np.add.outer(s, s)
    A = K * np.outer(n, n)
    return -0.5 * float(np.sum(np.where(ipj > M, ipj * A, 0.0)))


def total_mass(n: np.ndarray) -> float:
    """sum_s s n_s."""
    return float(np.dot(np.arange(1, n.size + 1, dtype=np.float64), n))


def number_density(n: np.ndarray) -> float:
    """N = sum_s n_s (the total density whose oscillations Fig. 3 shows)."""
    return float(np.sum(n))


# ---------------------------------------------------------------------------
# Right-hand side by the low-rank route (Sec. 1, Sec. 2): O(M R log M)
# ---------------------------------------------------------------------------
def rhs_terms_lowrank(n: np.ndarray, U: np.ndarray, V: np.ndarray, lam: float) -> dict:
    """Same terms as rhs_terms_direct, with K = U V substituted.

    birth: 1/2 sum_alpha (U_alpha n) * (V_alpha n), a linear convolution evaluated with
    zero-padded real FFTs (numpy's FFT is the library step); death and shattering
    from the rank-R sums m_alpha = sum_j V_{alpha,j} n_j and the four moments
      P_alpha  = sum_{i>=2} i U_{i,alpha} n_i,   P'_alpha = sum_{i>=2} U_{i,alpha} n_i,
      Q_alpha  = sum_{j>=2} V_{alpha,j} n_j,     Q'_alpha = sum_{j>=2} j V_{alpha,j} n_j,
    since sum_{i,j>=2} (i+j) K_ij n_i n_j = sum_alpha (P_alpha Q_alpha + P'_alpha Q'_alpha).
    """
    n = np.asarray(n, dtype=np.float64)
    M = n.size
    R = U.shape[1]
    L = 2 * M
    c = np.zeros(L)
    for a in range(R):
        fa = np.fft.rfft(U[:, a] * n, L)
        fb = np.fft.rfft(V[a, :] * n, L)
        c += np.fft.irfft(fa * fb, L)
    birth = np.zeros(M)
    birth[1:] = 0.5 * c[: M - 1]
    m = V @ n
    D = U @ m
    death = n * D
    shatter_loss = np.zeros(M)
    shatter_loss[1:] = lam * death[1:]
    s = np.arange(1, M + 1, dtype=np.float64)
    P = (s[1:] * n[1:]) @ U[1:, :]
    Pp = n[1:] @ U[1:, :]
    Q = V[:, 1:] @ n[1:]
    Qp = V[:, 1:] @ (s[1:] * n[1:])
    src = 0.5 * lam * float(np.sum(P * Q + Pp * Qp)) + lam * n[0] * float(np.dot(U[0, :], Qp))
    monomer_source = np.zeros(M)
    monomer_source[0] = src
    total = birth - death - shatter_loss + monomer_source
    return dict(birth=birth, death=death, shatter_loss=shatter_loss,
                monomer_source=monomer_source, total=total)


def rhs_entries_direct(n: np.ndarray, kfun, lam: float, sizes) -> np.ndarray:
    """S_s(n) for the listed sizes s >= 2 one by one, by the direct sums of Eq. (4).

    kfun(i, j) evaluates K_{i,j} elementwise on 1-based integer arrays. Cost O(M) per
    entry, so it serves full-size problems on sampled outputs."""
    n = np.asarray(n, dtype=np.float64)
    M = n.size
    out = np.empty(len(sizes))
    jall = np.arange(1, M + 1)
    for t, s in enumerate(sizes):
        if s < 2 or s > M:
            raise ValueError("rhs_entries_direct takes sizes 2..M")
        i = np.arange(1, s)
        birth = 0.5 * np.sum(kfun(i, s - i) * n[i - 1] * n[s - i - 1])
        rate = np.sum(kfun(np.full(M, s), jall) * n)
        out[t] = birth - (1.0 + lam) * n[s - 1] * rate
    return out


class System:
    """The ODE system dn/dt = S(n) of Eq. (5) for Eq. (4) with a given kernel.

    route='direct' uses a dense K (O(M^2), the definition); route='lowrank' uses the
    factors U, V and the FFT route. sources: {s: P_s} (1-based sizes), the constant
    injection terms P_k of Eq. (3); with lam = 0 the system is Eq. (3) (Sec. 3.1 uses
    P_1 = 1, P_100 = p). They are added to the total and reported as the term
    'sources'."""

    def __init__(self, M, lam, K=None, U=None, V=None, route="direct", sources=None):
        self.M, self.lam, self.route = int(M), float(lam), route
        self.K, self.U, self.V = K, U, V
        self.P = np.zeros(self.M)
        for k, v in (sources or {}).items():
            if not 1 <= int(k) <= self.M:
                raise ValueError("source size outside 1..M")
            self.P[int(k) - 1] += float(v)
        if route == "direct" and K is None:
            self.K = kernel_from_factors(U, V)
        if route == "lowrank" and (U is None or V is None):
            raise ValueError("lowrank route needs U and V")
        self._cache: dict = {}
        self.evals = 0

    def rhs_terms(self, n):
        self.evals += 1
        if self.route == "direct":
            d = rhs_terms_direct(n, self.K, self.lam, self._cache)
        else:
            d = rhs_terms_lowrank(n, self.U, self.V, self.lam)
        d["sources"] = self.P.copy()
        d["total"] = d["total"] + self.P
        return d

    def rhs(self, n):
        return self.rhs_terms(n)["total"]

    __call__ = rhs

    def collision_rate(self, n):
        """sum_j K_{i,j} n_j for every i (the quantity of the Euler criterion)."""
        if self.K is not None and self.route == "direct":
            return self.K @ n
        return self.U @ (self.V @ n)


def euler_tau0(system: System, n: np.ndarray, a: float = 0.1) -> float:
    """Euler stability criterion of Sec. 1: tau <= a [max_i sum_j K_ij n_j]^{-1}."""
    rate = float(np.max(system.collision_rate(n)))
    return a / rate if rate > 0 else 1.0


# ---------------------------------------------------------------------------
# Explicit RK schemes of Sec. 2 (k_i = tau S(.))
# ---------------------------------------------------------------------------
def rk2_step(S, n, tau, S_n=None):
    """Second-order RK of Sec. 2: k1 = tau S(n), k2 = tau S(n + k1), n + (k1+k2)/2."""
    k1 = tau * (S(n) if S_n is None else S_n)
    k2 = tau * S(n + k1)
    return n + (k1 + k2) / 2.0


def rk4_step(S, n, tau, S_n=None):
    """Classical fourth-order RK of Sec. 2."""
    k1 = tau * (S(n) if S_n is None else S_n)
    k2 = tau * S(n + 0.5 * k1)
    k3 = tau * S(n + 0.5 * k2)
    k4 = tau * S(n + k3)
    return n + (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0


def rkf45_step(S, n, tau, S_n=None):
    """Runge-Kutta-Fehlberg 4(5) of Sec. 2. Returns (n^{k+1}, n_RK5): the fourth-order
    solution that is propagated and the fifth-order one used only for the error."""
    k1 = tau * (S(n) if S_n is None else S_n)
    k2 = tau * S(n + k1 / 4.0)
    k3 = tau * S(n + (3.0 * k1 + 9.0 * k2) / 32.0)
    k4 = tau * S(n + (1932.0 * k1 - 7200.0 * k2 + 7296.0 * k3) / 2197.0)
    k5 = tau * S(n + 439.0 / 216.0 * k1 - 8.0 * k2 + 3680.0 / 513.0 * k3 - 845.0 / 4104.0 * k4)
    k6 = tau * S(n - 8.0 / 27.0 * k1 + 2.0 * k2 - 3544.0 / 2565.0 * k3 + 1859.0 / 4104.0 * k4
                 - 11.0 / 40.0 * k5)
    n5 = n + 16.0 / 135.0 * k1 + 6656.0 / 12825.0 * k3 + 28561.0 / 56430.0 * k4 - 9.0 / 50.0 * k5 \
        + 2.0 / 55.0 * k6
    n4 = n + 25.0 / 216.0 * k1 + 1408.0 / 2565.0 * k3 + 2197.0 / 4104.0 * k4 - 1.0 / 5.0 * k5
    return n4, n5


# RHS evaluations per RK step (stages); order p of each scheme.
STAGES = {"rk2": 2, "rk4": 4, "rkf45": 6}
ORDER = {"rk2": 2, "rk4": 4, "rkf45": 4}


# ---------------------------------------------------------------------------
# Step-size controllers (Sec. 2)
# ---------------------------------------------------------------------------
def _clamp(x, lo, hi):
    return lo if x < lo else (hi if x > hi else x)


def ctrl_rkf45(tau, err, tol, safety=0.9, fac_min=0.1, fac_max=4.0):
    """Fehlberg's rule: accept iff err <= tol; tau_new = 0.9 tau (tol/err)^(1/5)."""
    accept = err <= tol
    fac = fac_max if err == 0.0 else _clamp(safety * (tol / err) ** 0.2, fac_min, fac_max)
    return accept, tau * fac


def ctrl_formula(tau, err, tol, p, s=0.25, fac_min=0.1, fac_max=4.0):
    """Eq. (6): tau_new = s tau (tol / ||n_hat - n||_2)^(1/p), s = 1/4; accept iff err <= tol."""
    accept = err <= tol
    fac = fac_max if err == 0.0 else _clamp(s * (tol / err) ** (1.0 / p), fac_min, fac_max)
    return accept, tau * fac


def ctrl_double_halve(tau, err, tol):
    """Sec. 2: above tol the step is halved and the test repeated; below, the next
    step is taken with twice the step."""
    accept = err <= tol
    return accept, (2.0 * tau if accept else 0.5 * tau)


# ---------------------------------------------------------------------------
# Adaptive integration driver
# ---------------------------------------------------------------------------
@dataclass
class Options:
    scheme: str = "rkf45"          # 'rk2' | 'rk4' | 'rkf45'
    ctrl: str = "double_halve"     # RK2/RK4 only: 'double_halve' | 'formula'
    norm: str = "abs"              # 'abs' | 'rel'
    tau0: float = 0.0              # <= 0: Euler criterion with euler_a
    euler_a: float = 0.1
    tau_min_rel: float = 1e-12     # stop with ESTEP_UNDERFLOW below tau_min_rel*max(1,|t|)
    max_attempts: int = 10 ** 9
    steady_rtol: float = 0.0       # > 0: stop when ||S(n)||_2 / ||n||_2 < steady_rtol
    fixed_tau: float = 0.0         # > 0: constant steps, no error control
    fac_min: float = 0.1
    fac_max: float = 4.0
    log: bool = False


def _norm(v):
    return math.sqrt(float(np.dot(v, v)))


def integrate(S, n0, t0, t1, tol, opts: Options | None = None, tau0_system: System | None = None):
    """Integrate dn/dt = S(n) from t0 to t1 with the schemes and controllers of Sec. 2.

    Returns (n, stats, log): stats holds t, tau_next, err_last, rhs_evals (actual),
    rhs_evals_paper (stages x RK steps evaluated, the count the paper's tables use),
    accepted, rejected, status; log lists (t, tau, err, accepted) per attempt.
    """
    o = opts or Options()
    if o.scheme not in STAGES:
        raise ValueError(o.scheme)
    p = ORDER[o.scheme]
    n = np.array(n0, dtype=np.float64, copy=True)
    t = float(t0)
    if o.tau0 > 0:
        tau = float(o.tau0)
    elif o.fixed_tau > 0:
        tau = float(o.fixed_tau)
    else:
        tau = euler_tau0(tau0_system if tau0_system is not None else S, n, o.euler_a)
    st = dict(t=t, tau_next=tau, err_last=0.0, rhs_evals=0, rhs_evals_paper=0,
              accepted=0, rejected=0, status=OK)
    log = []
    attempts = 0
    S_n = None
    while t < t1:
        if attempts >= o.max_attempts:
            st["status"] = EMAXATTEMPTS
            break
        clamped = tau >= t1 - t
        h = (t1 - t) if clamped else tau
        # a rejected step is repeated from the same n (Sec. 2), whose S(n) is kept
        if S_n is None:
            S_n = S(n)
            st["rhs_evals"] += 1
        if o.steady_rtol > 0:
            nn = _norm(n)
            if nn > 0 and _norm(S_n) / nn < o.steady_rtol:
                st["status"] = STEADY
                break
        if o.scheme == "rkf45":
            n4, n5 = rkf45_step(S, n, h, S_n)
            st["rhs_evals"] += 5
            st["rhs_evals_paper"] += 6
            cand, err = n4, _norm(n5 - n4)
        elif o.fixed_tau > 0:
            cand = (rk2_step if o.scheme == "rk2" else rk4_step)(S, n, h, S_n)
            st["rhs_evals"] += STAGES[o.scheme] - 1
            st["rhs_evals_paper"] += STAGES[o.scheme]
            err = 0.0
        else:
            step = rk2_step if o.scheme == "rk2" else rk4_step
            full = step(S, n, h, S_n)
            half = step(S, n, 0.5 * h, S_n)
            half = step(S, half, 0.5 * h)
            # S(n^k) is shared by the full step and the first half step: 3p - 1 calls
            # in all, one of them already counted above
            st["rhs_evals"] += 3 * STAGES[o.scheme] - 2
            st["rhs_evals_paper"] += 3 * STAGES[o.scheme]
            cand, err = half, _norm(half - full)
        if o.norm == "rel":
            nn = _norm(n)
            err = err / nn if nn > 0 else err
        attempts += 1
        st["err_last"] = err
        if not math.isfinite(err) or not np.all(np.isfinite(cand)):
            st["status"] = ENONFINITE
            break
        if o.fixed_tau > 0:
            accept, tau_new = True, tau
        elif o.scheme == "rkf45":
            accept, tau_new = ctrl_rkf45(h, err, tol, fac_min=o.fac_min, fac_max=o.fac_max)
        elif o.ctrl == "formula":
            accept, tau_new = ctrl_formula(h, err, tol, p, fac_min=o.fac_min, fac_max=o.fac_max)
        else:
            accept, tau_new = ctrl_double_halve(h, err, tol)
        if o.log:
            log.append((t, h, err, accept))
        if accept:
            n = cand
            S_n = None
            t = t1 if clamped else t + h
            st["accepted"] += 1
            if not clamped:
                tau = tau_new
        else:
            st["rejected"] += 1
            tau = tau_new
        if t < t1 and tau < o.tau_min_rel * max(1.0, abs(t)):
            st["status"] = ESTEP_UNDERFLOW
            break
    st["t"] = t
    st["tau_next"] = tau
    st["attempts"] = attempts
    return n, st, log
