"""Seeded problem inputs: kernel factors, states and workload recipes.

Everything here is a problem *input* in the sense of the operator form dn/dt = S(n),
n(0) = n0 of the paper (Sec. 2, Eq. (5)): the low-rank factors U (M x R), V (R x M)
with K_ij = sum_a U_ia V_aj (Sec. 1), the shattering rate lambda and the initial or
sample state. Sizes are 1-based in the paper and 0-based here: n[s-1] = n_s.
"""
from __future__ import annotations

import numpy as np

# Physics kernels of the paper and their exact low-rank factors.
#   const           K_ij = 1                                  (Sec. 3.1, rank 1)
#   brownian        K_ij = (i/j)^a + (j/i)^a                  (Sec. 3.1 / 3.2, rank 2)
#   brownian_const  K_ij = (i/j)^a + (j/i)^a + c              (Sec. 1 example with a=1/3, c=2; rank 3)
KERNELS = ("const", "brownian", "brownian_const")


def kernel_factors(kind: str, M: int, a: float = 0.0, c: float = 2.0):
    """Return (U, V) float64 with U of shape (M, R) and V of shape (R, M)."""
    if M < 1:
        raise ValueError("M must be >= 1")
    s = np.arange(1, M + 1, dtype=np.float64)
    if kind == "const":
        U = np.ones((M, 1))
        V = np.ones((1, M))
    elif kind in ("brownian", "brownian_const"):
        up = s ** a
        um = s ** (-a)
        cols = [up, um]
        rows = [um, up]
        if kind == "brownian_const":
            cols.append(np.ones(M))
            rows.append(np.full(M, float(c)))
        U = np.stack(cols, axis=1)
        V = np.stack(rows, axis=0)
    else:
        raise ValueError(f"unknown kernel {kind!r}")
    return np.ascontiguousarray(U), np.ascontiguousarray(V)


def monodisperse(M: int) -> np.ndarray:
    """n_k(0) = delta_{k,1} (the initial condition of every experiment in Sec. 3)."""
    n = np.zeros(M)
    n[0] = 1.0
    return n


def sample_state(M: int, lam: float, seed: int = 20240723) -> np.ndarray:
    """A realistic mid-run state shaped like the stationary law of Sec. 3.2,
    n_k ~ k^{-3/2} exp(-lambda^2 k), with 10% seeded multiplicative noise,
    scaled so that the total mass sum_k k n_k equals 1."""
    rng = np.random.default_rng(seed)
    s = np.arange(1, M + 1, dtype=np.float64)
    n = s ** -1.5 * np.exp(-(lam ** 2) * s) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, M))
    return n / np.dot(s, n)


def random_state(M: int, seed: int, decay: float | None = None) -> np.ndarray:
    """Positive random state with an exponential envelope (spans several decades)."""
    rng = np.random.default_rng(seed)
    s = np.arange(1, M + 1, dtype=np.float64)
    if decay is None:
        decay = max(M / 8.0, 1.0)
    return np.exp(-s / decay) * rng.uniform(0.2, 1.0, M)


def random_factors(M: int, R: int, seed: int):
    """Positive, non-symmetric random low-rank factors (U: M x R, V: R x M) with
    power-law envelopes, for tests that must not rely on kernel symmetry."""
    rng = np.random.default_rng(seed)
    s = np.arange(1, M + 1, dtype=np.float64)
    U = np.empty((M, R))
    V = np.empty((R, M))
    for a in range(R):
        pu, pv = rng.uniform(-0.6, 0.6, 2)
        U[:, a] = s ** pu * rng.uniform(0.5, 1.5, M)
        V[a, :] = s ** pv * rng.uniform(0.5, 1.5, M)
    return U, V


def batch_recipe(count: int = 256, seed: int = 2407, m_lo: int = 10, m_hi: int = 16):
    """Independent systems of the batched workload: M = 2^round(U(m_lo, m_hi)),
    exponent a ~ U(0.2, 0.9) of the kernel (i/j)^a + (j/i)^a, lambda log-uniform in
    [0.005, 0.1], monodisperse start."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        M = int(2 ** int(round(rng.uniform(m_lo, m_hi))))
        a = float(rng.uniform(0.2, 0.9))
        lam = float(np.exp(rng.uniform(np.log(0.005), np.log(0.1))))
        out.append({"M": M, "a": a, "lam": lam})
    return out


# The five workloads, described by what they are.
WORKLOADS = {
    "shatter_M512_brownian0.3": dict(M=512, kernel="brownian", a=0.3, lam=0.01, t0=0.0, t1=200.0,
                                     tol=1e-8, scheme="rkf45", precision="fp64"),
    "relax_M65536_brownian_const": dict(M=65536, kernel="brownian_const", a=1.0 / 3.0, c=2.0, lam=0.1,
                                        t0=0.0, t1=1e4, tol=1e-9, steady_rtol=1e-10, precision="fp64"),
    "oscill_M131072_brownian0.9": dict(M=131072, kernel="brownian", a=0.9, lam=0.005, t0=0.0, t1=5000.0,
                                       tol=1e-8, scheme="rkf45", precision="fp64"),
    "relax_M65536_brownian_const_fp32conv": dict(M=65536, kernel="brownian_const", a=1.0 / 3.0, c=2.0,
                                                 lam=0.1, t0=0.0, t1=1e4, tol=1e-9, precision="fp32conv"),
    "batch256_brownian": dict(count=256, seed=2407, t0=0.0, t1=1000.0, tol=1e-8, precision="fp32conv"),
}
