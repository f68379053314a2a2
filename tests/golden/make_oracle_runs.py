"""Writes the oracle trajectories that the GPU parity tests and the benchmark's
time-to-solution legs compare against (tests/golden/oracle_<name>.npz).

Calls only the FP64 oracle (oracle/) and the seeded input generators (synth/); nothing
here comes from the CUDA path. Each run integrates Eq. (4) with the paper's schemes
(Sec. 2) from the monodisperse start and stops at every checkpoint of its list (the last
step before a checkpoint is clamped to it, and the next segment starts with the proposed
step tau_next, exactly as a caller resuming with smol_set_tau0 does). Per checkpoint it
stores the mass sum_s s n_s, N = sum_s n_s, ||S(n)||_2 and the cumulative attempt
counts, and (at every checkpoint, or every head_every-th one) the first `head` entries
of n(t) with the 2-norm of the remaining entries.

Usage: python tests/golden/make_oracle_runs.py [name ...]   (default: every run; each
run is its own process, started with the spawn method).

The runs (workloads of Sec. 3 of the paper, synthetic by definition: (M, K, lambda, n0)
specify them completely):
  relax_rkf45_tol1e-9, relax_rkf45_tol1e-6: M = 2^16, K = (i/j)^{1/3} + (j/i)^{1/3} + 2
      (rank 3), lambda = 0.1, RKF45, 20 checkpoints log-spaced over [0.1, 100].
  relax_rkf45_steady: the same at tol 1e-9 through 26 checkpoints log-spaced over
      [0.1, 10^4], stopping where ||S(n)||_2 / ||n||_2 < 1e-10 (the steady state).
  relax_rk2_tol1e-9, relax_rk4_tol1e-9: the same system with step doubling (the
      halve/double rule), checkpoints log-spaced over [0.01, 1].
  fig2_const: K = 1, lambda = 0.01, M = 32768, RKF45 tol 1e-8 to t = 10^4 (Fig. 2).
  fig3_a095_M2048: K = (i/j)^0.95 + (j/i)^0.95, lambda = 0.01, M = 2048, RKF45 tol 1e-8,
      N(t) at every unit of t up to 130 (the oscillations of Fig. 3), states every 10.
  oscill_a09_M2048: the oscillatory workload's kernel and rate (a = 0.9,
      lambda = 0.005) at M = 2048 to t = 200, N(t) at every unit of t, states every 10.
  oscill_a09_M131072_window: the oscillatory workload at full size, M = 2^17, over its
      first 0.2 time units (every 0.01).
  batch_small: the systems of the 256-system batch recipe (seed 2407) with M = 1024, each
      to t = 2 (RKF45 tol 1e-8); full states.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _relax(M=1 << 16):
    return dict(M=M, kind="brownian_const", a=1.0 / 3.0, lam=0.1)


RUNS = {
    "relax_rkf45_tol1e-9": dict(sys=_relax(), scheme="rkf45", tol=1e-9, ts=np.logspace(-1, 2, 20).tolist(),
                                head=2048),
    "relax_rkf45_tol1e-6": dict(sys=_relax(), scheme="rkf45", tol=1e-6, ts=np.logspace(-1, 2, 20).tolist(),
                                head=2048),
    "relax_rkf45_steady": dict(sys=_relax(), scheme="rkf45", tol=1e-9, ts=np.logspace(-1, 4, 26).tolist(),
                               head=2048, steady_rtol=1e-10),
    "relax_rk2_tol1e-9": dict(sys=_relax(), scheme="rk2", tol=1e-9, ts=np.logspace(-2, 0, 8).tolist(), head=2048),
    "relax_rk4_tol1e-9": dict(sys=_relax(), scheme="rk4", tol=1e-9, ts=np.logspace(-2, 0, 8).tolist(), head=2048),
    "fig2_const": dict(sys=dict(M=32768, kind="const", a=0.0, lam=0.01), scheme="rkf45", tol=1e-8,
                       ts=[1.0, 10.0, 100.0, 1000.0, 5000.0, 10000.0], head=4096),
    "fig3_a095_M2048": dict(sys=dict(M=2048, kind="brownian", a=0.95, lam=0.01), scheme="rkf45", tol=1e-8,
                            ts=np.arange(1.0, 131.0, 1.0).tolist(), head=2048, head_every=10),
    "oscill_a09_M2048": dict(sys=dict(M=2048, kind="brownian", a=0.9, lam=0.005), scheme="rkf45", tol=1e-8,
                             ts=np.arange(1.0, 201.0, 1.0).tolist(), head=2048, head_every=10),
    "oscill_a09_M131072_window": dict(sys=dict(M=1 << 17, kind="brownian", a=0.9, lam=0.005), scheme="rkf45",
                                      tol=1e-8, ts=np.round(np.arange(0.01, 0.2001, 0.01), 10).tolist(), head=4096),
    "batch_small": dict(batch=dict(count=256, seed=2407, M=1024), scheme="rkf45", tol=1e-8, ts=[0.5, 1.0, 2.0],
                        head=1024),
}


def _system(spec):
    import oracle
    from synth import kernel_factors
    U, V = kernel_factors(spec["kind"], spec["M"], a=spec["a"])
    return oracle.System(spec["M"], spec["lam"], U=U, V=V, route="lowrank")


def _trajectory(osys, M, scheme, tol, ts, head, steady_rtol=0.0, verbose=False, head_every=1):
    """Integrates from the monodisperse start through the checkpoints ts; the leading
    entries are kept at every head_every-th checkpoint (indices in head_idx)."""
    import oracle
    from synth import monodisperse
    n = monodisperse(M)
    t, tau = 0.0, 0.0
    cum = dict(attempts=0, accepted=0, rejected=0, rhs_evals=0)
    rec = dict(t=[], head=[], head_idx=[], tail_norm=[], mass=[], N=[], snorm=[], attempts=[], accepted=[],
               rejected=[], rhs_evals=[], status=[], tau_next=[])
    for kc, tc in enumerate(ts):
        o = oracle.Options(scheme=scheme, tau0=tau, steady_rtol=steady_rtol)
        n, st, _ = oracle.integrate(osys, n, t, tc, tol, o)
        for k in cum:
            cum[k] += st[k]
        t, tau = st["t"], st["tau_next"]
        S = osys.rhs(n)
        rec["t"].append(t)
        if kc % head_every == 0 or kc == len(ts) - 1:
            rec["head"].append(n[:head].copy())
            rec["head_idx"].append(kc)
            rec["tail_norm"].append(float(np.linalg.norm(n[head:])))
        rec["mass"].append(oracle.total_mass(n))
        rec["N"].append(oracle.number_density(n))
        rec["snorm"].append(float(np.linalg.norm(S)))
        for k in cum:
            rec[k].append(cum[k])
        rec["status"].append(st["status"])
        rec["tau_next"].append(tau)
        if verbose:
            print(f"  t={t:.6g} attempts={cum['attempts']} status={st['status']}", flush=True)
        if st["status"] != oracle.OK:
            break
    return {k: np.asarray(v) for k, v in rec.items()}


def run(name):
    spec = RUNS[name]
    t0 = time.time()
    if "batch" in spec:
        from synth import batch_recipe
        b = spec["batch"]
        rec = batch_recipe(b["count"], seed=b["seed"])
        idx = [q for q, r in enumerate(rec) if r["M"] == b["M"]]
        out = {"systems": np.asarray(idx)}
        for q in idx:
            r = rec[q]
            osys = _system(dict(M=r["M"], kind="brownian", a=r["a"], lam=r["lam"]))
            tr = _trajectory(osys, r["M"], spec["scheme"], spec["tol"], spec["ts"], spec["head"])
            for k, v in tr.items():
                out[f"s{q}_{k}"] = v
    else:
        osys = _system(spec["sys"])
        out = _trajectory(osys, spec["sys"]["M"], spec["scheme"], spec["tol"], spec["ts"], spec["head"],
                          spec.get("steady_rtol", 0.0), verbose=bool(os.environ.get("ORACLE_RUNS_VERBOSE")),
                          head_every=spec.get("head_every", 1))
    meta = dict(name=name, spec=spec, seconds=round(time.time() - t0, 1),
                generator="tests/golden/make_oracle_runs.py (oracle/ numpy FP64, FFT route)")
    path = os.path.join(HERE, f"oracle_{name}.npz")
    np.savez_compressed(path, meta=json.dumps(meta), **out)
    print(f"{name}: {meta['seconds']} s -> {os.path.relpath(path, ROOT)}", flush=True)


def main(names):
    names = names or list(RUNS)
    for n in names:
        if n not in RUNS:
            raise SystemExit(f"unknown run {n}; choose from {', '.join(RUNS)}")
    env = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update(env)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=run, args=(n,)) for n in names]
    for p in procs:
        p.start()
    rc = 0
    for p in procs:
        p.join()
        rc = rc or p.exitcode
    return rc


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
