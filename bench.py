"""Throughput of the adaptive RKF45 integrator for the aggregation-shattering system.

Workload (oscillatory regime): M = 2^17 sizes, kernel K_ij = (i/j)^0.9 + (j/i)^0.9
(rank 2), shattering rate lambda = 0.005, monodisperse start n_s(0) = delta_{s1}, RKF45
with tol 1e-8 (Sec. 2 schemes, Eq. (4) system). Synthetic by definition: the paper's
experiments are fully specified by (M, K, lambda, n0).

One step = one RKF45 attempt: 6 evaluations of S(n) (5 when it retries a rejected
attempt, whose S(n^k) it keeps), the stage combination, the embedded error norm and the
step-size control, all on the device (13 kernel launches
with the column passes of consecutive evaluations fused, 19 without; captured in a CUDA
graph). Before the timed steps the system is advanced from t = 0 to t = 5 (untimed), and
the FFT schedule and launch mode are tuned (untimed), so that the attempts run
mid-trajectory with the fastest schedule. The same workload is also timed in the FP32
form and in the double-float form (FP64-accurate), and the 256-system batch.
value = S evaluations made per second over the K timed steps (counted by the device);
accepted RK steps per second are reported beside it. L2 (129 MB) is flushed between steps by writing a 256 MB
buffer outside the timed events (the system's working set, ~35 MB, would otherwise
stay resident).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32conv]
       python bench.py --impl reference ...   (the FP64 oracle on the host cores)
Under torchrun (N > 1) every rank integrates its own replica (the single system does not
shard); value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="oscill_M131072_brownian0.9_rkf45", M=131072, a=0.9, lam=0.005, tol=1e-8, t1=5000.0,
                t_setup=5.0, scheme="rkf45")
EVALS_PER_STEP = 6          # RKF45 stages
LAUNCHES_FUSED = 13         # forward columns, 6 x row kernel, 5 x fused inverse+forward columns,
                            # fused last inverse + combination / control
LAUNCHES_UNFUSED = 19       # 6 x (forward columns, rows, inverse columns) + combination / control
FLAG_NO_FUSE = 32           # smol_opts.flags bits (SMOL_FLAG_NO_FUSE, SMOL_FLAG_PERSISTENT: one
FLAG_PERSISTENT = 64        # cooperative launch per chunk of attempts; the timed chunk is one attempt)
L2_FLUSH_BYTES = 256 << 20
CTL_BYTES = 328             # the device control block of one system (smol::Ctl)

# Peaks. HBM: the copy bandwidth of MEASURED_PEAKS.json (written by the pool's driver;
# read at run time), else the fallback figure. FP64 and FP32 arithmetic: measured live
# before the timed region by smol_fma_rate (independent chains of dependent fused
# multiply-adds on every SM, CUDA events); the count 152 SMs x 2070 MHz x 2 FP64 FMA per
# clock is used only if that measurement fails, and is then labelled as derived.
HBM_FALLBACK_GBS = 6800.0
FP64_DERIVED_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12
FMA_ITERS = {"fp64": 20000, "fp32conv": 1000000}

# Element widths (bytes) of each form's compulsory traffic: the state read by stage
# inputs (the FP32 and double-float forms read their R-typed shadow of it), stage
# vectors k_i, weight vectors W_t, and the shadow written with each accepted state.
WIDTHS = {
    "fp64": dict(ws=8, wk=8, ww=8, shadow=0),
    "fp32conv": dict(ws=4, wk=4, ww=4, shadow=4),
    "df64": dict(ws=8, wk=8, ww=8, shadow=8),
}
RKF45_FINAL_TERMS = 5       # stage vectors the RKF45 candidate and error combine (k2 has weight 0)

# A schedule given on the command line (--schedule), per form; empty: autotuned.
FIXED_SCHEDULE = {}

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by
# (precision, kernel class); valid only while the kernel sources are unchanged.
TRAFFIC = {
    # (precision, kernel class, log2 N1 of the benched schedule): dram read + write per
    # launch from the ncu captures summarised in profiles/ (k_inv_fwd_M131072_*.md,
    # k_rows_M131072_*.md); used only while the kernel sources are the captured ones
    ("fp64", "inv_fwd", 9): {"bytes": 6413312.0, "src": "3d8769fd488ba7a2"},
    ("fp64", "rows", 9): {"bytes": 8491264.0, "src": "3d8769fd488ba7a2"},
    ("fp32conv", "inv_fwd", 8): {"bytes": 3231744.0, "src": "3d8769fd488ba7a2"},
    ("fp32conv", "rows", 8): {"bytes": 4298240.0, "src": "3d8769fd488ba7a2"},
    ("df64", "inv_fwd", 8): {"bytes": 6430720.0, "src": "3d8769fd488ba7a2"},
}


def src_digest() -> str:
    """Digest of the kernels' device code (the .cuh headers that define them) with
    comments and blank lines removed: a change of kernel code invalidates the recorded
    traffic, a change of comments or of the host code (tuners, entry points) does not.
    The traffic table is also keyed by the schedule's log2 N1."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2407_16559_gb300", "csrc")
    for f in sorted(x for x in os.listdir(d) if x.endswith(".cuh")):
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            code = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in code.splitlines():
            line = line.split("//", 1)[0].rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


# ---------------------------------------------------------------------------
# Algorithmic work per launch of each kernel class (FP64 flops / compulsory bytes)
# ---------------------------------------------------------------------------
def algorithmic(M: int, T: int, csz: int, lgn1: int = 0):
    """Per launch: flops of the FFT stages a kernel performs (5 N log2 N convention for
    a complex length-N transform, the real-FFT split / merge counted as one stage) and
    the bytes it must move (inputs read once, outputs written once). lgn1: log2 of the
    column length N1 of the four-step split (0: the rule, ceil(log2 Mp / 2))."""
    lg = (M - 1).bit_length()
    Mp = 1 << lg
    lg1 = lgn1 if lgn1 > 0 else (lg + 1) // 2
    lg2 = lg - lg1
    fl = {
        "fwd_cols": T * 5.0 * Mp * lg1,
        "rows": (T + 1) * 5.0 * Mp * (lg2 + 1),
        "inv_cols": 5.0 * Mp * lg1,
    }
    by = {
        # stage input (n and up to 5 stage vectors, ~3 on average) + T weights, T spectra out
        "fwd_cols": 8.0 * M * (3 + T) + T * csz * Mp,
        "rows": (T + 1) * csz * Mp,
        "inv_cols": csz * Mp + 8.0 * M * (2 + T) + 8.0 * M,
    }
    # the fused column kernels do both passes (inverse of one stage, forward of the next)
    fl["inv_fwd"] = fl["inv_cols"] + fl["fwd_cols"]
    by["inv_fwd"] = by["inv_cols"] + by["fwd_cols"]
    return fl, by


def compulsory(precision: str, T: int, stages: int = EVALS_PER_STEP, final_terms: int = RKF45_FINAL_TERMS):
    """Compulsory bytes per element (size s) of one RKF45 attempt and each kernel class's
    share of them per launch: every stage reads the state and the earlier stage vectors
    once, the T distinct weight vectors once, and writes its k_i once; the final
    combination reads the FP64 state and the stage vectors it combines and writes the
    new FP64 state (and its shadow). The spectra that move between the passes of the
    multi-pass FFT are not compulsory (an evaluation held on chip would not move them)."""
    w = WIDTHS[precision]
    reads = [w["ws"] + (i - 1) * w["wk"] + T * w["ww"] for i in range(1, stages + 1)]
    final = 8 + final_terms * w["wk"] + 8 + w["shadow"]
    attempt = sum(reads) + stages * w["wk"] + final
    per = {
        "fwd_cols": reads[0],                                   # stage 1 input and weights
        "rows": 0.0,                                            # spectra only
        "inv_cols": float(w["wk"]),                             # writes k_i
        "inv_fwd": w["wk"] + sum(reads[1:]) / (stages - 1),     # k_i out, stage i+1 in (mean)
        "inv_step": w["wk"] + final,                            # k_6 out, final combination
        "step": float(final),
    }
    return attempt, per


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.fh = None

    def __enter__(self):
        try:
            self.fh = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.fh is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.fh.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.fh.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle as it stands
# ---------------------------------------------------------------------------
def oracle_rate(seconds: float, max_evals: int | None = None, M: int | None = None, kind: str = "brownian",
                a: float | None = None, lam: float | None = None, tol: float | None = None):
    """RHS evaluations per second of the oracle's O(M R log M) route (numpy FFT) inside
    its own adaptive RKF45 integration from the monodisperse start (the bench workload
    unless M, kind, a, lam, tol say otherwise), run in slices of two attempts until
    about `seconds` or max_evals evaluations."""
    import numpy as np

    import oracle
    from synth import kernel_factors, monodisperse

    w = WORKLOAD
    M = M or w["M"]
    U, V = kernel_factors(kind, M, a=w["a"] if a is None else a)
    lam = w["lam"] if lam is None else lam
    tol = w["tol"] if tol is None else tol
    sysm = oracle.System(M, lam, U=U, V=V, route="lowrank")
    n = monodisperse(M)
    sysm.rhs(n)  # warm
    evals, t, tau = 0, 0.0, 1e-3
    t0 = time.perf_counter()
    while True:
        n, st, _ = oracle.integrate(sysm, n, t, w["t1"], tol, oracle.Options(scheme="rkf45", tau0=tau, max_attempts=2))
        evals += st["rhs_evals"]
        t, tau = st["t"], st["tau_next"]
        el = time.perf_counter() - t0
        if el >= seconds or (max_evals is not None and evals >= max_evals) or st["status"] not in (0, -5):
            break
    return evals / el, evals, el, float(np.sum(n))


def direct_numbers(seconds: float):
    """The oracle's direct O(M^2) route (the definition of Eq. (4)): RHS evaluations per
    second at M = 512; the time of one direct RHS at M = 2^17, extrapolated from the
    direct per-entry sums of a timed sample of sizes (a dense 2^17 x 2^17 kernel matrix
    would need 137 GB); and the accepted RKF45 steps per second of the M = 512 shattering
    workload (K = (i/j)^0.3 + (j/i)^0.3, lambda = 0.01, tol 1e-8 from the monodisperse
    start towards t = 200, for at most `seconds`)."""
    import numpy as np

    import oracle
    from synth import kernel_factors, monodisperse, sample_state

    out = {}
    U, V = kernel_factors("brownian", 512, a=0.3)
    osys = oracle.System(512, 0.01, U=U, V=V, route="direct")
    n = sample_state(512, 0.01)
    osys.rhs(n)
    k, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < min(2.0, seconds / 4):
        osys.rhs(n)
        k += 1
    out["direct_rhs_per_s_M512"] = k / (time.perf_counter() - t0)
    M = 1 << 17
    a = WORKLOAD["a"]
    nb = sample_state(M, WORKLOAD["lam"])
    sizes = np.random.default_rng(7).integers(2, M + 1, 32)
    t0 = time.perf_counter()
    oracle.rhs_entries_direct(nb, lambda i, j: (i / j) ** a + (j / i) ** a, WORKLOAD["lam"], sizes)
    per_entry = (time.perf_counter() - t0) / len(sizes)
    out["direct_rhs_seconds_M131072_extrapolated"] = per_entry * M
    out["direct_rhs_M131072_sample"] = f"{len(sizes)} direct per-entry sums timed, x M/{len(sizes)}"
    n = monodisperse(512)
    t, tau, acc = 0.0, 0.0, 0
    t0 = time.perf_counter()
    while t < 200.0 and time.perf_counter() - t0 < seconds / 2:
        n, st, _ = oracle.integrate(osys, n, t, 200.0, 1e-8, oracle.Options(scheme="rkf45", tau0=tau, max_attempts=20))
        acc += st["accepted"]
        t, tau = st["t"], st["tau_next"]
        if st["status"] not in (0, -5):
            break
    el = time.perf_counter() - t0
    out["shatter_M512_accepted_steps_per_s"] = acc / el
    out["shatter_M512_t_reached"] = t
    return out


def cpu_worker(args):
    if args.cpu_worker == "direct":
        print(json.dumps(direct_numbers(args.cpu_seconds)))
        return 0
    M = int(args.cpu_worker) if args.cpu_worker.isdigit() else None
    kw = dict(M=M, kind="brownian_const", a=1.0 / 3.0, lam=0.1, tol=1e-9) if M == 65536 else dict(M=M)
    rate, evals, el, _ = oracle_rate(args.cpu_seconds, args.cpu_max_evals, **kw)
    print(json.dumps({"rate": rate, "evals": evals, "seconds": el}))
    return 0


def _cpu_procs(kind: str, nproc: int, seconds: float, max_evals: int | None = None):
    """Runs `nproc` oracle worker processes of one kind at once (one thread each) and
    returns their JSON results (None if any failed)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", kind, "--cpu-seconds", str(seconds)]
    if max_evals:
        cmd += ["--cpu-max-evals", str(max_evals)]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, env=env)
          for _ in range(nproc)]
    res = []
    for p in ps:
        out, _ = p.communicate(timeout=900)
        if p.returncode != 0:
            return None
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res


def run_cpu_baseline(seconds: float):
    """The oracle as it stands on the host cores: its FFT-route RHS evaluations per
    second on the bench workload with one process per core (the headline baseline) and
    with one, the same at M = 2^16 (relaxation workload), and the direct-route numbers."""
    ncores = os.cpu_count() or 1
    allc = _cpu_procs("131072", ncores, seconds)
    if not allc:
        return None
    one = _cpu_procs("131072", 1, seconds)
    m16 = _cpu_procs("65536", 1, seconds / 2)
    direct = _cpu_procs("direct", 1, seconds)
    evals = sum(r["evals"] for r in allc)
    wall = max(r["seconds"] for r in allc)
    out = {"value": evals / wall, "unit": "RHS evals/s", "cores": ncores, "kind": "oracle",
           "sample": f"{evals} evaluations of S(n) (numpy-FFT route, M=2^17) in oracle RKF45 attempts from the "
                     f"monodisperse start, {ncores} single-threaded processes for {wall:.1f} s"}
    if one:
        out["value_1thread"] = one[0]["rate"]
    if m16:
        out["fft_rhs_per_s_M65536_1thread"] = m16[0]["rate"]
    out["fft_rhs_per_s_M131072_1thread"] = out.get("value_1thread")
    if direct:
        out.update(direct[0])
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each step = one RKF45 attempt of the oracle (six evaluations of S(n), a bounded
    # sample of the workload), spread over one single-threaded process per host core
    ncores = os.cpu_count() or 1
    steps = args.steps + args.warmup
    per = EVALS_PER_STEP * max(1, -(-steps // ncores))
    res = _cpu_procs("131072", ncores, 1e9, max_evals=per)
    if not res:
        print(json.dumps({"impl": "reference", "unavailable": "oracle subprocess failed"}))
        return 0
    evals = sum(r["evals"] for r in res)
    wall = max(r["seconds"] for r in res)
    v = evals / wall
    line = {
        "impl": "reference", "metric": "rhs_evals_per_s", "value": v, "unit": "RHS evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": EVALS_PER_STEP * 1000.0 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_dict("fp64"), n0="monodisperse, oracle attempts from t = 0", l2="n/a (host cores)"),
        "cpu_baseline": {"value": v, "unit": "RHS evals/s", "cores": ncores, "kind": "oracle",
                         "sample": f"{evals} evaluations of S(n) (numpy-FFT route) inside oracle RKF45 attempts "
                                   f"at M=2^17 from the monodisperse start, {ncores} single-threaded processes"},
        "e2e": {"value": v, "unit": "RHS evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict(precision: str):
    w = WORKLOAD
    return {"workload": w["name"], "M": w["M"], "kernel": f"(i/j)^{w['a']}+(j/i)^{w['a']} (rank 2)",
            "lambda": w["lam"], "n0": "monodisperse, advanced to t=5 before timing", "scheme": "rkf45",
            "tol": w["tol"], "precision": precision,
            "step": "one RKF45 attempt (6 RHS evaluations; 5 when it retries a rejected step, whose S(n^k) "
                    "it keeps); value counts the evaluations made",
            "l2": "flushed between timed steps (256 MB write outside the events)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_form(smol, torch, precision: str, K: int, W: int, stream, flush, rank: int, tune: bool = True):
    import numpy as np

    from synth import kernel_factors, monodisperse

    w = WORKLOAD
    U, V = kernel_factors("brownian", w["M"], a=w["a"])
    sysm = smol.System(U, V, w["lam"], precision=precision, stream=stream, tau0=1e-3, max_attempts=20000)
    n = torch.from_numpy(monodisperse(w["M"])).cuda()
    n, st0 = sysm.integrate(n, 0.0, w["t_setup"], w["tol"], scheme="rkf45")
    # FFT schedule and launch mode: timed candidates from this state (untimed set-up)
    sched = dict(FIXED_SCHEDULE.get(precision, {}))
    if tune and not sched:
        sched, tune_us = smol.tune(U, V, w["lam"], n, w["tol"], precision=precision, attempts=64, stream=stream)
        sched = dict(sched, tuned_us_per_attempt=round(tune_us, 1))
    opts = {k: v for k, v in sched.items() if k in smol.SCHEDULE_KEYS}
    # timed run: chunk of one attempt per graph launch
    tsys = smol.System(U, V, w["lam"], precision=precision, stream=stream, tau0=st0["tau_next"], chunk=1, **opts)
    run = tsys.start(n, st0["t"], w["t1"], w["tol"], scheme="rkf45")
    for _ in range(W):
        tsys.advance()
    # counters before the timed attempts (a retry of a rejected attempt reuses S(n^k),
    # so evaluations are counted, not assumed; the run continues after finish)
    _, stw = tsys.finish()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            tsys.advance()
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    run, stats = tsys.finish()
    timed = {k: stats[k] - stw[k] for k in ("rhs_evals", "accepted", "rejected", "attempts")}
    prof_ms, prof_cnt = tsys.profile(reps=10)
    _, stp = tsys.finish()
    # evaluations the profiled attempts skipped (retries keep S(n^k)): their forward and
    # row launches return at once and their inverse pass only rescales k_1
    prof_cnt["skipped"] = EVALS_PER_STEP * (stp["attempts"] - stats["attempts"]) - \
        (stp["rhs_evals"] - stats["rhs_evals"])
    del run
    return ms, dict(stats, timed=timed), prof_ms, prof_cnt, tsys, U, V, sched


def roofline(precision: str, prof_ms: dict, prof_cnt: dict, T: int, sched: dict, peaks: dict | None = None) -> dict:
    """Roofline of the dominant kernel class of one form. The FP64 form is bound by the
    FP64 pipe (its transforms' arithmetic): algorithmic FLOPs per launch over the
    measured FP64 FMA rate. The FP32 and double-float forms are reported against the
    measured copy bandwidth with their compulsory bytes per launch (compulsory); the
    FFT pass traffic they actually move is given beside it as a labelled diagnostic.
    Durations are the live CUDA-event means per launch; peaks: the live measurements
    {'fp64_tflops', 'fp32_tflops'} (None: derived FP64 figure)."""
    peaks = peaks or {}
    csz = 8 if precision == "fp32conv" else 16
    M = WORKLOAD["M"]
    fl, by = algorithmic(M, T, csz, sched.get("fft_lgn1", 0))
    _, comp = compulsory(precision, T)
    cb = {k: v * M for k, v in comp.items()}
    per_step = {k: prof_ms[k] * prof_cnt[k] for k in prof_ms}
    dom = max(("fwd_cols", "rows", "inv_cols", "inv_fwd"), key=lambda k: per_step.get(k, 0.0))
    hbm, hbm_src = measured_peaks()
    # work per launch averaged over the profiled launches: a skipped evaluation (the retry
    # of a rejected attempt) makes one forward-column and one row launch do nothing and
    # one inverse pass only rescale k_1
    n, sk = max(prof_cnt[dom], 1), prof_cnt.get("skipped", 0)
    drop = {"fwd_cols": 1.0, "rows": 1.0, "inv_cols": 1.0, "inv_fwd": fl["inv_cols"] / fl["inv_fwd"]}[dom]
    fl = dict(fl, **{dom: fl[dom] * (1.0 - drop * sk / n)})
    drop_b = {"fwd_cols": 1.0, "rows": 1.0, "inv_cols": 1.0, "inv_fwd": by["inv_cols"] / by["inv_fwd"]}[dom]
    by = dict(by, **{dom: by[dom] * (1.0 - drop_b * sk / n)})
    dt = prof_ms[dom] * 1e-3
    if precision == "fp64":
        pk = peaks.get("fp64_tflops")
        src = "FP64 FMA rate measured live (smol_fma_rate)" if pk else \
            "derived: 152 SMs x 2070 MHz x 2 DFMA/clk (live measurement unavailable)"
        pk = pk or FP64_DERIVED_TFLOPS
        achieved = fl[dom] / dt / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "peak_source": src, "algorithmic_per_launch": fl[dom],
                "algorithmic_unit": "FP64 flop (5 N log2 N per complex length-N transform stage set)"}
    else:
        pk = float(hbm.get("hbm_gbs", HBM_FALLBACK_GBS))
        # a skipped evaluation's forward pass reads nothing; its inverse pass still writes k_1
        comp_dom = cb[dom] * (1.0 - sk / n) if dom == "fwd_cols" else cb[dom]
        achieved = comp_dom / dt / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk, "unit": "GB/s",
                "frac": achieved / pk, "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({hbm_src})",
                "algorithmic_per_launch": comp_dom, "algorithmic_unit": "compulsory bytes",
                "fft_pass_bytes_per_launch": by[dom], "fft_pass_gbs": by[dom] / dt / 1e9,
                "fft_flop_rate_tflops": fl[dom] / dt / 1e12}
        if precision == "fp32conv" and peaks.get("fp32_tflops"):
            roof["fft_flop_frac_of_fp32"] = roof["fft_flop_rate_tflops"] / peaks["fp32_tflops"]
    tr = TRAFFIC.get((precision, dom, sched.get("fft_lgn1", 0)))
    roof["traffic"] = tr["bytes"] if tr and tr.get("src") == src_digest() else None
    roof["profiled_evals_skipped"] = sk
    roof["kernel_ms"] = {k: round(v * 1000.0, 3) for k, v in prof_ms.items()}
    roof["kernel_ms_unit"] = "us per launch (CUDA events, one kernel at a time)"
    return roof


def attempt_hbm(precision: str, T: int, elements: int, ms_per_step: float) -> dict:
    """Compulsory bytes of one attempt over the attempt's device time, as a fraction of
    the measured copy bandwidth (the per-attempt view beside the per-kernel roofline)."""
    per_el, _ = compulsory(precision, T)
    pk = float(measured_peaks()[0].get("hbm_gbs", HBM_FALLBACK_GBS))
    b = per_el * elements
    gbs = b / (ms_per_step * 1e-3) / 1e9
    return {"compulsory_bytes": b, "bytes_per_element": per_el, "gbs": gbs, "peak_gbs": pk, "frac": gbs / pk}


def live_peaks(smol, stream) -> dict:
    """FP64 and FP32 FMA rates measured now, on this GPU (untimed set-up)."""
    out = {}
    for key, prec in (("fp64_tflops", "fp64"), ("fp32_tflops", "fp32conv")):
        try:
            tf, ms = smol.fma_rate(prec, FMA_ITERS[prec], stream=stream)
            out[key] = tf
            out[key.replace("tflops", "ms")] = ms
        except Exception as e:  # reported, and the FP64 roofline falls back to the derived figure
            out[key] = None
            out[key.replace("tflops", "error")] = str(e)
    # dependent-chain latencies (SM cycles per operation, one warp; FP64 FMA also with 8)
    try:
        lat = {op: round(smol.op_latency(op, 1, stream=stream), 1) for op in smol.OP_LATENCY_OPS}
        lat["dfma_8warps"] = round(smol.op_latency("dfma", 8, stream=stream), 1)
        out["latency_cycles"] = lat
    except Exception as e:
        out["latency_error"] = str(e)
    return out


def gpu_arm(args):
    import numpy as np
    import torch

    import paper_2407_16559_gb300 as smol

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    K, W = args.steps, args.warmup
    precision = args.precision

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.only_batch:
        msb, stb, Ms, _, _ = time_batch(smol, torch, "fp32conv", K, W, stream, flush, args.batch,
                                     tune=not args.no_tune)
        if rank == 0:
            print(json.dumps({"batch_ms_per_step": msb / K, "systems": args.batch, "steps": K}))
        return 0
    peaks = {} if args.no_peaks else live_peaks(smol, stream)  # untimed set-up
    barrier()
    with ClockSampler(local) as clk:
        ms, stats, prof_ms, prof_cnt, tsys, U, V, sched = time_form(smol, torch, precision, K, W, stream, flush, rank,
                                                                    tune=not args.no_tune)
    barrier()
    clocks = clk.summary()
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    tm = stats["timed"]  # counters of the K timed attempts
    value = world * tm["rhs_evals"] / (ms / 1000.0)
    accepted_per_s = world * tm["accepted"] / (ms / 1000.0)

    # e2e: public API with host buffers, per step H2D state -> one attempt -> D2H state + stats
    sopts = {k: v for k, v in sched.items() if k in smol.SCHEDULE_KEYS}
    e2e = e2e_leg(smol, torch, precision, max(10, min(K, 400)), U, V, stream, sopts)

    T = tsys.num_transforms
    roof = roofline(precision, prof_ms, prof_cnt, T, sched, peaks)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = run_cpu_baseline(args.cpu_seconds)
    line = {
        "metric": "rhs_evals_per_s", "value": value, "unit": "RHS evals/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32conv": "f32+f64", "df64": "f32x2+f64"}[precision], "data": "synthetic",
        "config": dict(config_dict(precision), parallelism=f"replicas{world}",
                       schedule=sched or "rule (untuned)"),
        "accepted_steps_per_s": accepted_per_s,
        "attempts": {"accepted": tm["accepted"], "rejected": tm["rejected"], "rhs_evals": tm["rhs_evals"],
                     "t_end": stats["t"]},
        "roofline": roof, "attempt_hbm": attempt_hbm(precision, T, WORKLOAD["M"], ms / K),
        "peaks_live": peaks, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": K * (1 if sched.get("flags", 0) & FLAG_PERSISTENT else
                             (LAUNCHES_UNFUSED if sched.get("flags", 0) & FLAG_NO_FUSE else LAUNCHES_FUSED)),
        "clocks": clocks,
    }
    if args.both and precision == "fp64":
        for form in ("fp32conv", "df64"):
            msf, stf, pmf, pcf, tsf, _, _, schf = time_form(smol, torch, form, K, W, stream, flush, rank,
                                                            tune=not args.no_tune)
            vf = world * stf["timed"]["rhs_evals"] / (msf / 1000.0)
            line[form] = {"value": vf, "ms_per_step": msf / K, "rhs_evals_per_s_vs_fp64": vf / value,
                          "accepted_steps_per_s": world * stf["timed"]["accepted"] / (msf / 1000.0),
                          "kernel_us": {k: round(v * 1000.0, 3) for k, v in pmf.items()}, "schedule": schf,
                          "roofline": roofline(form, pmf, pcf, tsf.num_transforms, schf, peaks),
                          "attempt_hbm": attempt_hbm(form, tsf.num_transforms, WORKLOAD["M"], msf / K),
                          "rhs_rel_err_vs_fp64": rhs_accuracy(smol, torch, U, V, form)}
        line["df64"]["note"] = ("FFTs, products and element-wise terms in double-float (FP32 pairs) on the FP32 "
                                "pipes; state, update, error, control in FP64; parity bar 1e-10 as FP64")
    if args.tts and world == 1:
        line["time_to_solution"] = tts_relax(smol, torch, stream)
    if args.batch > 0:
        # the batch shards across ranks by cost (smol_partition, no exchange while it
        # runs); one gather of the stats at the end
        from synth import batch_recipe
        rec = batch_recipe(args.batch)
        rank_of, _ = smol.partition([r["M"] for r in rec], world)
        shard = smol.shard_indices(rank_of, rank) if world > 1 else None
        Kb = max(20, K)
        elements = int(sum(rec[q]["M"] for q in (shard if shard is not None else range(len(rec)))))
        forms = ("fp32conv", "df64", "fp64") if args.both else ("fp32conv",)
        res = {}
        for form in forms:
            barrier()
            msb, stb, Ms, bflags, bsched = time_batch(smol, torch, form, Kb, W, stream, flush, args.batch,
                                                      tune=not args.no_tune, shard=shard)
            if dist is not None:
                t = torch.tensor([msb], dtype=torch.float64, device="cuda")
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                msb = float(t.item())
            stb = smol.gather_shards(stb, rank_of, dist) if world > 1 else stb
            evb = sum(x["rhs_evals"] for x in stb) if stb else 0
            acc = sum(x["accepted"] for x in stb) if stb else 0
            res[form] = {"ms_per_step": msb / Kb, "rhs_evals_per_s": evb / (msb / 1000.0),
                         "accepted_steps_per_s": acc / (msb / 1000.0), "launch_flags": bflags,
                         "schedules": bsched or "rule",
                         "attempt_hbm": attempt_hbm(form, 2, elements, msb / Kb)}
        b = dict(res["fp32conv"], systems=args.batch, precision="fp32conv", steps=Kb,
                 scaling="strong" if world > 1 else "n/a", elements=int(sum(r["M"] for r in rec)),
                 note="one step = one RKF45 attempt of every system; systems from seed 2407, M = 2^round(U(10,16)), "
                      "a ~ U(0.2,0.9), lambda log-uniform [0.005, 0.1]; with N ranks the systems are split by cost, "
                      "time = slowest rank")
        for form in forms[1:]:
            b[form] = res[form]
        if "fp64" in res:
            for form in ("fp32conv", "df64"):
                b[f"{form}_attempt_speedup_vs_fp64"] = res["fp64"]["ms_per_step"] / res[form]["ms_per_step"]
        if args.tts and world == 1:
            b["time_to_solution"] = tts_batch(smol, torch, stream, args.batch, forms)
        line["batch"] = b
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


def _golden(name: str):
    """Oracle trajectory written by tests/golden/make_oracle_runs.py (oracle/ only)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.npz")
    if not os.path.exists(path):
        return None
    return dict(np.load(path, allow_pickle=False))


def rel_err_bound(head, tail_norm, ref_head, ref_tail):
    """Upper bound of ||n - n_ref||_2 / ||n_ref||_2 from the leading entries of both and
    the 2-norms of their remaining entries (triangle inequality on the remainder)."""
    import numpy as np
    d2 = float(np.sum((head - ref_head) ** 2)) + (tail_norm + ref_tail) ** 2
    return float(np.sqrt(d2 / (float(np.sum(ref_head ** 2)) + ref_tail ** 2)))


def tts_relax(smol, torch, stream):
    """Time to solution on the relaxation workload in its reduced-precision form setting
    (M = 2^16, K = (i/j)^{1/3} + (j/i)^{1/3} + 2, lambda = 0.1, RKF45 from the
    monodisperse start to t = 100 through 20 log-spaced checkpoints) in each form at tol
    1e-9 and 1e-6: device wall time, attempts, and the relative error of n(t) against the
    oracle's trajectory at every checkpoint (tests/golden). Each form's speedup over the
    FP64 solver is quoted with its worst checkpoint error."""
    import numpy as np

    from synth import kernel_factors, monodisperse
    M = 1 << 16
    U, V = kernel_factors("brownian_const", M, a=1.0 / 3.0)
    out = {"workload": "relax_M65536_brownian_const_lambda0.1_rkf45_to_t100", "checkpoints": 20}
    for tol, name in ((1e-9, "relax_rkf45_tol1e-9"), (1e-6, "relax_rkf45_tol1e-6")):
        g = _golden(name)
        if g is None:
            out[f"tol{tol:g}"] = "oracle trajectory missing"
            continue
        H = g["head"].shape[1]
        row = {}
        for form in ("fp64", "df64", "fp32conv"):
            sysm = smol.System(U, V, 0.1, precision=form, stream=stream, chunk=64)
            # untimed warm-up: graph capture and first-use costs stay out of the timing
            sysm.integrate(torch.from_numpy(monodisperse(M)).cuda(), 0.0, float(g["t"][0]), tol, scheme="rkf45")
            sysm.set_tau0(0.0)
            n = torch.from_numpy(monodisperse(M)).cuda()
            t, heads, tails, att = 0.0, [], [], 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for tc in g["t"]:
                n, st = sysm.integrate(n, t, float(tc), tol, scheme="rkf45", inplace=True)
                sysm.set_tau0(st["tau_next"])
                t = st["t"]
                att += st["attempts"]
                heads.append(n[:H].clone())
                tails.append(torch.linalg.vector_norm(n[H:]))
                if st["status"] != 0:
                    break
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            hidx = list(g["head_idx"]) if "head_idx" in g else list(range(len(g["head"])))
            errs = [rel_err_bound(heads[k].cpu().numpy(), float(tails[k]), g["head"][j], float(g["tail_norm"][j]))
                    for j, k in enumerate(hidx) if k < len(heads)]
            row[form] = {"seconds": wall, "attempts": att, "oracle_attempts": int(g["attempts"][len(errs) - 1]),
                         "max_rel_err_vs_oracle": max(errs), "first_rel_err": errs[0],
                         "mass_drift": abs(st["mass"] - float(g["mass"][len(errs) - 1])), "status": st["status"]}
        for form in ("df64", "fp32conv"):
            row[form]["speedup_vs_fp64"] = row["fp64"]["seconds"] / row[form]["seconds"]
        out[f"tol{tol:g}"] = row
    return out


def tts_batch(smol, torch, stream, count: int, forms):
    """Time to solution of the whole batch from the monodisperse starts to t = 2 (RKF45,
    tol 1e-8) in each form: device wall time, the largest attempt count of any system,
    the relative error against the oracle's trajectories of the batch's M = 1024 systems
    (tests/golden) and, for the reduced forms, against the FP64 batch over every system."""
    import numpy as np

    from synth import batch_recipe, kernel_factors, monodisperse
    g = _golden("batch_small")
    rec = batch_recipe(count)
    Us, Vs, lams = [], [], []
    for r in rec:
        U, V = kernel_factors("brownian", r["M"], a=r["a"])
        Us.append(U)
        Vs.append(V)
        lams.append(r["lam"])
    out, finals = {"t1": 2.0, "tol": 1e-8}, {}
    for form in forms:
        b = smol.Batch(Us, Vs, lams, precision=form, stream=stream, tau0=1e-3, chunk=64)
        ns = [torch.from_numpy(monodisperse(r["M"])).cuda() for r in rec]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, att, states = 0.0, np.zeros(count, dtype=np.int64), {}
        for tc in (0.5, 1.0, 2.0):
            ns, st = b.integrate(ns, t, tc, 1e-8, inplace=True)
            b.set_tau0([x["tau_next"] for x in st])
            att += np.array([x["attempts"] for x in st])
            t = tc
            states[tc] = [x.clone() for x in ns] if g is not None else None
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        row = {"seconds": wall, "max_attempts": int(att.max()), "sum_attempts": int(att.sum()),
               "statuses": sorted({x["status"] for x in st})}
        if g is not None:
            errs = []
            for q in g["systems"]:
                for k, tc in enumerate((0.5, 1.0, 2.0)):
                    ref = g[f"s{q}_head"][k]
                    got = states[tc][q].cpu().numpy()
                    errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
            row["max_rel_err_vs_oracle"] = max(errs)
            row["oracle_systems"] = len(g["systems"])
        finals[form] = [x.cpu().numpy() for x in ns]
        out[form] = row
    if "fp64" in finals:
        for form in forms:
            if form == "fp64":
                continue
            e = [float(np.linalg.norm(a - r) / np.linalg.norm(r)) for a, r in zip(finals[form], finals["fp64"])]
            out[form]["max_rel_err_vs_fp64_all_systems"] = max(e)
            out[form]["median_rel_err_vs_fp64_all_systems"] = float(np.median(e))
            out[form]["speedup_vs_fp64"] = out["fp64"]["seconds"] / out[form]["seconds"]
    return out


def time_batch(smol, torch, precision: str, K: int, W: int, stream, flush, count: int = 256, tune: bool = True,
               shard=None):
    """The batched workload: `count` independent systems (M = 2^round(U(10,16)), kernel
    (i/j)^a + (j/i)^a with a ~ U(0.2, 0.9), lambda log-uniform in [0.005, 0.1],
    monodisperse starts, seed 2407), each with its own adaptive RKF45 step (tol 1e-8).
    One step = one attempt of every system (one graph launch whose kernels span all
    systems). Returns device ms over K steps and the systems' stats."""
    from synth import batch_recipe, kernel_factors, monodisperse
    rec = batch_recipe(count)
    if shard is not None:  # this rank's systems (smol_partition)
        rec = [rec[q] for q in shard]
    Us, Vs, lams, n0s = [], [], [], []
    for r in rec:
        U, V = kernel_factors("brownian", r["M"], a=r["a"])
        Us.append(U)
        Vs.append(V)
        lams.append(r["lam"])
        n0s.append(torch.from_numpy(monodisperse(r["M"])).cuda())
    tables = {}
    if tune:  # FFT schedules per size class, then the launch mode (untimed set-up)
        tables, _ = smol.batch_tune_schedules(Us, Vs, lams, n0s, 1e-8, attempts=4, precision=precision,
                                              stream=stream, tau0=1e-3, chunk=1)
    b = smol.Batch(Us, Vs, lams, precision=precision, stream=stream, tau0=1e-3, chunk=1, **tables)
    flags = b.tune(n0s, 1e-8, attempts=8)[0] if tune else 0
    b.start(n0s, 0.0, 1000.0, 1e-8, scheme="rkf45")
    for _ in range(W):
        b.advance()
    _, stw = b.finish()  # counters before the timed attempts (the run continues)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            b.advance()
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev)
    _, stats = b.finish()
    # per system: the counters of the K timed attempts
    stats = [{k: x[k] - y[k] for k in ("rhs_evals", "accepted", "rejected", "attempts")} for x, y in zip(stats, stw)]
    Ms = [r["M"] for r in rec]
    sched = {str(1 << k): [int(tables["batch_lgn1"][k]), int(tables["batch_g"][k])]
             for k in range(len(tables.get("batch_lgn1", []))) if tables["batch_lgn1"][k] or tables["batch_g"][k]}
    return ms, stats, Ms, flags, sched


def rhs_accuracy(smol, torch, U, V, precision: str = "fp32conv"):
    """Normwise relative error of the reduced-precision S(n) against the FP64 one (which
    matches the oracle to ~1e-15) on the workload's mid-run sample state."""
    from synth import sample_state
    w = WORKLOAD
    n = torch.from_numpy(sample_state(w["M"], w["lam"])).cuda()
    a = smol.System(U, V, w["lam"]).rhs(n)
    b = smol.System(U, V, w["lam"], precision=precision).rhs(n)
    return float((a - b).norm() / a.norm())


def e2e_leg(smol, torch, precision, K, U, V, stream, sched=None):
    """Per step: pinned host state -> device, one RKF45 attempt through smol_integrate,
    device -> pinned host state; wall time of K steps."""
    from synth import monodisperse
    w = WORKLOAD
    M = w["M"]
    sysm = smol.System(U, V, w["lam"], precision=precision, stream=stream, tau0=1e-3, max_attempts=1, chunk=1,
                       **(sched or {}))
    h = torch.from_numpy(monodisperse(M)).pin_memory()
    d = torch.empty(M, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(3):
        d.copy_(h, non_blocking=True)
        sysm.integrate(d, t, w["t1"], w["tol"], inplace=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tc = 0.0
    evals = 0
    with torch.cuda.stream(stream):
        for _ in range(K):
            d.copy_(h, non_blocking=True)
            _, st = sysm.integrate(d, tc, w["t1"], w["tol"], inplace=True)
            h.copy_(d, non_blocking=True)
            stream.synchronize()
            tc = st["t"]
            evals += st["rhs_evals"]
    el = time.perf_counter() - t0
    # state both ways, plus the control block (CTL_BYTES) uploaded at start and read back
    # (status snapshot and final read) by smol_integrate
    return {"value": evals / el, "unit": "RHS evals/s", "h2d_bytes_per_step": 8 * M + CTL_BYTES,
            "d2h_bytes_per_step": 8 * M + 2 * CTL_BYTES, "steps": K}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32conv", "df64"])
    ap.add_argument("--both", action="store_true", default=True)
    ap.add_argument("--no-both", dest="both", action="store_false")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the live FMA-rate measurement (profiling runs; the FP64 roofline then uses the "
                         "derived figure and says so)")
    ap.add_argument("--tts", action="store_true", default=True,
                    help="time-to-solution legs against the oracle's trajectories (default on)")
    ap.add_argument("--no-tts", dest="tts", action="store_false")
    ap.add_argument("--batch", type=int, default=256, help="systems of the batched workload (0: skip)")
    ap.add_argument("--only-batch", action="store_true", help="time only the batched workload (profiling aid)")
    ap.add_argument("--no-tune", action="store_true", help="use the rule's FFT schedule and launch mode")
    ap.add_argument("--schedule", default=None,
                    help="fixed schedule 'lgn1,g,flags' for the headline form (skips its tuning; "
                         "for profiling runs that must not launch the tuner's kernels)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-max-evals", type=int, default=None)
    ap.add_argument("--cpu-worker", default=None, help="internal: one oracle worker process")
    ap.add_argument("--t-setup", type=float, default=WORKLOAD["t_setup"],
                    help="untimed integration span before the timed steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_worker:
        return cpu_worker(args)
    WORKLOAD["t_setup"] = args.t_setup
    if args.schedule:
        lg, g, fl = (int(x) for x in args.schedule.split(","))
        FIXED_SCHEDULE[args.precision] = {"fft_lgn1": lg, "fft_g": g, "flags": fl}
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main() or 0)
