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
FLAG_NO_FUSE = 32           # smol_opts.flags bit (SMOL_FLAG_NO_FUSE)
L2_FLUSH_BYTES = 256 << 20
CTL_BYTES = 240             # the device control block of one system (smol::Ctl)

# Measured peaks (MEASURED_PEAKS.json of this machine, written by the pool's driver; read
# at run time when present) and the FP64 ALU peak: 152 SMs x 2070 MHz x 2 FP64 FMA per
# clock per SM x 2 flop = 1.259 TFLOP/s (a probe of dependent DFMA chains measured
# 1.20 TFLOP/s at ~1.97 GHz, i.e. 2 FMA / clk / SM).
HBM_FALLBACK_GBS = 6800.0
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12

# A schedule given on the command line (--schedule), per form; empty: autotuned.
FIXED_SCHEDULE = {}

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by
# (precision, kernel class); valid only while the kernel sources are unchanged.
TRAFFIC = {
    # profiles/k_rows_M131072_*.md, profiles/k_inv_fwd_M131072_*.md (dram read + write)
    ("fp64", "rows"): {"bytes": 8504320.0, "src": "516ef981546e9f6b"},
    ("fp64", "inv_fwd"): {"bytes": 9546752.0, "src": "516ef981546e9f6b"},
    ("fp32conv", "inv_fwd"): {"bytes": 4803072.0, "src": "516ef981546e9f6b"},
    ("fp32conv", "rows"): {"bytes": 4296448.0, "src": "516ef981546e9f6b"},
    ("df64", "inv_fwd"): {"bytes": 9574912.0, "src": "516ef981546e9f6b"},
    ("df64", "rows"): {"bytes": 8525824.0, "src": "516ef981546e9f6b"},
}


def src_digest() -> str:
    """Digest of the kernel sources with comments and blank lines removed (a change of
    code invalidates the recorded traffic, a change of comments does not)."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2407_16559_gb300", "csrc")
    for f in sorted(os.listdir(d)):
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
def oracle_rate(seconds: float, max_evals: int | None = None):
    """RHS evaluations per second of the oracle's O(M R log M) route (numpy FFT) inside
    its own adaptive RKF45 integration of the bench workload from the monodisperse
    start, run in slices of two attempts until about `seconds` or max_evals evaluations."""
    import numpy as np

    import oracle
    from synth import kernel_factors, monodisperse

    w = WORKLOAD
    U, V = kernel_factors("brownian", w["M"], a=w["a"])
    sysm = oracle.System(w["M"], w["lam"], U=U, V=V, route="lowrank")
    n = monodisperse(w["M"])
    sysm.rhs(n)  # warm
    evals, t, tau = 0, 0.0, 1e-3
    t0 = time.perf_counter()
    while True:
        n, st, _ = oracle.integrate(sysm, n, t, w["t1"], w["tol"],
                                    oracle.Options(scheme="rkf45", tau0=tau, max_attempts=2))
        evals += st["rhs_evals"]
        t, tau = st["t"], st["tau_next"]
        el = time.perf_counter() - t0
        if el >= seconds or (max_evals is not None and evals >= max_evals) or st["status"] not in (0, -5):
            break
    return evals / el, evals, el, float(np.sum(n))


def cpu_worker(args):
    rate, evals, el, _ = oracle_rate(args.cpu_seconds, args.cpu_max_evals)
    print(json.dumps({"rate": rate, "evals": evals, "seconds": el}))


def run_cpu_baseline(seconds: float, max_evals: int | None = None):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--cpu-seconds", str(seconds)]
    if max_evals:
        cmd += ["--cpu-max-evals", str(max_evals)]
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each step = one right-hand-side evaluation of the oracle (a bounded sample of
    # the workload's RKF45 attempt, which makes six of them)
    env_steps = args.steps + args.warmup
    res = run_cpu_baseline(seconds=1e9, max_evals=6 * max(1, (env_steps + 5) // 6))
    if res is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle subprocess failed"}))
        return 0
    v = res["rate"]
    line = {
        "impl": "reference", "metric": "rhs_evals_per_s", "value": v, "unit": "RHS evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": EVALS_PER_STEP * 1000.0 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config_dict("fp64"), n0="monodisperse, oracle attempts from t = 0", l2="n/a (host cores)"),
        "cpu_baseline": {"value": v, "unit": "RHS evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"{res['evals']} evaluations of S(n) (numpy-FFT route) inside oracle RKF45 "
                                   f"attempts at M=2^17 from the monodisperse start, one thread"},
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


def roofline(precision: str, prof_ms: dict, prof_cnt: dict, T: int, sched: dict) -> dict:
    """Roofline of the dominant kernel class of one form: FP64 against the FP64 pipe
    (the bound of its FFTs), the FP32 and double-float forms against the measured copy
    bandwidth (their bound in principle: they are latency-bound, and the fraction says
    how far they are from streaming). Durations are the live CUDA-event means per
    launch; work per launch from `algorithmic`."""
    csz = 8 if precision == "fp32conv" else 16
    fl, by = algorithmic(WORKLOAD["M"], T, csz, sched.get("fft_lgn1", 0))
    per_step = {k: prof_ms[k] * prof_cnt[k] for k in prof_ms}
    dom = max(("fwd_cols", "rows", "inv_cols", "inv_fwd"), key=lambda k: per_step.get(k, 0.0))
    peaks, pk_src = measured_peaks()
    # work per launch averaged over the profiled launches: a skipped evaluation (the retry
    # of a rejected attempt) makes one forward-column and one row launch do nothing and
    # one inverse pass only rescale k_1
    n, sk = max(prof_cnt[dom], 1), prof_cnt.get("skipped", 0)
    drop = {"fwd_cols": 1.0, "rows": 1.0, "inv_cols": 1.0, "inv_fwd": fl["inv_cols"] / fl["inv_fwd"]}[dom]
    fl = dict(fl, **{dom: fl[dom] * (1.0 - drop * sk / n)})
    drop_b = {"fwd_cols": 1.0, "rows": 1.0, "inv_cols": 1.0, "inv_fwd": by["inv_cols"] / by["inv_fwd"]}[dom]
    by = dict(by, **{dom: by[dom] * (1.0 - drop_b * sk / n)})
    if precision == "fp64":
        achieved = fl[dom] / (prof_ms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "FP64 FMA pipe: 152 SMs x 2070 MHz x 2 DFMA/clk",
                "algorithmic_per_launch": fl[dom]}
    else:
        pk = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
        achieved = by[dom] / (prof_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk, "unit": "GB/s",
                "frac": achieved / pk, "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({pk_src})",
                "algorithmic_per_launch": by[dom]}
    tr = TRAFFIC.get((precision, dom))
    roof["traffic"] = tr["bytes"] if tr and tr.get("src") == src_digest() else None
    roof["profiled_evals_skipped"] = sk
    roof["kernel_ms"] = {k: round(v * 1000.0, 3) for k, v in prof_ms.items()}
    roof["kernel_ms_unit"] = "us per launch (CUDA events, one kernel at a time)"
    return roof


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
        msb, stb, Ms, _ = time_batch(smol, torch, "fp32conv", K, W, stream, flush, args.batch,
                                     tune=not args.no_tune)
        if rank == 0:
            print(json.dumps({"batch_ms_per_step": msb / K, "systems": args.batch, "steps": K}))
        return 0
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

    roof = roofline(precision, prof_ms, prof_cnt, tsys.num_transforms, sched)

    cpu = None
    if rank == 0 and not args.no_cpu:
        res = run_cpu_baseline(args.cpu_seconds)
        if res:
            cpu = {"value": res["rate"], "unit": "RHS evals/s", "cores": 1, "kind": "oracle",
                   "sample": f"{res['evals']} evaluations of S(n) (numpy-FFT route, M=2^17) in oracle RKF45 "
                             f"attempts, {res['seconds']:.1f} s, one thread"}
    line = {
        "metric": "rhs_evals_per_s", "value": value, "unit": "RHS evals/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32conv": "f32+f64", "df64": "f32x2+f64"}[precision], "data": "synthetic",
        "config": dict(config_dict(precision), parallelism=f"replicas{world}",
                       schedule=sched or "rule (untuned)"),
        "accepted_steps_per_s": accepted_per_s,
        "attempts": {"accepted": tm["accepted"], "rejected": tm["rejected"], "rhs_evals": tm["rhs_evals"],
                     "t_end": stats["t"]},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": K * (LAUNCHES_UNFUSED if sched.get("flags", 0) & FLAG_NO_FUSE
                                                        else LAUNCHES_FUSED),
        "clocks": clocks,
    }
    if args.both and precision == "fp64":
        ms32, st32, pm32, pc32, tsys32, _, _, sch32 = time_form(smol, torch, "fp32conv", K, W, stream, flush, rank,
                                                                tune=not args.no_tune)
        v32 = world * st32["timed"]["rhs_evals"] / (ms32 / 1000.0)
        line["fp32conv"] = {"value": v32, "ms_per_step": ms32 / K, "speedup_vs_fp64": v32 / value,
                            "kernel_us": {k: round(v * 1000.0, 3) for k, v in pm32.items()}, "schedule": sch32,
                            "roofline": roofline("fp32conv", pm32, pc32, tsys32.num_transforms, sch32),
                            "rhs_rel_err_vs_fp64": rhs_accuracy(smol, torch, U, V)}
        # the FP64-accurate double-float form (FP64 parity tolerance 1e-10)
        msd, std_, pmd, pcd, tsysd, _, _, schd = time_form(smol, torch, "df64", K, W, stream, flush, rank,
                                                           tune=not args.no_tune)
        vd = world * std_["timed"]["rhs_evals"] / (msd / 1000.0)
        line["df64"] = {"value": vd, "ms_per_step": msd / K, "speedup_vs_fp64": vd / value,
                        "kernel_us": {k: round(v * 1000.0, 3) for k, v in pmd.items()}, "schedule": schd,
                        "roofline": roofline("df64", pmd, pcd, tsysd.num_transforms, schd),
                        "rhs_rel_err_vs_fp64": rhs_accuracy(smol, torch, U, V, "df64"),
                        "note": "FFTs, products and element-wise terms in double-float (FP32 pairs) on the "
                                "FP32 pipes; state, update, error, control in FP64; parity bar 1e-10 as FP64"}
    if args.batch > 0:
        # the batch shards across ranks by cost (smol_partition, no exchange while it
        # runs); one gather of the stats at the end
        from synth import batch_recipe
        rank_of, _ = smol.partition([r["M"] for r in batch_recipe(args.batch)], world)
        shard = smol.shard_indices(rank_of, rank) if world > 1 else None
        Kb = max(3, K // 10)
        barrier()
        msb, stb, Ms, bflags = time_batch(smol, torch, "fp32conv", Kb, W, stream, flush, args.batch,
                                          tune=not args.no_tune, shard=shard)
        if dist is not None:
            t = torch.tensor([msb], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            msb = float(t.item())
        stb = smol.gather_shards(stb, rank_of, dist) if world > 1 else stb
        evb = sum(x["rhs_evals"] for x in stb) if stb else 0
        acc = sum(x["accepted"] for x in stb) if stb else 0
        line["batch"] = {"systems": args.batch, "precision": "fp32conv", "steps": Kb, "ms_per_step": msb / Kb,
                         "rhs_evals_per_s": evb / (msb / 1000.0),
                         "accepted_steps_per_s": acc / (msb / 1000.0),
                         "scaling": "strong" if world > 1 else "n/a",
                         "elements": int(sum(r["M"] for r in batch_recipe(args.batch))), "launch_flags": bflags,
                         "note": "one step = one RKF45 attempt of every system; systems from seed 2407, "
                                 "M = 2^round(U(10,16)), a ~ U(0.2,0.9), lambda log-uniform [0.005, 0.1]; "
                                 "with N ranks the systems are split by cost, time = slowest rank"}
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


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
    b = smol.Batch(Us, Vs, lams, precision=precision, stream=stream, tau0=1e-3, chunk=1)
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
    return ms, stats, Ms, flags


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
    ap.add_argument("--batch", type=int, default=256, help="systems of the batched workload (0: skip)")
    ap.add_argument("--only-batch", action="store_true", help="time only the batched workload (profiling aid)")
    ap.add_argument("--no-tune", action="store_true", help="use the rule's FFT schedule and launch mode")
    ap.add_argument("--schedule", default=None,
                    help="fixed schedule 'lgn1,g,flags' for the headline form (skips its tuning; "
                         "for profiling runs that must not launch the tuner's kernels)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-max-evals", type=int, default=None)
    ap.add_argument("--cpu-worker", action="store_true")
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
