"""GB300 (sm_103a) solver for the truncated aggregation-shattering Smoluchowski system
with a low-rank kernel, after Matveev, Zhilin, Smirnov, "Adaptive time-stepping for
aggregation-shattering kinetics" (arXiv 2407.16559).

This module is a thin ctypes binding of the C interface in ``include/smol.h``: it only
marshals arguments. Every step of the computation (right-hand side of Eq. (4), RK
stages, error norms, step control) runs in the CUDA kernels of ``libsmol.so``.
PyTorch provides the device memory (workspace, state vectors) and the stream.
There is no CPU fallback: importing this package fails if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmol.so")

OK, STEADY = 0, 1
EINVAL, ECUDA, ENONFINITE, ESTEP_UNDERFLOW, EMAXATTEMPTS, ETIMEOUT, ENOSPACE, EUNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8)
SCHEMES = {"rk2": 0, "rk4": 1, "rkf45": 2}
PRECISIONS = {"fp64": 0, "fp32conv": 1, "df64": 2}
CTRLS = {"double_halve": 0, "formula": 1}
NORMS = {"abs": 0, "rel": 1}


class SmolError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("ctrl", ctypes.c_int32), ("norm", ctypes.c_int32),
        ("log_capacity", ctypes.c_int32), ("tau0", ctypes.c_double), ("euler_a", ctypes.c_double),
        ("tau_min_rel", ctypes.c_double), ("steady_rtol", ctypes.c_double), ("fixed_tau", ctypes.c_double),
        ("fac_min", ctypes.c_double), ("fac_max", ctypes.c_double), ("max_attempts", ctypes.c_int64),
        ("chunk", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p),
        ("fft_lgn1", ctypes.c_int32), ("fft_g", ctypes.c_int32),
        ("batch_lgn1", ctypes.c_int8 * 24), ("batch_g", ctypes.c_int8 * 24),
    ]


SIZE_CLASSES = 24  # SMOL_SIZE_CLASSES: batch_lgn1 / batch_g entry k serves Mp = 2^k


class Stats(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("tau_next", ctypes.c_double), ("err_last", ctypes.c_double),
        ("mass", ctypes.c_double), ("rhs_evals", ctypes.c_int64), ("rhs_evals_paper", ctypes.c_int64), ("accepted", ctypes.c_int64),
        ("rejected", ctypes.c_int64), ("attempts", ctypes.c_int64), ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_P, _D, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t

# name -> (restype, argtypes); the exported symbols of include/smol.h
SIGNATURES = {
    "smol_default_opts": (None, [ctypes.POINTER(Opts)]),
    "smol_max_m": (_I64, [_I32, _I32]),
    "smol_workspace_bytes": (_SZ, [_I64, _I32, ctypes.POINTER(Opts)]),
    "smol_init_system": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I32, _P, _P, _D, ctypes.POINTER(Opts), _P, _SZ]),
    "smol_set_stream": (ctypes.c_int, [_P, _P]),
    "smol_rhs": (ctypes.c_int, [_P, _P, _P]),
    "smol_rhs_terms": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "smol_integrate": (ctypes.c_int, [_P, _P, _D, _D, _D, _I32, ctypes.POINTER(Stats)]),
    "smol_integrate_start": (ctypes.c_int, [_P, _P, _D, _D, _D, _I32]),
    "smol_integrate_advance": (ctypes.c_int, [_P]),
    "smol_integrate_finish": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "smol_profile_attempts": (ctypes.c_int, [_P, _I32, _P, _P, _I32]),
    "smol_get_log": (ctypes.c_int, [_P, _P, _P, _P, _P, _I32, ctypes.POINTER(_I64)]),
    "smol_num_transforms": (ctypes.c_int, [_P]),
    "smol_destroy": (None, [_P]),
    "smol_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "smol_rhs_static": (ctypes.c_int, [_I64, _I32, _P, _P, _D, _P, _P, _P]),
    "smol_batch_workspace_bytes": (_SZ, [_I32, _P, _I32, ctypes.POINTER(Opts)]),
    "smol_batch_init": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _P, _I32, _P, _P, _P, ctypes.POINTER(Opts), _P,
                                       _SZ]),
    "smol_batch_set_stream": (ctypes.c_int, [_P, _P]),
    "smol_batch_integrate": (ctypes.c_int, [_P, _P, _D, _D, _D, _I32, _P]),
    "smol_batch_integrate_start": (ctypes.c_int, [_P, _P, _D, _D, _D, _I32]),
    "smol_batch_integrate_advance": (ctypes.c_int, [_P]),
    "smol_batch_integrate_finish": (ctypes.c_int, [_P, _P]),
    "smol_batch_get_log": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _I32, ctypes.POINTER(_I64)]),
    "smol_batch_destroy": (None, [_P]),
    "smol_tune": (ctypes.c_int, [_I64, _I32, _P, _P, _D, _P, _D, _I32, _I32, ctypes.POINTER(Opts), ctypes.POINTER(_D)]),
    "smol_batch_tune": (ctypes.c_int, [_P, _P, _D, _I32, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_D)]),
    "smol_partition": (ctypes.c_int, [_I32, _P, _P, _I32, _P, _P]),
    "smol_set_sources": (ctypes.c_int, [_P, _I32, _P, _P]),
    "smol_batch_set_sources": (ctypes.c_int, [_P, _I32, _I32, _P, _P]),
    "smol_set_tau0": (ctypes.c_int, [_P, _D]),
    "smol_fma_rate": (ctypes.c_int, [_I32, _I64, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "smol_op_latency": (ctypes.c_int, [_I32, _I32, _P, ctypes.POINTER(_D)]),
    "smol_max_m_transforms": (_I64, [_I32, _I32]),
    "smol_lowrank_kernel": (ctypes.c_int, [_I32, _P, _I64, _D, _I32, _P, _P, ctypes.POINTER(_I32),
                                           ctypes.POINTER(_D)]),
    "smol_batch_set_tau0": (ctypes.c_int, [_P, _P]),
    "smol_batch_tune_schedules": (ctypes.c_int, [_I32, _P, _I32, _P, _P, _P, _P, _D, _I32, _I32, _P,
                                                 ctypes.POINTER(_D)]),
}

# option flags (smol_opts.flags)
FLAG_NO_PDL, FLAG_NO_PDL_FWD_COLS, FLAG_NO_PDL_ROWS, FLAG_NO_PDL_INV_COLS, FLAG_NO_PDL_STEP = 1, 2, 4, 8, 16
FLAG_NO_FUSE = 32
FLAG_PERSISTENT = 64
FLAG_WIDE_COLS = 128
SCHEDULE_KEYS = ("fft_lgn1", "fft_g", "flags")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libsmol.so not built at {path}; run `python paper_2407_16559_gb300/build.py` "
                          "(needs nvcc; the kernels are the only implementation, there is no fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def strerror(code: int) -> str:
    return _lib.smol_strerror(int(code)).decode()


def default_opts() -> Opts:
    o = Opts()
    _lib.smol_default_opts(ctypes.byref(o))
    return o


def max_m(R: int, precision: str = "fp64") -> int:
    return int(_lib.smol_max_m(R, PRECISIONS[precision]))


STATIC_MAX_M, STATIC_MAX_R = 65536, 3


def rhs_static(U, V, lam: float, n, out=None, stream=None):
    """smol_rhs_static: S(n) without a system object or workspace (FP64). U (M, R) and
    V (R, M) are device tensors (or arrays copied to the device); n a device tensor."""
    torch = _torch()
    n = torch.as_tensor(n).to(device="cuda", dtype=torch.float64).contiguous()
    U = torch.as_tensor(U).to(device=n.device, dtype=torch.float64).contiguous()
    V = torch.as_tensor(V).to(device=n.device, dtype=torch.float64).contiguous()
    M, R = U.shape
    if out is None:
        out = torch.empty_like(n)
    st = stream if stream is not None else torch.cuda.current_stream(n.device)
    _check(_lib.smol_rhs_static(M, R, U.data_ptr(), V.data_ptr(), float(lam), n.data_ptr(), out.data_ptr(),
                                st.cuda_stream), "smol_rhs_static")
    return out


KERNELS = {"const": 0, "brownian": 1, "free_molecular": 2}
MAX_R = 16


def max_m_transforms(T: int, precision: str = "fp64") -> int:
    """Largest M for T distinct forward transforms (smol_max_m_transforms)."""
    return int(_lib.smol_max_m_transforms(int(T), PRECISIONS[precision]))


def lowrank_kernel(kind: str, M: int, tol: float = 1e-10, max_rank: int = MAX_R, a: float = 0.0, c: float = 0.0):
    """smol_lowrank_kernel: symmetric cross approximation K ~= U V of a kernel of Sec. 3.1
    on sizes 1..M (host code). Returns (U (M, R), V (R, M), sampled max relative entry
    error)."""
    U = np.zeros(M * max_rank)
    V = np.zeros(max_rank * M)
    par = np.array([a, c], dtype=np.float64)
    r, e = ctypes.c_int32(), ctypes.c_double()
    _check(_lib.smol_lowrank_kernel(KERNELS[kind], par.ctypes.data, int(M), float(tol), int(max_rank), U.ctypes.data,
                                    V.ctypes.data, ctypes.byref(r), ctypes.byref(e)), "smol_lowrank_kernel")
    R = r.value
    return U[: M * R].reshape(M, R).copy(), V[: R * M].reshape(R, M).copy(), e.value


def fma_rate(precision: str = "fp64", iters: int = 20000, stream=None):
    """smol_fma_rate: measured fused multiply-add rate (TFLOP/s, FMA = 2 flop) and the
    timed kernel's milliseconds, in FP64 ('fp64') or FP32 ('fp32conv')."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.smol_fma_rate(PRECISIONS[precision], int(iters), ctypes.c_void_p(stream.cuda_stream),
                              ctypes.byref(tf), ctypes.byref(ms)), "smol_fma_rate")
    return tf.value, ms.value


OP_LATENCY_OPS = {"dfma": 0, "dadd": 1, "ffma": 2, "f2f_dmul": 3}


def op_latency(op: str, warps: int = 1, stream=None) -> float:
    """smol_op_latency: SM cycles per operation of a dependent chain of `op` ('dfma',
    'dadd', 'ffma', 'f2f_dmul') run by `warps` warps of one CTA."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    c = ctypes.c_double()
    _check(_lib.smol_op_latency(OP_LATENCY_OPS[op], int(warps), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(c)), "smol_op_latency")
    return c.value


def tune(U, V, lam: float, n0, tol: float, scheme: str = "rkf45", precision: str = "fp64", attempts: int = 64,
         stream=None, device=None, **opts):
    """smol_tune: times the candidate FFT schedules and launch modes of this problem
    and returns ({fft_lgn1, fft_g, flags}, microseconds per attempt); pass the dict as
    options to System."""
    torch = _torch()
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    M, R = U.shape
    o, dev, _ = _make_opts(precision, stream, device, opts)
    n0 = torch.as_tensor(n0).to(device=dev, dtype=torch.float64).contiguous()
    us = ctypes.c_double()
    _check(_lib.smol_tune(M, R, U.ctypes.data, V.ctypes.data, float(lam), n0.data_ptr(), float(tol), SCHEMES[scheme],
                          int(attempts), ctypes.byref(o), ctypes.byref(us)), "smol_tune")
    return {k: int(getattr(o, k)) for k in SCHEDULE_KEYS}, us.value


def partition(Ms, nranks: int, weights=None):
    """smol_partition: rank of each system of a batch across nranks GPUs (cost-balanced,
    deterministic) and each rank's load."""
    Ms = np.ascontiguousarray(Ms, dtype=np.int64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    rank_of = np.zeros(Ms.size, dtype=np.int32)
    load = np.zeros(int(nranks), dtype=np.float64)
    _check(_lib.smol_partition(Ms.size, Ms.ctypes.data, None if w is None else w.ctypes.data, int(nranks),
                               rank_of.ctypes.data, load.ctypes.data), "smol_partition")
    return rank_of, load


def shard_indices(rank_of, rank: int):
    """The systems of this rank, in batch order."""
    return [q for q, r in enumerate(rank_of) if int(r) == int(rank)]


def gather_shards(local: list, rank_of, dist=None, dst: int = 0):
    """One gather at the end of a sharded batch run: `local` holds this rank's results in
    the order of shard_indices(rank_of, rank); the destination rank receives all results
    in batch order (others receive None). Host objects only (states copied to the host
    by the caller); torch.distributed with any backend."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(local)
    rank, world = dist.get_rank(), dist.get_world_size()
    parts = [None] * world if rank == dst else None
    dist.gather_object(list(local), parts, dst=dst)
    if rank != dst:
        return None
    out = [None] * len(rank_of)
    for r in range(world):
        for q, item in zip(shard_indices(rank_of, r), parts[r]):
            out[q] = item
    return out


def _check(rc: int, what: str):
    if rc < 0:
        raise SmolError(rc, what)
    return rc


def _torch():
    import torch  # imported lazily: the CPU-only symbol tests need no torch
    return torch


def _make_opts(precision: str, stream, device, opts: dict):
    torch = _torch()
    o = default_opts()
    o.precision = PRECISIONS[precision]
    for k, v in opts.items():
        if k == "ctrl":
            v = CTRLS[v]
        elif k == "norm":
            v = NORMS[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        if k in ("batch_lgn1", "batch_g"):
            vals = [int(x) for x in v]
            if len(vals) > SIZE_CLASSES:
                raise ValueError(f"{k}: at most {SIZE_CLASSES} entries")
            v = (ctypes.c_int8 * SIZE_CLASSES)(*(vals + [0] * (SIZE_CLASSES - len(vals))))
        setattr(o, k, v)
    dev = torch.device(device if device is not None else "cuda")
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    o.stream = ctypes.c_void_p(stream.cuda_stream)
    return o, dev, stream


def batch_tune_schedules(Us, Vs, lams, n0s, tol: float, scheme: str = "rkf45", attempts: int = 8,
                         precision: str = "fp64", stream=None, device=None, **opts):
    """smol_batch_tune_schedules: FFT schedules per size class for the batch (Us, Vs,
    lams) from the states n0s (device tensors or arrays); returns ({'batch_lgn1': [...],
    'batch_g': [...]}, microseconds per attempt of the whole batch). Pass the dict as
    options to Batch."""
    torch = _torch()
    U = [np.ascontiguousarray(u, dtype=np.float64) for u in Us]
    V = [np.ascontiguousarray(v, dtype=np.float64) for v in Vs]
    count, R = len(U), U[0].shape[1]
    M = np.array([u.shape[0] for u in U], dtype=np.int64)
    lam = np.ascontiguousarray(lams, dtype=np.float64)
    o, dev, _ = _make_opts(precision, stream, device, opts)
    ns = [torch.as_tensor(n).to(device=dev, dtype=torch.float64).contiguous() for n in n0s]
    pU = (ctypes.c_void_p * count)(*[u.ctypes.data for u in U])
    pV = (ctypes.c_void_p * count)(*[v.ctypes.data for v in V])
    pn = (ctypes.c_void_p * count)(*[n.data_ptr() for n in ns])
    us = ctypes.c_double()
    _check(_lib.smol_batch_tune_schedules(count, M.ctypes.data, R, pU, pV, lam.ctypes.data, pn, float(tol),
                                          SCHEMES[scheme], int(attempts), ctypes.byref(o), ctypes.byref(us)),
           "smol_batch_tune_schedules")
    return {"batch_lgn1": list(o.batch_lgn1), "batch_g": list(o.batch_g)}, us.value


class Batch:
    """A batch of independent systems advanced together (smol_batch_*): systems q =
    0..count-1 with U[q] (M_q, R), V[q] (R, M_q), lam[q]; the same options for all."""

    def __init__(self, Us, Vs, lams, precision: str = "fp64", stream=None, device=None, **opts):
        torch = _torch()
        self.U = [np.ascontiguousarray(u, dtype=np.float64) for u in Us]
        self.V = [np.ascontiguousarray(v, dtype=np.float64) for v in Vs]
        self.count = len(self.U)
        self.R = self.U[0].shape[1]
        self.M = np.array([u.shape[0] for u in self.U], dtype=np.int64)
        for u, v in zip(self.U, self.V):
            if u.shape[1] != self.R or v.shape != (self.R, u.shape[0]):
                raise ValueError("every U must be (M_q, R) and V (R, M_q) with the same R")
        self.lam = np.ascontiguousarray(lams, dtype=np.float64)
        self.opts, self.device, self.stream = _make_opts(precision, stream, device, opts)
        nbytes = int(_lib.smol_batch_workspace_bytes(self.count, self.M.ctypes.data, self.R, ctypes.byref(self.opts)))
        if nbytes == 0:
            raise SmolError(EUNSUPPORTED, "batch shape")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ws = (self.workspace.data_ptr() + 255) & ~255
        self._pU = (ctypes.c_void_p * self.count)(*[u.ctypes.data for u in self.U])
        self._pV = (ctypes.c_void_p * self.count)(*[v.ctypes.data for v in self.V])
        self._h = ctypes.c_void_p()
        _check(_lib.smol_batch_init(ctypes.byref(self._h), self.count, self.M.ctypes.data, self.R, self._pU, self._pV,
                                    self.lam.ctypes.data, ctypes.byref(self.opts), ws, nbytes), "smol_batch_init")

    def _states(self, ns):
        torch = _torch()
        out = []
        for q, n in enumerate(ns):
            if not isinstance(n, torch.Tensor):
                n = torch.as_tensor(np.asarray(n, dtype=np.float64))
            n = n.to(device=self.device, dtype=torch.float64).contiguous()
            if n.numel() != self.M[q]:
                raise ValueError(f"state {q} has {n.numel()} entries, expected {self.M[q]}")
            out.append(n)
        return out, (ctypes.c_void_p * self.count)(*[n.data_ptr() for n in out])

    def integrate(self, n0s, t0: float, t1: float, tol: float, scheme: str = "rkf45", inplace: bool = False):
        """Integrates every system from t0 to t1; returns (list of device states, list
        of stats dicts)."""
        ns, ptrs = self._states(n0s)
        if not inplace:
            ns = [n.clone() for n in ns]
            ptrs = (ctypes.c_void_p * self.count)(*[n.data_ptr() for n in ns])
        st = (Stats * self.count)()
        rc = _lib.smol_batch_integrate(self._h, ptrs, float(t0), float(t1), float(tol), SCHEMES[scheme], st)
        if rc in (EINVAL, ECUDA, ENOSPACE, EUNSUPPORTED):
            raise SmolError(rc, "smol_batch_integrate")
        return ns, [s.as_dict() for s in st]

    def set_sources(self, system: int, sources: dict):
        """Point sources {s: P_s} (1-based sizes) of Eq. (3) for one system of the batch."""
        k = np.ascontiguousarray(list(sources.keys()), dtype=np.int64)
        v = np.ascontiguousarray(list(sources.values()), dtype=np.float64)
        _check(_lib.smol_batch_set_sources(self._h, int(system), k.size, k.ctypes.data, v.ctypes.data),
               "smol_batch_set_sources")

    def set_tau0(self, tau0s):
        """First steps of the next integration, per system (0: the batch's tau0 option);
        resuming with each system's stats['tau_next'] continues its step sequence."""
        v = np.ascontiguousarray(tau0s, dtype=np.float64)
        if v.size != self.count:
            raise ValueError("one tau0 per system")
        _check(_lib.smol_batch_set_tau0(self._h, v.ctypes.data), "smol_batch_set_tau0")

    def tune(self, n0s, tol: float, scheme: str = "rkf45", attempts: int = 16):
        """smol_batch_tune: keeps the fastest launch mode for this batch; returns
        (flags, microseconds per attempt of the whole batch)."""
        ns, ptrs = self._states(n0s)
        fl, us = ctypes.c_int32(), ctypes.c_double()
        _check(_lib.smol_batch_tune(self._h, ptrs, float(tol), SCHEMES[scheme], int(attempts), ctypes.byref(fl),
                                    ctypes.byref(us)), "smol_batch_tune")
        self.opts.flags = fl.value
        return fl.value, us.value

    def start(self, n0s, t0, t1, tol, scheme="rkf45"):
        ns, ptrs = self._states(n0s)
        self._run = ns
        _check(_lib.smol_batch_integrate_start(self._h, ptrs, float(t0), float(t1), float(tol), SCHEMES[scheme]),
               "smol_batch_integrate_start")
        return ns

    def advance(self):
        _check(_lib.smol_batch_integrate_advance(self._h), "smol_batch_integrate_advance")

    def finish(self):
        st = (Stats * self.count)()
        rc = _lib.smol_batch_integrate_finish(self._h, st)
        if rc in (EINVAL, ECUDA):
            raise SmolError(rc, "smol_batch_integrate_finish")
        return self._run, [s.as_dict() for s in st]  # the run may continue after finish

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.smol_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """One system of Eq. (4) with kernel K = U V on the current CUDA device.

    U: (M, R) and V: (R, M) float64 arrays (host; copied). lam: shattering rate.
    Options map to the fields of smol_opts (precision 'fp64' | 'fp32conv', ctrl
    'double_halve' | 'formula', norm 'abs' | 'rel', tau0, euler_a, tau_min_rel,
    steady_rtol, fixed_tau, fac_min, fac_max, max_attempts, chunk, log_capacity).
    The workspace is a torch uint8 tensor owned by this object.
    """

    def __init__(self, U, V, lam: float, precision: str = "fp64", stream=None, device=None, **opts):
        torch = _torch()
        U = np.ascontiguousarray(U, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        if U.ndim != 2 or V.ndim != 2 or V.shape != (U.shape[1], U.shape[0]):
            raise ValueError("U must be (M, R) and V (R, M)")
        self.M, self.R = U.shape
        self.lam = float(lam)
        self.device = torch.device(device if device is not None else "cuda")
        self.opts = default_opts()
        self.opts.precision = PRECISIONS[precision]
        for k, v in opts.items():
            if k == "ctrl":
                v = CTRLS[v]
            elif k == "norm":
                v = NORMS[v]
            if not hasattr(self.opts, k):
                raise TypeError(f"unknown option {k!r}")
            setattr(self.opts, k, v)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.opts.stream = ctypes.c_void_p(stream.cuda_stream)
        nbytes = int(_lib.smol_workspace_bytes(self.M, self.R, ctypes.byref(self.opts)))
        if nbytes == 0:
            raise SmolError(EUNSUPPORTED, f"M={self.M}, R={self.R}")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._h = ctypes.c_void_p()
        self._U, self._V = U, V
        _check(_lib.smol_init_system(ctypes.byref(self._h), self.M, self.R, U.ctypes.data, V.ctypes.data,
                                     self.lam, ctypes.byref(self.opts), self._ws_ptr, nbytes), "smol_init_system")

    # -- helpers -------------------------------------------------------------
    def _vec(self, n):
        torch = _torch()
        if not isinstance(n, torch.Tensor):
            n = torch.as_tensor(np.asarray(n, dtype=np.float64))
        n = n.to(device=self.device, dtype=torch.float64).contiguous()
        if n.numel() != self.M:
            raise ValueError(f"state has {n.numel()} entries, expected M={self.M}")
        return n

    @property
    def num_transforms(self) -> int:
        return int(_lib.smol_num_transforms(self._h))

    # -- C interface ------------------------------------------------------------
    def set_sources(self, sources: dict):
        """Point sources {s: P_s} (1-based sizes) of Eq. (3); {} removes them."""
        k = np.ascontiguousarray(list(sources.keys()), dtype=np.int64)
        v = np.ascontiguousarray(list(sources.values()), dtype=np.float64)
        _check(_lib.smol_set_sources(self._h, k.size, k.ctypes.data, v.ctypes.data), "smol_set_sources")

    def set_tau0(self, tau0: float):
        """First step of the next integration (0: the tau0 option); resuming with the
        previous call's stats['tau_next'] continues its step sequence."""
        _check(_lib.smol_set_tau0(self._h, float(tau0)), "smol_set_tau0")

    def rhs(self, n, out=None):
        """S(n) of Eq. (4) (device tensor of M doubles)."""
        torch = _torch()
        n = self._vec(n)
        if out is None:
            out = torch.empty_like(n)
        _check(_lib.smol_rhs(self._h, n.data_ptr(), out.data_ptr()), "smol_rhs")
        return out

    def rhs_terms(self, n):
        """(birth, loss, source): S = birth - loss, plus source at s = 1."""
        torch = _torch()
        n = self._vec(n)
        birth, loss = torch.empty_like(n), torch.empty_like(n)
        src = torch.empty(1, dtype=torch.float64, device=self.device)
        _check(_lib.smol_rhs_terms(self._h, n.data_ptr(), birth.data_ptr(), loss.data_ptr(), src.data_ptr()),
               "smol_rhs_terms")
        return birth, loss, src

    def integrate(self, n0, t0: float, t1: float, tol: float, scheme: str = "rkf45", inplace: bool = False):
        """Integrates from t0 to t1; returns (n(t_end) device tensor, stats dict).
        Negative statuses (errors) are returned in stats, not raised, so that the caller
        can inspect the state reached; SMOL_EINVAL / SMOL_ECUDA raise."""
        n = self._vec(n0)
        if not inplace:
            n = n.clone()
        st = Stats()
        rc = _lib.smol_integrate(self._h, n.data_ptr(), float(t0), float(t1), float(tol), SCHEMES[scheme],
                                 ctypes.byref(st))
        if rc in (EINVAL, ECUDA, ENOSPACE, EUNSUPPORTED):
            raise SmolError(rc, "smol_integrate")
        return n, st.as_dict()

    # asynchronous form: start / advance / finish
    def start(self, n, t0: float, t1: float, tol: float, scheme: str = "rkf45"):
        """Begins an integration of the device tensor n in place (kept referenced until
        finish); returns n."""
        n = self._vec(n)
        self._run = n
        _check(_lib.smol_integrate_start(self._h, n.data_ptr(), float(t0), float(t1), float(tol), SCHEMES[scheme]),
               "smol_integrate_start")
        return n

    def advance(self):
        """Enqueues one captured chunk of attempts; does not synchronise."""
        _check(_lib.smol_integrate_advance(self._h), "smol_integrate_advance")

    def finish(self):
        st = Stats()
        rc = _lib.smol_integrate_finish(self._h, ctypes.byref(st))
        if rc in (EINVAL, ECUDA):
            raise SmolError(rc, "smol_integrate_finish")
        return self._run, st.as_dict()  # the run may continue (advance) after finish

    PROF_KINDS = ("fwd_cols", "rows", "inv_cols", "step", "inv_fwd", "inv_step")

    def profile(self, reps: int = 20):
        """Per-kernel-class average durations (ms) and launch counts over `reps` attempts
        of the current run, each kernel bracketed by CUDA events."""
        ms = np.zeros(len(self.PROF_KINDS))
        cnt = np.zeros(len(self.PROF_KINDS), dtype=np.int64)
        _check(_lib.smol_profile_attempts(self._h, int(reps), ms.ctypes.data, cnt.ctypes.data, len(ms)),
               "smol_profile_attempts")
        return dict(zip(self.PROF_KINDS, ms)), dict(zip(self.PROF_KINDS, cnt.tolist()))

    def get_log(self, cap: int | None = None):
        """Step log of the last integrate: arrays t, tau, err, accepted (oldest first)."""
        cnt = ctypes.c_int64()
        cap = int(cap if cap is not None else self.opts.log_capacity)
        t = np.zeros(cap)
        h = np.zeros(cap)
        e = np.zeros(cap)
        a = np.zeros(cap, dtype=np.int32)
        _check(_lib.smol_get_log(self._h, t.ctypes.data, h.ctypes.data, e.ctypes.data, a.ctypes.data, cap,
                                 ctypes.byref(cnt)), "smol_get_log")
        k = min(cnt.value, cap, max(self.opts.log_capacity, 0))
        return t[:k], h[:k], e[:k], a[:k].astype(bool), cnt.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.smol_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
