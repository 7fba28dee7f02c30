"""Python binding of libftgcr, the GB300 FT-GCR(k) solver (C ABI in
include/ftgcr.h).  Argument marshalling only: every step of the solve runs in
the library's CUDA kernels.  There is no fallback: if the library cannot be
built or loaded, every call raises.

Arrays are numpy (host) or torch (host or CUDA) FP64 arrays of shape
[nlat, nlon]; the library detects where they live.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libftgcr.so")
SOURCES = ["ftgcr.cu", "ftgcr_k4.cu", "ftgcr_k8.cu", "ftgcr_k16.cu", "ftgcr_k4s.cu", "ftgcr_k8s.cu", "ftgcr_k16s.cu",
           "ftgcr_k4t.cu", "ftgcr_k8t.cu", "ftgcr_k16t.cu",
           "ftgcr_k4w.cu", "ftgcr_k8w.cu", "ftgcr_k16w.cu", "ftgcr_server.cu", "ftgcr_tune.cu", "ftgcr_probe.cu"]
HEADERS = ["ftgcr_device.cuh", "ftgcr_phases.cuh", "ftgcr_stream.cuh", "ftgcr_instances.h", "ftgcr_serve.h"]
# --fmad=false: device multiply-adds are fused only where the code says fma();
# -ffp-contract=off: the same for the host-side geometry (GCC contracts by
# default on aarch64)
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "--fmad=false",
              "-Xcompiler", "-fPIC,-ffp-contract=off"]

FP64, MIXED = 0, 1
PRECOND = {"line": 0, "jacobi": 1, "identity": 2}
VEC = {"x": 0, "r": 1, "p": 2, "ap": 3, "e": 4}
MAX_FAULTS, MAX_K, MAX_DETECT, MAX_LOSSES = 64, 16, 16, 16
FLAG_UNPROTECTED, FLAG_SPLIT_ROUNDS, FLAG_FUSED_ROUNDS, FLAG_STREAMED_ROUNDS, FLAG_ORACLE_ORDER = 1, 2, 4, 8, 16
FLAG_ZERO_GUESS = 32

OK, NOT_CONVERGED, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUDGET, ERR_STATE = 0, 1, -1, -2, -3, -4, -5, -6
PENDING = 2

# every symbol include/ftgcr.h declares
EXPORTS = ["ftgcr_create", "ftgcr_solve", "ftgcr_solve_async", "ftgcr_stats", "ftgcr_solve_batch",
           "ftgcr_apply_operator", "ftgcr_apply_precond", "ftgcr_footprint", "ftgcr_destroy", "ftgcr_error_string",
           "ftgcr_solve_noalloc", "ftgcr_set_coeffs", "ftgcr_server_create", "ftgcr_server_submit",
           "ftgcr_server_poll", "ftgcr_server_wait", "ftgcr_server_next", "ftgcr_server_info",
           "ftgcr_server_destroy", "ftgcr_server_set_max_points", "ftgcr_tune", "ftgcr_fp64_fma_rate",
           "ftgcr_solve_host_async"]
NOALLOC_MAX_POINTS, NOALLOC_MAX_K = 16384, 4
TUNE_MAX_CONCURRENCY = 256

_lock = threading.Lock()
_lib = None


class Grid(ctypes.Structure):
    _fields_ = [("nlon", ctypes.c_int32), ("nlat", ctypes.c_int32), ("mu", ctypes.c_double),
                ("precision", ctypes.c_int32), ("precond", ctypes.c_int32), ("max_steps", ctypes.c_int64),
                ("tiles", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class Coeffs(ctypes.Structure):
    _fields_ = [("D", ctypes.c_void_p), ("key", ctypes.c_uint64)]


class Fault(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("vec", ctypes.c_int32), ("index", ctypes.c_int64), ("bit", ctypes.c_int32)]


class Loss(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("rank", ctypes.c_int32), ("nranks", ctypes.c_int32),
                ("count", ctypes.c_int64), ("seed", ctypes.c_uint64)]


class FaultPlan(ctypes.Structure):
    _fields_ = [("faults", ctypes.POINTER(Fault)), ("n", ctypes.c_int32), ("losses", ctypes.POINTER(Loss)),
                ("nlosses", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("cycles", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("faults_injected", ctypes.c_int64), ("faults_detected", ctypes.c_int64), ("outer", ctypes.c_int64),
                ("ndetect", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("detect_step", ctypes.c_int64 * MAX_DETECT), ("detect_ratio", ctypes.c_double * MAX_DETECT),
                ("res0", ctypes.c_double), ("res_final_rec", ctypes.c_double), ("res_final_true", ctypes.c_double),
                ("norm_R", ctypes.c_double), ("bytes_resident", ctypes.c_int64), ("bytes_backup", ctypes.c_int64),
                ("tiles", ctypes.c_int32), ("status", ctypes.c_int32), ("loss_events", ctypes.c_int64),
                ("split_rounds", ctypes.c_int32), ("global_factors", ctypes.c_int32)]


class ServerInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "queued", "running", "epochs", "handles",
                                              "bytes_in_use", "budget_bytes")]


class Tuning(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int32), ("flags", ctypes.c_int32), ("ms", ctypes.c_double),
                ("default_tiles", ctypes.c_int32), ("default_ms", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("cached", ctypes.c_int32)]


class FTGCRError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = lib().ftgcr_error_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")
        self.status = status


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(_INCLUDE, "ftgcr.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libftgcr.so for sm_103a in-tree (paper_2103_07210_gb300/_build)."""
    with _lock:
        if not force and not _stale():
            return LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tag = ".%d" % os.getpid()
        objs, procs = [], []
        for src in SOURCES:  # translation units compile in parallel
            obj = os.path.join(_BUILD, src.replace(".cu", tag + ".o"))
            cmd = ["nvcc"] + NVCC_FLAGS + ["-c", "-o", obj, os.path.join(_CSRC, src)]
            if verbose:
                print(" ".join(cmd))
            procs.append((subprocess.Popen(cmd, cwd=_CSRC), cmd))
            objs.append(obj)
        for pr, cmd in procs:
            if pr.wait() != 0:
                raise subprocess.CalledProcessError(pr.returncode, cmd)
        tmp = LIB_PATH + tag + ".tmp"
        subprocess.check_call(["nvcc", "-shared", "-o", tmp] + objs, cwd=_CSRC)
        os.replace(tmp, LIB_PATH)
        for o in objs:
            os.remove(o)
        return LIB_PATH


def lib():
    """Load libftgcr.so (building it first if needed); raises if that fails."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or _stale():
            build()
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.ftgcr_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Coeffs), i32, dbl, ctypes.POINTER(vp)]
        L.ftgcr_solve.argtypes = [vp, vp, vp, ctypes.POINTER(FaultPlan), vp]
        L.ftgcr_solve_async.argtypes = [vp, vp, vp, ctypes.POINTER(FaultPlan), vp]
        L.ftgcr_solve_host_async.argtypes = [vp, vp, vp, ctypes.POINTER(FaultPlan), vp]
        L.ftgcr_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.ftgcr_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(ctypes.POINTER(FaultPlan)), i32, vp]
        L.ftgcr_apply_operator.argtypes = [vp, vp, vp, vp]
        L.ftgcr_apply_precond.argtypes = [vp, vp, vp, vp]
        L.ftgcr_footprint.argtypes = [ctypes.POINTER(Grid), i32]
        L.ftgcr_footprint.restype = i64
        L.ftgcr_destroy.argtypes = [vp]
        L.ftgcr_destroy.restype = None
        L.ftgcr_error_string.argtypes = [ctypes.c_int]
        L.ftgcr_error_string.restype = ctypes.c_char_p
        L.ftgcr_solve_noalloc.argtypes = [ctypes.POINTER(Grid), vp, i32, dbl, vp, vp, ctypes.POINTER(Stats), vp]
        L.ftgcr_set_coeffs.argtypes = [vp, ctypes.POINTER(Coeffs), vp]
        L.ftgcr_tune.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Coeffs), i32, dbl, i32, ctypes.POINTER(Tuning)]
        L.ftgcr_server_create.argtypes = [i64, i32, i32, ctypes.POINTER(vp)]
        L.ftgcr_server_submit.argtypes = [vp, ctypes.POINTER(Grid), ctypes.POINTER(Coeffs), i32, dbl, vp, vp,
                                          ctypes.POINTER(FaultPlan), ctypes.POINTER(i64)]
        L.ftgcr_server_poll.argtypes = [vp, i64, ctypes.POINTER(Stats)]
        L.ftgcr_server_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(Stats)]
        L.ftgcr_server_next.argtypes = [vp, dbl, ctypes.POINTER(i64), ctypes.POINTER(Stats)]
        L.ftgcr_server_info.argtypes = [vp, ctypes.POINTER(ServerInfo)]
        L.ftgcr_server_destroy.argtypes = [vp]
        L.ftgcr_server_set_max_points.argtypes = [vp, i64]
        L.ftgcr_fp64_fma_rate.argtypes = [i32, ctypes.POINTER(dbl), vp]
        for f in EXPORTS:
            if not hasattr(L, f):
                raise RuntimeError(f"libftgcr.so does not export {f}")
        _lib = L
    return _lib


def _ptr(a):
    """(pointer, keep-alive) of a contiguous FP64 numpy array or torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float64 numpy array")
        return a.ctypes.data, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 torch tensor")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def _plan(faults, losses=()):
    """(FaultPlan, keep-alive) of single flips (step, vec, index, bit) and
    data-loss events (step, rank, nranks, count, seed)."""
    if not faults and not losses:
        return None, None
    if len(faults) > MAX_FAULTS or len(losses) > MAX_LOSSES:
        raise ValueError("too many faults")
    arr = (Fault * max(1, len(faults)))()
    for q, (step, vec, idx, bit) in enumerate(faults):
        arr[q].step, arr[q].vec, arr[q].index, arr[q].bit = int(step), VEC.get(vec, vec), int(idx), int(bit)
    larr = (Loss * max(1, len(losses)))()
    for q, (step, rank, nranks, count, seed) in enumerate(losses):
        larr[q].step, larr[q].rank, larr[q].nranks = int(step), int(rank), int(nranks)
        larr[q].count, larr[q].seed = int(count), int(seed) & 0xFFFFFFFFFFFFFFFF
    plan = FaultPlan(ctypes.cast(arr, ctypes.POINTER(Fault)), len(faults), ctypes.cast(larr, ctypes.POINTER(Loss)),
                     len(losses))
    return plan, (arr, larr)


ROUNDS = {"auto": 0, "split": FLAG_SPLIT_ROUNDS, "fused": FLAG_FUSED_ROUNDS, "streamed": FLAG_STREAMED_ROUNDS}


def _grid(nlon, nlat, mu, precision, precond, max_steps, tiles, inner_tol, max_outer, protect=True, rounds="auto",
          oracle_order=False, zero_guess=False):
    prec = {"fp64": FP64, "mixed": MIXED}.get(precision, precision)
    pc = PRECOND.get(precond, precond)
    flags = (0 if protect else FLAG_UNPROTECTED) | ROUNDS[rounds] | (FLAG_ORACLE_ORDER if oracle_order else 0)
    flags |= FLAG_ZERO_GUESS if zero_guess else 0
    return Grid(int(nlon), int(nlat), float(mu), int(prec), int(pc), int(max_steps), int(tiles), float(inner_tol),
                int(max_outer), flags)


def footprint(nlon, nlat, k=4, precision="fp64", precond="line", tiles=0) -> int:
    g = _grid(nlon, nlat, 1.0, precision, precond, 0, tiles, 0.0, 0)
    return int(lib().ftgcr_footprint(ctypes.byref(g), int(k)))


class Solver:
    """One FT-GCR(k) problem resident on the GPU (ftgcr_create)."""

    def __init__(self, D, mu, k=4, tol=1e-10, precision="fp64", precond="line", max_steps=0, tiles=0,
                 inner_tol=0.0, max_outer=0, protect=True, rounds="auto", oracle_order=False, zero_guess=False):
        """protect=False: plain GCR(k), the paper's unprotected baseline (no
        fault test, no restore).  rounds: "auto", "split", "fused" or
        "streamed" (FTGCR_FLAG_SPLIT_ROUNDS / FTGCR_FLAG_FUSED_ROUNDS /
        FTGCR_FLAG_STREAMED_ROUNDS).  oracle_order (FP64):
        FTGCR_FLAG_ORACLE_ORDER, the oracle's compensated inner products and
        serial row solves.  zero_guess: every solve
        starts from x = 0 and x is output only (FTGCR_FLAG_ZERO_GUESS)."""
        L = lib()
        nlat, nlon = D.shape
        self.nlon, self.nlat, self.k, self.tol = int(nlon), int(nlat), int(k), float(tol)
        self.precision = precision
        g = _grid(nlon, nlat, mu, precision, precond, max_steps, tiles, inner_tol, max_outer, protect, rounds,
                  oracle_order, zero_guess)
        dp, keep = _ptr(D)
        c = Coeffs(dp, 0)
        h = ctypes.c_void_p()
        st = L.ftgcr_create(ctypes.byref(g), ctypes.byref(c), int(k), float(tol), ctypes.byref(h))
        del keep
        if st != OK:
            raise FTGCRError(st, "ftgcr_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ftgcr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, rhs, x, faults=(), stream=None, losses=()) -> int:
        """Blocking solve; x holds the initial guess on entry and the solution
        on exit.  faults: single flips (step, vec, index, bit); losses:
        data-loss events (step, rank, nranks, count, seed).  Returns OK or
        NOT_CONVERGED, raises on errors."""
        rp, rk = _ptr(rhs)
        xp, xk = _ptr(x)
        plan, keep = _plan(faults, losses)
        st = lib().ftgcr_solve(self.h, rp, xp, ctypes.byref(plan) if plan else None, _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_solve")
        return st

    def solve_async(self, rhs, x, faults=(), stream=None, losses=()) -> None:
        rp, rk = _ptr(rhs)
        xp, xk = _ptr(x)
        plan, keep = _plan(faults, losses)
        st = lib().ftgcr_solve_async(self.h, rp, xp, ctypes.byref(plan) if plan else None, _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_solve_async")

    def solve_host_async(self, rhs, x, faults=(), stream=None, losses=()) -> None:
        """Enqueue a solve whose rhs and x may be host arrays (pinned for the
        copies to overlap other work): staging copies, finiteness check,
        solve and the copy back into x, all on `stream`, without waiting.
        rhs and x must stay alive until the stream has passed the solve;
        stats()["status"] then gives its status."""
        rp, rk = _ptr(rhs)
        xp, xk = _ptr(x)
        plan, keep = _plan(faults, losses)
        st = lib().ftgcr_solve_host_async(self.h, rp, xp, ctypes.byref(plan) if plan else None, _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_solve_host_async")

    def stats(self) -> dict:
        s = Stats()
        st = lib().ftgcr_stats(self.h, ctypes.byref(s))
        if st < 0:
            raise FTGCRError(st, "ftgcr_stats")
        n = s.ndetect
        return dict(steps=s.steps, cycles=s.cycles, restarts=s.restarts, faults_injected=s.faults_injected,
                    faults_detected=s.faults_detected, outer=s.outer, converged=bool(s.converged),
                    detect_steps=[s.detect_step[i] for i in range(n)],
                    detect_ratio=[s.detect_ratio[i] for i in range(n)], res0=s.res0, res_final_rec=s.res_final_rec,
                    res_final_true=s.res_final_true, norm_R=s.norm_R, bytes_resident=s.bytes_resident,
                    bytes_backup=s.bytes_backup, tiles=s.tiles, status=s.status, loss_events=s.loss_events,
                    split_rounds=s.split_rounds == 1, streamed_rounds=s.split_rounds == 2,
                    global_factors=bool(s.global_factors))

    def apply_operator(self, inp, out, stream=None):
        ip, ik = _ptr(inp)
        op, ok = _ptr(out)
        st = lib().ftgcr_apply_operator(self.h, ip, op, _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_apply_operator")

    def apply_precond(self, inp, out, stream=None):
        ip, ik = _ptr(inp)
        op, ok = _ptr(out)
        st = lib().ftgcr_apply_precond(self.h, ip, op, _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_apply_precond")

    def set_coeffs(self, D, stream=None):
        """Rebuild the operator and preconditioner from a new D (same grid)."""
        dp, keep = _ptr(D)
        c = Coeffs(dp, 0)
        st = lib().ftgcr_set_coeffs(self.h, ctypes.byref(c), _stream_ptr(stream))
        if st < 0:
            raise FTGCRError(st, "ftgcr_set_coeffs")


def _stats_dict(s: Stats) -> dict:
    n = s.ndetect
    return dict(steps=s.steps, cycles=s.cycles, restarts=s.restarts, faults_injected=s.faults_injected,
                faults_detected=s.faults_detected, outer=s.outer, converged=bool(s.converged),
                detect_steps=[s.detect_step[i] for i in range(n)], detect_ratio=[s.detect_ratio[i] for i in range(n)],
                res0=s.res0, res_final_rec=s.res_final_rec, res_final_true=s.res_final_true, norm_R=s.norm_R,
                bytes_resident=s.bytes_resident, bytes_backup=s.bytes_backup, tiles=s.tiles, status=s.status,
                loss_events=s.loss_events, split_rounds=s.split_rounds == 1, streamed_rounds=s.split_rounds == 2,
                global_factors=bool(s.global_factors))


def tune(D, mu, k=4, tol=1e-10, precision="mixed", precond="line", concurrency=1, max_steps=0, inner_tol=0.0,
         max_outer=0, protect=True, oracle_order=False, zero_guess=False) -> dict:
    """Tile autotuner (ftgcr_tune): the fastest row-band count and round
    layout for `concurrency` solves of this shape in one launch, by timing.
    Returns dict(tiles, rounds, ms, default_tiles, default_ms, candidates,
    cached); pass tiles= and rounds= to Solver (or Server.submit)."""
    nlat, nlon = D.shape
    g = _grid(nlon, nlat, mu, precision, precond, max_steps, 0, inner_tol, max_outer, protect,
              oracle_order=oracle_order, zero_guess=zero_guess)
    dp, keep = _ptr(D)
    t = Tuning()
    st = lib().ftgcr_tune(ctypes.byref(g), ctypes.byref(Coeffs(dp, 0)), int(k), float(tol), int(concurrency),
                          ctypes.byref(t))
    del keep
    if st != OK:
        raise FTGCRError(st, "ftgcr_tune")
    rounds = ("split" if t.flags & FLAG_SPLIT_ROUNDS else "fused" if t.flags & FLAG_FUSED_ROUNDS else
              "streamed" if t.flags & FLAG_STREAMED_ROUNDS else "auto")
    return dict(tiles=t.tiles, rounds=rounds, ms=t.ms, default_tiles=t.default_tiles, default_ms=t.default_ms,
                candidates=t.candidates, cached=bool(t.cached))


def solve_noalloc(D, mu, rhs, x, k=4, tol=1e-10, max_steps=0, tiles=0, stream=None):
    """FP64 solve without any device allocation (ftgcr_solve_noalloc): for
    callers that cannot allocate device memory when they solve.  D, rhs, x:
    CUDA float64 tensors; x holds the initial guess and receives the solution.
    Returns (status, stats)."""
    nlat, nlon = D.shape
    g = _grid(nlon, nlat, mu, "fp64", "line", max_steps, tiles, 0.0, 0)
    dp, dk = _ptr(D)
    rp, rk = _ptr(rhs)
    xp, xk = _ptr(x)
    s = Stats()
    st = lib().ftgcr_solve_noalloc(ctypes.byref(g), dp, int(k), float(tol), rp, xp, ctypes.byref(s),
                                   _stream_ptr(stream))
    if st < 0:
        raise FTGCRError(st, "ftgcr_solve_noalloc")
    return st, _stats_dict(s)


def fp64_fma_rate(iters=4096, stream=None) -> float:
    """The device's measured FP64 fused multiply-add rate in TFLOP/s
    (ftgcr_fp64_fma_rate): the ceiling of the FP64 path's arithmetic."""
    t = ctypes.c_double(0.0)
    st = lib().ftgcr_fp64_fma_rate(int(iters), ctypes.byref(t), _stream_ptr(stream))
    if st < 0:
        raise FTGCRError(st, "ftgcr_fp64_fma_rate")
    return t.value


def solve_batch(solvers, rhs, xs, faults=None, stream=None, losses=None) -> None:
    """Enqueue all solves in one persistent launch (ftgcr_solve_batch)."""
    n = len(solvers)
    H = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    keep = []
    Rp = (ctypes.c_void_p * n)()
    Xp = (ctypes.c_void_p * n)()
    for i in range(n):
        p, k = _ptr(rhs[i])
        Rp[i] = p
        keep.append(k)
        p, k = _ptr(xs[i])
        Xp[i] = p
        keep.append(k)
    P = (ctypes.POINTER(FaultPlan) * n)()
    for i in range(n):
        f = faults[i] if faults else ()
        lo = losses[i] if losses else ()
        plan, arr = _plan(f, lo)
        if plan is not None:
            keep += [plan, arr]
            P[i] = ctypes.pointer(plan)
    st = lib().ftgcr_solve_batch(H, Rp, Xp, P, n, _stream_ptr(stream))
    if st < 0:
        raise FTGCRError(st, "ftgcr_solve_batch")


class Server:
    """Continuous batching of independent solves (ftgcr_server_*): submit
    returns a ticket at once; poll / wait return (status, stats) once the
    solve has finished.  The arrays passed to submit are kept alive here until
    their result has been taken."""

    def __init__(self, budget_bytes=0, max_slots=64, epoch_rounds=48):
        srv = ctypes.c_void_p()
        st = lib().ftgcr_server_create(int(budget_bytes), int(max_slots), int(epoch_rounds), ctypes.byref(srv))
        if st != OK:
            raise FTGCRError(st, "ftgcr_server_create")
        self.srv = srv
        self._keep = {}

    def submit(self, D, mu, rhs, x, k=4, tol=1e-10, precision="fp64", precond="line", faults=(), max_steps=0,
               tiles=0, inner_tol=0.0, max_outer=0, losses=(), protect=True, coeff_key=0, rounds="auto",
               oracle_order=False, zero_guess=False) -> int:
        """coeff_key: 0, or an identity of D's contents; the same (D, key) pair
        lets a pooled handle already set up from it skip the set-up."""
        nlat, nlon = D.shape
        g = _grid(nlon, nlat, mu, precision, precond, max_steps, tiles, inner_tol, max_outer, protect, rounds,
                  oracle_order, zero_guess)
        dp, dk = _ptr(D)
        rp, rk = _ptr(rhs)
        xp, xk = _ptr(x)
        plan, arr = _plan(faults, losses)
        t = ctypes.c_int64()
        st = lib().ftgcr_server_submit(self.srv, ctypes.byref(g), ctypes.byref(Coeffs(dp, int(coeff_key))), int(k), float(tol), rp,
                                       xp, ctypes.byref(plan) if plan else None, ctypes.byref(t))
        if st < 0:
            raise FTGCRError(st, "ftgcr_server_submit")
        self._keep[t.value] = (dk, rk, xk)
        return t.value

    def _result(self, ticket, st, s):
        if st == PENDING:
            return None
        self._keep.pop(ticket, None)
        return st, _stats_dict(s)

    def _check(self, ticket):
        if ticket not in self._keep:
            raise FTGCRError(ERR_ARG, f"unknown or already collected ticket {ticket}")

    def poll(self, ticket):
        """None while running, else (status, stats); the status is that of
        ftgcr_solve (OK, NOT_CONVERGED or a negative error)."""
        self._check(ticket)
        s = Stats()
        return self._result(ticket, lib().ftgcr_server_poll(self.srv, int(ticket), ctypes.byref(s)), s)

    def wait(self, ticket, timeout=None):
        """Block until done (or timeout seconds: None on timeout)."""
        self._check(ticket)
        s = Stats()
        st = lib().ftgcr_server_wait(self.srv, int(ticket), -1.0 if timeout is None else float(timeout),
                                     ctypes.byref(s))
        return self._result(ticket, st, s)

    def next(self, timeout=None):
        """The earliest-finished request not yet collected: (ticket, status,
        stats), or None if none finishes within timeout seconds."""
        s = Stats()
        t = ctypes.c_int64()
        st = lib().ftgcr_server_next(self.srv, -1.0 if timeout is None else float(timeout), ctypes.byref(t),
                                     ctypes.byref(s))
        if st == PENDING:
            return None
        if st == ERR_STATE and not self._keep:
            raise FTGCRError(st, "no request outstanding")
        self._keep.pop(t.value, None)
        return t.value, st, _stats_dict(s)

    def set_max_points(self, max_points: int):
        """Admission limit on the grid points running at once per precision
        (0: none); see ftgcr_server_set_max_points."""
        st = lib().ftgcr_server_set_max_points(self.srv, int(max_points))
        if st != OK:
            raise FTGCRError(st, "ftgcr_server_set_max_points")

    def info(self) -> dict:
        i = ServerInfo()
        st = lib().ftgcr_server_info(self.srv, ctypes.byref(i))
        if st < 0:
            raise FTGCRError(st, "ftgcr_server_info")
        return {n: getattr(i, n) for n, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "srv", None):
            lib().ftgcr_server_destroy(self.srv)
            self.srv = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
