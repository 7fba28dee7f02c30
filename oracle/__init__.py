"""FT-GCR(k) oracle: ctypes shim over the plain FP64 C implementation in
``ftgcr_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the CPU-baseline leg of ``bench.py`` may import this module.  The product path
(the CUDA library and its Python binding) never imports it, and this module
imports nothing from the product.

The oracle follows Algorithm 1 of the paper (FT-GCR(k)) step by step; see the
header of ``ftgcr_oracle.c`` for the readings of the printed algorithm and the
2-D latitude-longitude stand-in for the paper's operator (Eq. (1), Section 3).

Parity status per function (what pins it, see ``tests/test_oracle_*.py``):
  geometry / face_coeffs   pinned: total area 4*pi, spherical-harmonic
                           eigenvalues of the Laplacian (closed form).
  apply_L                  pinned: symmetry, definiteness, constant null
                           vector of the flux part, harmonic consistency.
  apply_P / solve_P        pinned: P equals the diagonal-block part of L,
                           P(P^-1 r) = r, dense LAPACK solve.
  dot                      pinned: numpy on the same data.
  splitmix64               pinned: the published SplitMix64 reference outputs
                           for seed 1234567.
  data-loss events         pinned: flip positions and bits against an
                           independent Python restatement; XOR involution.
  flip_bit                 pinned: numpy bit pattern XOR.
  ftgcr                    pinned: dense direct solve, manufactured solution,
                           strictly decreasing norms, exact preconditioner
                           converges in one step with beta = -1, finite
                           termination for k >= N, orthogonality of the
                           L(p) within a cycle, fault-tolerance invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftgcr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libftgcr_oracle.so")
_lock = threading.Lock()
_lib = None

VEC_X, VEC_R, VEC_P, VEC_AP, VEC_E = 0, 1, 2, 3, 4
VEC_NAMES = {"x": VEC_X, "r": VEC_R, "p": VEC_P, "ap": VEC_AP, "e": VEC_E}
PRECOND_LINE, PRECOND_JACOBI, PRECOND_IDENTITY, PRECOND_DENSE = 0, 1, 2, 3
EVENT_ACCEPT, EVENT_FAULT, EVENT_EXIT = 0, 1, 2
MAX_DETECT = 64


class _Fault(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("vec", ctypes.c_int32), ("index", ctypes.c_int64),
                ("bit", ctypes.c_int32)]


class _Problem(ctypes.Structure):
    _fields_ = [("nlon", ctypes.c_int32), ("nlat", ctypes.c_int32), ("mu", ctypes.c_double),
                ("k", ctypes.c_int32), ("tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("precond", ctypes.c_int32), ("D", ctypes.c_void_p), ("dense_pinv", ctypes.c_void_p),
                ("protect", ctypes.c_int32)]


class _Loss(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("rank", ctypes.c_int32), ("nranks", ctypes.c_int32),
                ("count", ctypes.c_int64), ("seed", ctypes.c_uint64), ("nbits", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("cycles", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("faults_injected", ctypes.c_int64), ("faults_detected", ctypes.c_int64),
                ("loss_events", ctypes.c_int64), ("converged", ctypes.c_int32), ("ndetect", ctypes.c_int32),
                ("detect_step", ctypes.c_int64 * MAX_DETECT), ("nrm2_R", ctypes.c_double),
                ("nrm2_0", ctypes.c_double), ("nrm2_final", ctypes.c_double), ("res_true", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no fused multiply-add
    contraction) into ``oracle/_build``; return the library path."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.c_void_p
        L.orc_geometry.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_face_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        for f in (L.orc_apply_L, L.orc_apply_P):
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp]
        L.orc_solve_P.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.orc_dot.argtypes = [ctypes.c_long, dp, dp]
        L.orc_dot.restype = ctypes.c_double
        L.orc_flip_bit.argtypes = [ctypes.c_double, ctypes.c_int]
        L.orc_flip_bit.restype = ctypes.c_double
        L.orc_ftgcr.argtypes = [ctypes.POINTER(_Problem), dp, dp, ctypes.POINTER(_Fault), ctypes.c_int,
                                ctypes.POINTER(_Loss), ctypes.c_int, ctypes.POINTER(_Result), dp, dp, dp, dp]
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_ftgcr.restype = ctypes.c_int
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def geometry(nlon: int, nlat: int):
    """Per-row (cx, cy, area) of the latitude-longitude grid."""
    cx, cy, area = (np.empty(nlat) for _ in range(3))
    lib().orc_geometry(nlon, nlat, _ptr(cx), _ptr(cy), _ptr(area))
    return cx, cy, area


def face_coeffs(D: np.ndarray):
    """(Tx, Ty, area) for the cell-centred coefficient D[nlat, nlon]."""
    D = _f64(D)
    nlat, nlon = D.shape
    Tx, Ty = np.empty_like(D), np.empty_like(D)
    area = np.empty(nlat)
    lib().orc_face_coeffs(nlon, nlat, _ptr(D), _ptr(Tx), _ptr(Ty), _ptr(area))
    return Tx, Ty, area


def apply_L(D: np.ndarray, mu: float, phi: np.ndarray) -> np.ndarray:
    Tx, Ty, area = face_coeffs(D)
    phi = _f64(phi)
    out = np.empty_like(phi)
    nlat, nlon = phi.shape
    lib().orc_apply_L(nlon, nlat, mu, _ptr(Tx), _ptr(Ty), _ptr(area), _ptr(phi), _ptr(out))
    return out


def apply_P(D: np.ndarray, mu: float, phi: np.ndarray) -> np.ndarray:
    Tx, Ty, area = face_coeffs(D)
    phi = _f64(phi)
    out = np.empty_like(phi)
    nlat, nlon = phi.shape
    lib().orc_apply_P(nlon, nlat, mu, _ptr(Tx), _ptr(Ty), _ptr(area), _ptr(phi), _ptr(out))
    return out


def solve_P(D: np.ndarray, mu: float, r: np.ndarray, kind: int = PRECOND_LINE, dense_pinv=None) -> np.ndarray:
    Tx, Ty, area = face_coeffs(D)
    r = _f64(r)
    e = np.empty_like(r)
    nlat, nlon = r.shape
    dp = _f64(dense_pinv) if dense_pinv is not None else None
    lib().orc_solve_P(nlon, nlat, mu, _ptr(Tx), _ptr(Ty), _ptr(area), kind,
                      _ptr(dp) if dp is not None else None, _ptr(r), _ptr(e))
    return e


def dot(a: np.ndarray, b: np.ndarray) -> float:
    a, b = _f64(a).ravel(), _f64(b).ravel()
    return lib().orc_dot(a.size, _ptr(a), _ptr(b))


def flip_bit(v: float, bit: int) -> float:
    return lib().orc_flip_bit(float(v), int(bit))


def dense_matrix(apply, nlat: int, nlon: int) -> np.ndarray:
    """Assemble the N x N matrix of a linear map by applying it to unit vectors
    (tiny grids only)."""
    N = nlat * nlon
    M = np.empty((N, N))
    for c in range(N):
        u = np.zeros(N)
        u[c] = 1.0
        M[:, c] = apply(u.reshape(nlat, nlon)).ravel()
    return M


def splitmix64(seed: int, i: int) -> int:
    """Output i (i >= 1) of SplitMix64 started at state ``seed``."""
    return int(lib().orc_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, i))


def ftgcr(D, R, mu, k, tol, x0=None, faults=(), max_steps=None, precond=PRECOND_LINE, dense_pinv=None,
          trace_lp=False, losses=(), protect=True):
    """Run FT-GCR(k) (Algorithm 1).  ``faults`` is a sequence of
    (step, vec, index, bit) tuples, ``vec`` an int or one of x, r, p, ap, e.
    ``losses`` is a sequence of data-loss events (step, rank, nranks, count,
    seed, nbits) hitting e after the preconditioner (Section 3).
    ``protect=False`` runs plain GCR(k): no fault test, backup or restore.
    Returns a dict with the solution, status, counters and per-step history."""
    D, R = _f64(D), _f64(R)
    nlat, nlon = D.shape
    N = nlat * nlon
    if max_steps is None:
        max_steps = default_max_steps(nlon, nlat)
    x = np.zeros_like(R) if x0 is None else _f64(x0).copy()
    fa = (_Fault * max(1, len(faults)))()
    for q, (st, vec, idx, bit) in enumerate(faults):
        fa[q].step, fa[q].vec, fa[q].index, fa[q].bit = int(st), VEC_NAMES.get(vec, vec), int(idx), int(bit)
    la = (_Loss * max(1, len(losses)))()
    for q, (st, rank, nranks, count, seed, nbits) in enumerate(losses):
        la[q].step, la[q].rank, la[q].nranks = int(st), int(rank), int(nranks)
        la[q].count, la[q].seed, la[q].nbits = int(count), int(seed) & 0xFFFFFFFFFFFFFFFF, int(nbits)
    dpv = _f64(dense_pinv) if dense_pinv is not None else None
    pb = _Problem(nlon, nlat, float(mu), int(k), float(tol), int(max_steps), int(precond), D.ctypes.data,
                  dpv.ctypes.data if dpv is not None else None, 1 if protect else 0)
    res = _Result()
    nrm2 = np.full(max_steps, np.nan)
    ev = np.full(max_steps, -1, dtype=np.int32)
    beta = np.full(max_steps, np.nan)
    lpt = np.empty((max_steps, N)) if trace_lp else None
    st = lib().orc_ftgcr(ctypes.byref(pb), _ptr(R), _ptr(x), fa, len(faults), la, len(losses), ctypes.byref(res),
                         _ptr(nrm2), _ptr(ev), _ptr(beta), _ptr(lpt) if lpt is not None else None)
    if st < 0:
        raise ValueError("oracle rejected the arguments")
    n = res.steps
    out = dict(x=x, status=st, steps=n, cycles=res.cycles, restarts=res.restarts,
               faults_injected=res.faults_injected, faults_detected=res.faults_detected,
               loss_events=res.loss_events, converged=bool(res.converged), detect_steps=[res.detect_step[i] for i in range(res.ndetect)],
               nrm2_R=res.nrm2_R, nrm2_0=res.nrm2_0, nrm2_final=res.nrm2_final, res_true=res.res_true,
               nrm2_hist=nrm2[:n].copy(), events=ev[:n].copy(), beta_hist=beta[:n].copy())
    if trace_lp:
        out["lp_trace"] = lpt[:n].reshape(n, nlat, nlon)
    return out


def default_max_steps(nlon: int, nlat: int) -> int:
    """Executed-step limit used when none is given: 100 * ceil(sqrt(N)) + 100."""
    return 100 * int(np.ceil(np.sqrt(nlon * nlat))) + 100
