"""CPU oracle for the Feldman-Cousins grid fit -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and it never imports the CUDA
library.  The arithmetic lives in ``fc_oracle.c`` (plain C, binary64 fit,
binary32 sampler with correctly rounded operations); this module only builds
it with gcc and marshals numpy arrays through ctypes.

Citations (the method's passages): Eq. 1 (chi2 with the inverse covariance),
Algorithm 2 (residual form), Algorithm 1 (scan with strict "<", dchi2), §2
steps 1-6 (fluctuate, scan, argmin, refit the covariance at q_min, dchi2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

FLUCT_POISSON_SYS = 0
FLUCT_GAUSS = 1
COV_ITERATE = 0
COV_FIXED = 1
COV_IDENTITY = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fc_oracle.c into oracle/_build/liboracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        c_dp, c_fp = P(ctypes.c_double), P(ctypes.c_float)
        c_i32p, c_i64p, c_i8p, c_u32p = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_int8), P(ctypes.c_uint32)
        sig = {
            "oracle_philox4x32_10": (None, [c_u32p, c_u32p, c_u32p]),
            "oracle_u01": (ctypes.c_float, [ctypes.c_uint32]),
            "oracle_logf": (ctypes.c_float, [ctypes.c_float]),
            "oracle_expf": (ctypes.c_float, [ctypes.c_float]),
            "oracle_sincos_turns": (None, [ctypes.c_float, c_fp, c_fp]),
            "oracle_normals": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, c_fp]),
            "oracle_poisson_draws": (None, [ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int, c_i32p]),
            "oracle_poisson_indep": (None, [ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_int, c_i32p]),
            "oracle_cholesky": (ctypes.c_int, [ctypes.c_int, c_dp, c_dp]),
            "oracle_chol_sys": (ctypes.c_int, [ctypes.c_int, c_dp, c_dp, ctypes.c_int, c_dp]),
            "oracle_inv_cov": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_i32p, c_dp, c_dp, c_dp]),
            "oracle_collapse_spectra": (None, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, c_i32p, c_dp, c_dp]),
            "oracle_scan": (None, [ctypes.c_int64, ctypes.c_int, c_dp, c_dp, c_dp, c_dp]),
            "oracle_fake_data": (ctypes.c_int, [c_dp, ctypes.c_int64, ctypes.c_int, c_i32p, ctypes.c_int, c_dp,
                                                c_i64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                c_fp]),
            "oracle_run_points": (ctypes.c_int, [c_dp, ctypes.c_int64, ctypes.c_int, c_i32p, ctypes.c_int, c_dp,
                                                 c_i64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_i64p, c_i8p,
                                                 c_fp]),
            "oracle_run_samples": (ctypes.c_int, [c_dp, ctypes.c_int64, ctypes.c_int, c_i32p, ctypes.c_int, c_dp,
                                                  c_i64p, c_i32p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, c_dp, c_i64p, c_i8p]),
            "oracle_run_data": (ctypes.c_int, [c_dp, ctypes.c_int64, ctypes.c_int, c_i32p, ctypes.c_int, c_dp,
                                               c_i64p, ctypes.c_int, c_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               c_dp, c_i64p, c_i8p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# -- elementary pieces ------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def u01(x: int) -> float:
    return float(_load().oracle_u01(ctypes.c_uint32(x)))


def logf(x) -> np.ndarray:
    lib = _load()
    x = np.atleast_1d(np.asarray(x, np.float32))
    return np.array([lib.oracle_logf(float(v)) for v in x], np.float32)


def expf(x) -> np.ndarray:
    lib = _load()
    x = np.atleast_1d(np.asarray(x, np.float32))
    return np.array([lib.oracle_expf(float(v)) for v in x], np.float32)


def sincos_turns(u) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    u = np.atleast_1d(np.asarray(u, np.float32))
    s = np.empty_like(u)
    c = np.empty_like(u)
    a, b = ctypes.c_float(), ctypes.c_float()
    for i, v in enumerate(u):
        lib.oracle_sincos_turns(float(v), ctypes.byref(a), ctypes.byref(b))
        s[i], c[i] = a.value, b.value
    return s, c


def normals(seed: int, p: int, u: int, n: int) -> np.ndarray:
    z = np.empty(n, np.float32)
    _load().oracle_normals(seed, p, u, n, _ptr(z, ctypes.c_float))
    return z


def poisson_draws(lam: float, n: int, seed: int = 0, p: int = 0, u: int = 0, bin: int = 0) -> np.ndarray:
    """n consecutive draws from one stream (seed, p, u, bin)."""
    out = np.empty(n, np.int32)
    _load().oracle_poisson_draws(float(lam), seed, p, u, bin, n, _ptr(out, ctypes.c_int32))
    return out


def poisson_indep(lam: float, n: int, seed: int = 0, p: int = 0, bin: int = 0) -> np.ndarray:
    """n first draws of n universes' streams (u = 0..n-1), as the fake-data path uses them."""
    out = np.empty(n, np.int32)
    _load().oracle_poisson_indep(float(lam), seed, p, bin, n, _ptr(out, ctypes.c_int32))
    return out


# -- linear algebra ---------------------------------------------------------

def cholesky(M) -> np.ndarray:
    M = _c(M, np.float64)
    n = M.shape[0]
    L = np.zeros_like(M)
    if _load().oracle_cholesky(n, _ptr(M, ctypes.c_double), _ptr(L, ctypes.c_double)) != 0:
        raise np.linalg.LinAlgError("not SPD")
    return L


def chol_sys(s, F, gauss: bool = False) -> np.ndarray:
    s = _c(s, np.float64)
    F = _c(F, np.float64)
    n = s.shape[0]
    L = np.zeros((n, n))
    if _load().oracle_chol_sys(n, _ptr(s, ctypes.c_double), _ptr(F, ctypes.c_double), int(gauss),
                               _ptr(L, ctypes.c_double)) != 0:
        raise np.linalg.LinAlgError("not SPD")
    return L


def inv_cov(s, F, collapse=None, n_fit=None) -> np.ndarray:
    s = _c(s, np.float64)
    F = _c(F, np.float64)
    nf = s.shape[0]
    coll = None if collapse is None else _c(collapse, np.int32)
    nfit = nf if n_fit is None else int(n_fit)
    A = np.zeros((nfit, nfit))
    if _load().oracle_inv_cov(nf, nfit, _ptr(coll, ctypes.c_int32), _ptr(s, ctypes.c_double),
                              _ptr(F, ctypes.c_double), _ptr(A, ctypes.c_double)) != 0:
        raise np.linalg.LinAlgError("not SPD")
    return A


def collapse_spectra(S, collapse=None, n_fit=None) -> np.ndarray:
    S = _c(S, np.float64)
    G, nf = S.shape
    nfit = nf if n_fit is None else int(n_fit)
    coll = None if collapse is None else _c(collapse, np.int32)
    out = np.zeros((G, nfit))
    _load().oracle_collapse_spectra(G, nf, nfit, _ptr(coll, ctypes.c_int32), _ptr(S, ctypes.c_double),
                                    _ptr(out, ctypes.c_double))
    return out


def scan(Sfit, A, d) -> np.ndarray:
    Sfit = _c(Sfit, np.float64)
    A = _c(A, np.float64)
    d = _c(d, np.float64)
    G, nfit = Sfit.shape
    out = np.empty(G)
    _load().oracle_scan(G, nfit, _ptr(Sfit, ctypes.c_double), _ptr(A, ctypes.c_double), _ptr(d, ctypes.c_double),
                        _ptr(out, ctypes.c_double))
    return out


# -- the method -------------------------------------------------------------

def fake_data(S, F, points, seed: int, U: int, collapse=None, n_fit=None, fluct: int = FLUCT_POISSON_SYS):
    """Fit-space fake data [P][U][n_fit] (float32; integer counts in the Poisson mode)."""
    S = _c(S, np.float64)
    F = _c(F, np.float64)
    G, nf = S.shape
    nfit = nf if n_fit is None else int(n_fit)
    pts = _c(points, np.int64)
    coll = None if collapse is None else _c(collapse, np.int32)
    out = np.zeros((len(pts), U, nfit), np.float32)
    rc = _load().oracle_fake_data(_ptr(S, ctypes.c_double), G, nf, _ptr(coll, ctypes.c_int32), nfit,
                                  _ptr(F, ctypes.c_double), _ptr(pts, ctypes.c_int64), len(pts), seed, U, fluct,
                                  _ptr(out, ctypes.c_float))
    if rc != 0:
        raise np.linalg.LinAlgError("systematic covariance not SPD")
    return out


def run_points(S, F, points, seed: int, U: int, collapse=None, n_fit=None, max_iter: int = 5,
               fluct: int = FLUCT_POISSON_SYS, cov: int = COV_ITERATE, nthreads: int | None = None,
               want_fake: bool = False):
    """dchi2 [P][U], bestfit [P][U] (int64), nscans [P][U] (int8) and optionally the fake data."""
    S = _c(S, np.float64)
    F = _c(F, np.float64)
    G, nf = S.shape
    nfit = nf if n_fit is None else int(n_fit)
    pts = _c(points, np.int64)
    P = len(pts)
    coll = None if collapse is None else _c(collapse, np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    dchi2 = np.zeros((P, U))
    best = np.zeros((P, U), np.int64)
    ns = np.zeros((P, U), np.int8)
    fk = np.zeros((P, U, nfit), np.float32) if want_fake else None
    rc = _load().oracle_run_points(_ptr(S, ctypes.c_double), G, nf, _ptr(coll, ctypes.c_int32), nfit,
                                   _ptr(F, ctypes.c_double), _ptr(pts, ctypes.c_int64), P, seed, U, max_iter,
                                   fluct, cov, nthreads, _ptr(dchi2, ctypes.c_double), _ptr(best, ctypes.c_int64),
                                   _ptr(ns, ctypes.c_int8), _ptr(fk, ctypes.c_float))
    if rc == -1:
        raise ValueError("bad argument")
    if rc != 0:
        raise np.linalg.LinAlgError("covariance not SPD")
    if want_fake:
        return dchi2, best, ns, fk
    return dchi2, best, ns


def run_samples(S, F, points, universes, seed: int, collapse=None, n_fit=None, max_iter: int = 5,
                fluct: int = FLUCT_POISSON_SYS, cov: int = COV_ITERATE, nthreads: int | None = None):
    """dchi2, bestfit, nscans of sampled universes: entry i is universe universes[i] of true point points[i]."""
    S = _c(S, np.float64)
    F = _c(F, np.float64)
    G, nf = S.shape
    nfit = nf if n_fit is None else int(n_fit)
    pts = _c(points, np.int64)
    us = _c(universes, np.int32)
    n = len(pts)
    if len(us) != n:
        raise ValueError("points and universes differ in length")
    coll = None if collapse is None else _c(collapse, np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    dchi2 = np.zeros(n)
    best = np.zeros(n, np.int64)
    ns = np.zeros(n, np.int8)
    rc = _load().oracle_run_samples(_ptr(S, ctypes.c_double), G, nf, _ptr(coll, ctypes.c_int32), nfit,
                                    _ptr(F, ctypes.c_double), _ptr(pts, ctypes.c_int64), _ptr(us, ctypes.c_int32), n,
                                    seed, max_iter, fluct, cov, nthreads, _ptr(dchi2, ctypes.c_double),
                                    _ptr(best, ctypes.c_int64), _ptr(ns, ctypes.c_int8))
    if rc == -1:
        raise ValueError("bad argument")
    if rc != 0:
        raise np.linalg.LinAlgError("covariance not SPD")
    return dchi2, best, ns


def run_data(S, F, points, data, collapse=None, n_fit=None, max_iter: int = 5, cov: int = COV_ITERATE,
             nthreads: int | None = None):
    """The observed data's dchi2, bestfit, nscans at each grid point (the universe procedure on given data)."""
    S = _c(S, np.float64)
    F = _c(F, np.float64)
    G, nf = S.shape
    nfit = nf if n_fit is None else int(n_fit)
    pts = _c(points, np.int64)
    dv = _c(data, np.float32)
    if dv.shape != (nfit,):
        raise ValueError("data must have N_fit entries")
    coll = None if collapse is None else _c(collapse, np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    n = len(pts)
    dchi2 = np.zeros(n)
    best = np.zeros(n, np.int64)
    ns = np.zeros(n, np.int8)
    rc = _load().oracle_run_data(_ptr(S, ctypes.c_double), G, nf, _ptr(coll, ctypes.c_int32), nfit,
                                 _ptr(F, ctypes.c_double), _ptr(pts, ctypes.c_int64), n, _ptr(dv, ctypes.c_float),
                                 max_iter, cov, nthreads, _ptr(dchi2, ctypes.c_double), _ptr(best, ctypes.c_int64),
                                 _ptr(ns, ctypes.c_int8))
    if rc == -1:
        raise ValueError("bad argument")
    if rc != 0:
        raise np.linalg.LinAlgError("covariance not SPD")
    return dchi2, best, ns


def run_workload(w, U: int | None = None, points=None, nthreads: int | None = None, seed: int | None = None, **kw):
    """Convenience: oracle.run_points on a workloads.Workload."""
    pts = w.points if points is None else points
    return run_points(w.S, w.F, pts, w.seed if seed is None else seed, w.U if U is None else U,
                      collapse=w.collapse, n_fit=w.n_fit, max_iter=w.max_iter, nthreads=nthreads, **kw)
