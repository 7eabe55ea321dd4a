"""Thin ctypes binding of libfc.so (include/fc.h): same names, argument marshalling only.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); their data
pointers go straight through the C ABI.  Every step of the computation runs in
the library's CUDA kernels; if the library cannot be loaded this module raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build_lib

FC_OK, FC_PENDING = 0, 1
FC_ERR_ARG, FC_ERR_NOT_SPD, FC_ERR_BUDGET, FC_ERR_CUDA = -1, -2, -3, -4
FC_ERR_TIMEOUT, FC_ERR_CANCELLED, FC_ERR_NOT_FOUND, FC_ERR_STATE = -5, -6, -7, -8
FC_PREC_FP64, FC_PREC_MIXED = 0, 1
FC_FLUCT_POISSON_SYS, FC_FLUCT_GAUSS = 0, 1
FC_COV_ITERATE, FC_COV_FIXED, FC_COV_IDENTITY = 0, 1, 2
FC_QVEC_AUTO, FC_QVEC_SIMT, FC_QVEC_TC = 0, 1, 2
FC_GRID_RECOMPUTE = 1
FC_ROUND_AUTO, FC_ROUND_TOPK, FC_ROUND_LIST = 0, 1, 2
FC_DECIDED_CERT, FC_DECIDED_RESCORED, FC_DECIDED_TOP16, FC_DECIDED_LIST = 1, 2, 4, 8
FC_DECIDED_EXACT_LIST, FC_DECIDED_SCAN, FC_DECIDED_PLAIN = 16, 32, 64

_STATUS_NAMES = {0: "FC_OK", 1: "FC_PENDING", -1: "FC_ERR_ARG", -2: "FC_ERR_NOT_SPD", -3: "FC_ERR_BUDGET",
                 -4: "FC_ERR_CUDA", -5: "FC_ERR_TIMEOUT", -6: "FC_ERR_CANCELLED", -7: "FC_ERR_NOT_FOUND",
                 -8: "FC_ERR_STATE"}

EXPORTS = ["fc_default_opts", "fc_create", "fc_destroy", "fc_load_grid", "fc_set_frac_cov", "fc_unload_grid",
           "fc_run_points", "fc_run_point", "fc_fake_data", "fc_covariance", "fc_scan", "fc_quantiles",
           "fc_submit", "fc_poll", "fc_cancel", "fc_get_stats", "fc_last_error", "fc_fake_data_noalloc",
           "fc_set_tuning", "fc_get_tuning", "fc_autotune", "fc_get_serve_stats", "fc_data_dchi2", "fc_fc_region",
           "fc_fc_region_adaptive", "fc_load_grid_osc", "fc_load_grid_osc_ex", "fc_get_decided_by", "fc_set_wait_test", "fc_measure_peaks"]


class FCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fc_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32), ("top_k", ctypes.c_int32),
                ("fluct", ctypes.c_int32), ("cov", ctypes.c_int32)]


class fc_osc_model(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int32), ("axis_len", ctypes.c_void_p), ("axis_values", ctypes.c_void_p),
                ("n_terms", ctypes.c_int32), ("amp_axis", ctypes.c_void_p), ("dm2_axis", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("f", ctypes.c_void_p), ("L", ctypes.c_void_p), ("E", ctypes.c_void_p)]


class fc_stats(ctypes.Structure):
    _fields_ = [("universes", ctypes.c_int64), ("scans", ctypes.c_int64), ("chi2_evals", ctypes.c_int64),
                ("distinct_cov", ctypes.c_int64), ("screened", ctypes.c_int64), ("rescored", ctypes.c_int64),
                ("rescreened", ctypes.c_int64), ("fallback", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("screen_launches", ctypes.c_int64), ("screen_flops", ctypes.c_double)] + [
        (n, ctypes.c_double) for n in ("ms_fake", "ms_cov", "ms_prep", "ms_screen", "ms_rescore", "ms_fallback",
                                       "ms_scan64", "ms_finish", "ms_total")] + [
        ("evicted", ctypes.c_int64), ("cache_slots", ctypes.c_int64), ("max_distinct_cov", ctypes.c_int64),
        ("scan_waves", ctypes.c_int64), ("big_listed", ctypes.c_int64), ("screen_tiles", ctypes.c_int64),
        ("screen_rows", ctypes.c_int64), ("deferred", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("residuals", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fc_tuning(ctypes.Structure):
    _fields_ = [("qvec", ctypes.c_int32), ("screen_stages", ctypes.c_int32), ("screen_ybuf", ctypes.c_int32),
                ("cache_slots", ctypes.c_int32), ("first_round", ctypes.c_int32), ("slot_rows", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fc_job(ctypes.Structure):
    _fields_ = [("grid_id", ctypes.c_int32), ("ps", ctypes.c_void_p), ("P", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("U", ctypes.c_int32), ("opts", fc_opts), ("dchi2", ctypes.c_void_p),
                ("bestfit", ctypes.c_void_p), ("nscans", ctypes.c_void_p)]


_lib = None


def lib_path() -> str:
    return _build_lib.LIB


def load(build: bool = False):
    """Load libfc.so (building it first when asked).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build_lib.build()
    path = _build_lib.LIB
    if not os.path.exists(path):
        raise FCError(FC_ERR_STATE, f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "fc_default_opts": (None, [ctypes.POINTER(fc_opts)]),
        "fc_create": (st, [ctypes.POINTER(vp), ctypes.c_int, sz, vp]),
        "fc_destroy": (st, [vp]),
        "fc_load_grid": (st, [vp, vp, i64, i32, vp, i32, ctypes.POINTER(i32)]),
        "fc_load_grid_osc": (st, [vp, ctypes.POINTER(fc_osc_model), i32, vp, i32, ctypes.POINTER(i32)]),
        "fc_load_grid_osc_ex": (st, [vp, ctypes.POINTER(fc_osc_model), i32, vp, i32, ctypes.c_uint32,
                                     ctypes.POINTER(i32)]),
        "fc_set_frac_cov": (st, [vp, i32, vp, i32]),
        "fc_unload_grid": (st, [vp, i32]),
        "fc_run_points": (st, [vp, i32, vp, i32, u64, i32, ctypes.POINTER(fc_opts), vp, vp, vp]),
        "fc_run_point": (st, [vp, i32, i64, u64, i32, ctypes.POINTER(fc_opts), vp, vp, vp]),
        "fc_fake_data": (st, [vp, i32, vp, i32, u64, i32, i32, vp]),
        "fc_covariance": (st, [vp, i32, i64, vp, vp]),
        "fc_scan": (st, [vp, i32, vp, vp, i32, i32, i32, vp, vp]),
        "fc_quantiles": (st, [vp, vp, i32, i32, vp, i32, vp]),
        "fc_submit": (st, [vp, ctypes.POINTER(fc_job), ctypes.POINTER(u64)]),
        "fc_poll": (st, [vp, u64, ctypes.POINTER(ctypes.c_double)]),
        "fc_cancel": (st, [vp, u64]),
        "fc_get_stats": (st, [vp, ctypes.POINTER(fc_stats)]),
        "fc_get_serve_stats": (st, [vp, ctypes.POINTER(fc_stats)]),
        "fc_get_decided_by": (st, [vp, vp, i64]),
        "fc_set_wait_test": (st, [vp, u64, i64]),
        "fc_measure_peaks": (st, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "fc_data_dchi2": (st, [vp, i32, vp, vp, i32, ctypes.POINTER(fc_opts), vp, vp, vp]),
        "fc_fc_region": (st, [vp, vp, i32, i32, vp, ctypes.c_double, vp, vp]),
        "fc_fc_region_adaptive": (st, [vp, i32, vp, i32, vp, ctypes.c_double, i32, i32, ctypes.c_double, u64,
                                       ctypes.POINTER(fc_opts), vp, vp, vp]),
        "fc_set_tuning": (st, [vp, i32, ctypes.POINTER(fc_tuning)]),
        "fc_get_tuning": (st, [vp, i32, ctypes.POINTER(fc_tuning)]),
        "fc_autotune": (st, [vp, i32, ctypes.c_char_p, ctypes.POINTER(fc_tuning)]),
        "fc_last_error": (ctypes.c_char_p, [vp]),
        "fc_fake_data_noalloc": (st, [vp, i64, i32, vp, i32, vp, vp, i32, u64, i32, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, ctx=None):
    if status in (FC_OK, FC_PENDING):
        return status
    msg = load().fc_last_error(ctx)
    raise FCError(status, msg.decode() if msg else "")


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _host(a, dtype):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def _opts(opts) -> fc_opts:
    o = fc_opts()
    load().fc_default_opts(ctypes.byref(o))
    if opts is None:
        return o
    if isinstance(opts, fc_opts):
        return opts
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


# -- entry points (names of include/fc.h) -----------------------------------

def fc_default_opts(**over) -> fc_opts:
    return _opts(over)


def fc_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
    ctx = ctypes.c_void_p()
    _check(load().fc_create(ctypes.byref(ctx), device, hbm_budget_bytes, cuda_stream))
    return ctx


def fc_destroy(ctx):
    _check(load().fc_destroy(ctx), ctx)


def fc_load_grid(ctx, S, collapse=None, n_fit: int | None = None) -> int:
    S = _host(S, np.float64)
    G, nf = int(S.shape[0]), int(S.shape[1])
    coll = _host(collapse, np.int32)
    nfit = nf if n_fit is None else int(n_fit)
    gid = ctypes.c_int32()
    _check(load().fc_load_grid(ctx, _ptr(S), G, nf, _ptr(coll), nfit, ctypes.byref(gid)), ctx)
    return gid.value


def fc_load_grid_osc(ctx, axes, terms, b, f, L, E, collapse=None, n_fit: int | None = None,
                     recompute: bool = False, flags: int | None = None) -> int:
    """Grid spectra generated on the device: axes = list of 1-D value arrays (axis 0 slowest),
    terms = list of (amplitude axis, dm2 axis), b/L/E [N_full], f [n_terms][N_full].
    recompute: keep no spectra, evaluate the model wherever a row is read (FC_GRID_RECOMPUTE);
    flags, when given, are passed as they are."""
    axes = [_host(a, np.float64) for a in axes]
    lens = np.array([len(a) for a in axes], np.int32)
    vals = np.ascontiguousarray(np.concatenate(axes), np.float64)
    amp = np.array([t[0] for t in terms], np.int32)
    dm2 = np.array([t[1] for t in terms], np.int32)
    b, L, E = (_host(x, np.float64) for x in (b, L, E))
    f = np.ascontiguousarray(_host(f, np.float64).reshape(len(terms), -1))
    nf = int(b.shape[0])
    coll = _host(collapse, np.int32)
    nfit = nf if n_fit is None else int(n_fit)
    m = fc_osc_model(len(axes), _ptr(lens), _ptr(vals), len(terms), _ptr(amp), _ptr(dm2), _ptr(b), _ptr(f), _ptr(L),
                     _ptr(E))
    gid = ctypes.c_int32()
    _check(load().fc_load_grid_osc_ex(ctx, ctypes.byref(m), nf, _ptr(coll) if coll is not None else None, nfit,
                                      (FC_GRID_RECOMPUTE if recompute else 0) if flags is None else flags,
                                      ctypes.byref(gid)), ctx)
    return gid.value


def fc_load_grid_osc_ex(ctx, axes, terms, b, f, L, E, collapse=None, n_fit: int | None = None, flags: int = 0) -> int:
    """fc_load_grid_osc with the C entry point's flags (FC_GRID_RECOMPUTE)."""
    return fc_load_grid_osc(ctx, axes, terms, b, f, L, E, collapse, n_fit, flags=flags)


def fc_set_frac_cov(ctx, grid_id: int, F):
    F = _host(F, np.float64)
    _check(load().fc_set_frac_cov(ctx, grid_id, _ptr(F), int(F.shape[0])), ctx)


def fc_unload_grid(ctx, grid_id: int):
    _check(load().fc_unload_grid(ctx, grid_id), ctx)


def fc_run_points(ctx, grid_id: int, ps, seed: int, U: int, opts=None, dchi2=None, bestfit=None, nscans=None,
                  want_bestfit: bool = True, want_nscans: bool = True):
    """dchi2 [P][U] (+ bestfit, nscans).  Output buffers may be passed in (host or device)."""
    ps = _host(ps, np.int64)
    P = int(ps.shape[0])
    o = _opts(opts)
    if dchi2 is None:
        dchi2 = np.empty((P, U), np.float64)
    if bestfit is None and want_bestfit:
        bestfit = np.empty((P, U), np.int64)
    if nscans is None and want_nscans:
        nscans = np.empty((P, U), np.int8)
    _check(load().fc_run_points(ctx, grid_id, _ptr(ps), P, seed, U, ctypes.byref(o), _ptr(dchi2), _ptr(bestfit),
                                _ptr(nscans)), ctx)
    return dchi2, bestfit, nscans


def fc_run_point(ctx, grid_id: int, p: int, seed: int, U: int, opts=None):
    o = _opts(opts)
    d = np.empty(U, np.float64)
    b = np.empty(U, np.int64)
    n = np.empty(U, np.int8)
    _check(load().fc_run_point(ctx, grid_id, int(p), seed, U, ctypes.byref(o), _ptr(d), _ptr(b), _ptr(n)), ctx)
    return d, b, n


def fc_fake_data(ctx, grid_id: int, ps, seed: int, U: int, n_fit: int, fluct: int = FC_FLUCT_POISSON_SYS, out=None):
    ps = _host(ps, np.int64)
    P = int(ps.shape[0])
    if out is None:
        out = np.empty((P, U, n_fit), np.float32)
    _check(load().fc_fake_data(ctx, grid_id, _ptr(ps), P, seed, U, fluct, _ptr(out)), ctx)
    return out


def fc_covariance(ctx, grid_id: int, q: int, n_fit: int, n_full: int, want_A: bool = True, want_L: bool = True):
    A = np.empty((n_fit, n_fit)) if want_A else None
    L = np.empty((n_full, n_full)) if want_L else None
    _check(load().fc_covariance(ctx, grid_id, int(q), _ptr(A), _ptr(L)), ctx)
    return A, L


def fc_scan(ctx, grid_id: int, d, q_cov, precision: int = FC_PREC_MIXED, top_k: int = 8):
    d = _host(d, np.float32)
    q = _host(q_cov, np.int64)
    U = int(q.shape[0])
    best = np.empty(U, np.int64)
    chi2 = np.empty(U, np.float64)
    _check(load().fc_scan(ctx, grid_id, _ptr(d), _ptr(q), U, precision, top_k, _ptr(best), _ptr(chi2)), ctx)
    return best, chi2


def fc_data_dchi2(ctx, grid_id: int, d, ps, opts=None):
    """Observed data's (dchi2, bestfit, nscans) at each grid point of ps."""
    d = _host(d, np.float32)
    ps = _host(ps, np.int64)
    P = int(ps.shape[0])
    o = _opts(opts)
    dchi2 = np.empty(P, np.float64)
    best = np.empty(P, np.int64)
    ns = np.empty(P, np.int8)
    _check(load().fc_data_dchi2(ctx, grid_id, _ptr(d), _ptr(ps), P, ctypes.byref(o), _ptr(dchi2), _ptr(best),
                                _ptr(ns)), ctx)
    return dchi2, best, ns


def fc_fc_region(ctx, dchi2_univ, dchi2_data, cl: float):
    """(crit [P], accepted [P] uint8): cl-quantile of each point's universes and dchi2_data <= crit."""
    x = _host(dchi2_univ, np.float64)
    dd = _host(dchi2_data, np.float64)
    P, U = int(x.shape[0]), int(x.shape[1])
    crit = np.empty(P, np.float64)
    acc = np.empty(P, np.uint8)
    _check(load().fc_fc_region(ctx, _ptr(x), P, U, _ptr(dd), float(cl), _ptr(crit), _ptr(acc)), ctx)
    return crit, acc


def fc_fc_region_adaptive(ctx, grid_id: int, ps, dchi2_data, cl: float, U0: int, U_max: int, z: float = 3.0,
                          seed: int = 0, opts=None):
    """(accepted [P] uint8, U_used [P] int32, frac [P] float64): FC acceptance with universes added per point
    until the empirical distribution at the data's value is z standard errors from cl (or U_max)."""
    ps = _host(ps, np.int64)
    dd = _host(dchi2_data, np.float64)
    P = int(ps.shape[0])
    o = _opts(opts)
    acc = np.empty(P, np.uint8)
    used = np.empty(P, np.int32)
    frac = np.empty(P, np.float64)
    _check(load().fc_fc_region_adaptive(ctx, grid_id, _ptr(ps), P, _ptr(dd), float(cl), int(U0), int(U_max),
                                        float(z), int(seed), ctypes.byref(o), _ptr(acc), _ptr(used), _ptr(frac)),
           ctx)
    return acc, used, frac


def fc_quantiles(ctx, x, probs):
    x = _host(x, np.float64)
    p = _host(probs, np.float64)
    rows, n = int(x.shape[0]), int(x.shape[1])
    out = np.empty((rows, int(p.shape[0])), np.float64)
    _check(load().fc_quantiles(ctx, _ptr(x), rows, n, _ptr(p), int(p.shape[0]), _ptr(out)), ctx)
    return out


def fc_submit(ctx, grid_id: int, ps, seed: int, U: int, opts=None, dchi2=None, bestfit=None, nscans=None,
              want_bestfit: bool = False, want_nscans: bool = False):
    """Queue a job; the output arrays (returned) must stay alive until fc_poll reports it done."""
    ps = _host(ps, np.int64)
    P = int(ps.shape[0])
    if dchi2 is None:
        dchi2 = np.empty((P, U), np.float64)
    if bestfit is None and want_bestfit:
        bestfit = np.empty((P, U), np.int64)
    if nscans is None and want_nscans:
        nscans = np.empty((P, U), np.int8)
    j = fc_job()
    j.grid_id, j.ps, j.P, j.seed, j.U = grid_id, _ptr(ps), P, seed, U
    j.opts = _opts(opts)
    j.dchi2, j.bestfit, j.nscans = _ptr(dchi2), _ptr(bestfit), _ptr(nscans)
    t = ctypes.c_uint64()
    _check(load().fc_submit(ctx, ctypes.byref(j), ctypes.byref(t)), ctx)
    return t.value, (dchi2, bestfit, nscans)


def fc_poll(ctx, ticket: int):
    """(status, latency_ms): FC_PENDING while running; raises FCError for a failed job."""
    lat = ctypes.c_double(0.0)
    st = _check(load().fc_poll(ctx, ticket, ctypes.byref(lat)), ctx)
    return st, lat.value


def fc_cancel(ctx, ticket: int):
    _check(load().fc_cancel(ctx, ticket), ctx)


def fc_set_tuning(ctx, grid_id: int, qvec: int = 0, screen_stages: int = 0, screen_ybuf: int = 0,
                  cache_slots: int = 0, first_round: int = 0, slot_rows: int = 0):
    t = fc_tuning(qvec, screen_stages, screen_ybuf, cache_slots, first_round, slot_rows)
    _check(load().fc_set_tuning(ctx, grid_id, ctypes.byref(t)), ctx)


def fc_get_tuning(ctx, grid_id: int) -> dict:
    t = fc_tuning()
    _check(load().fc_get_tuning(ctx, grid_id, ctypes.byref(t)), ctx)
    return t.as_dict()


def fc_autotune(ctx, grid_id: int, cache_path: str | None = None) -> dict:
    t = fc_tuning()
    path = cache_path.encode() if cache_path else None
    _check(load().fc_autotune(ctx, grid_id, path, ctypes.byref(t)), ctx)
    return t.as_dict()


def fc_get_serve_stats(ctx) -> dict:
    s = fc_stats()
    _check(load().fc_get_serve_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def fc_measure_peaks(ctx) -> tuple[float, float]:
    """(fp64, fp32) fma TFLOP/s of the context's device, measured by probe kernels."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().fc_measure_peaks(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def fc_set_wait_test(ctx, wait_ns: int = 0, screen_stop_after: int = -1):
    """Test hook: limit of the screen's pipeline waits (0 = built-in) and a producer stop after n stages (-1 = off)."""
    _check(load().fc_set_wait_test(ctx, int(wait_ns), int(screen_stop_after)), ctx)


def fc_get_decided_by(ctx, n: int) -> np.ndarray:
    """Per universe of the last synchronous fit: OR of the FC_DECIDED_* bits of the rounds that decided it."""
    out = np.empty(int(n), np.uint8)
    _check(load().fc_get_decided_by(ctx, _ptr(out), int(n)), ctx)
    return out


def fc_get_stats(ctx) -> dict:
    s = fc_stats()
    _check(load().fc_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def fc_fake_data_noalloc(S, F, ps, seed: int, U: int, d, collapse=None, n_fit: int | None = None,
                         fluct: int = FC_FLUCT_POISSON_SYS, cuda_stream: int | None = None):
    """Fake data into the caller's device buffer d [P][U][N_fit] without any device allocation.

    S, F, ps, collapse and d must be CUDA tensors (device memory)."""
    G, nf = int(S.shape[0]), int(S.shape[1])
    nfit = nf if n_fit is None else int(n_fit)
    _check(load().fc_fake_data_noalloc(_ptr(S), G, nf, _ptr(collapse), nfit, _ptr(F), _ptr(ps), int(ps.shape[0]),
                                       seed, U, fluct, _ptr(d), cuda_stream))
    return d


def fc_last_error(ctx=None) -> str:
    m = load().fc_last_error(ctx)
    return m.decode() if m else ""
