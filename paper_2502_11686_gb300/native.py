"""ctypes binding of libks.so with the C ABI's own names (argument marshalling only).

Every step of the smoother runs in the library's CUDA kernels; nothing here computes.  Arrays
may be torch tensors (device or host) or numpy arrays (host); they are passed as raw pointers.
If libks.so has not been built, the first call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libks.so")

KS_OK, KS_ERR_ARG, KS_ERR_NOT_SPD, KS_ERR_SINGULAR, KS_ERR_OOM, KS_ERR_CUDA, KS_ERR_TIMEOUT, \
    KS_ERR_NO_FACTOR, KS_ERR_NONFINITE = range(9)
STATUS_NAMES = {0: "KS_OK", 1: "KS_ERR_ARG", 2: "KS_ERR_NOT_SPD", 3: "KS_ERR_SINGULAR",
                4: "KS_ERR_OOM", 5: "KS_ERR_CUDA", 6: "KS_ERR_TIMEOUT", 7: "KS_ERR_NO_FACTOR",
                8: "KS_ERR_NONFINITE"}
KS_FP64, KS_FP32_REFINE = 0, 1
KS_TI_F, KS_TI_H, KS_TI_K, KS_TI_G, KS_TI_C = 1, 2, 4, 8, 16

# Every symbol include/ks.h declares.
EXPORTS = ("ks_default_options", "ks_create", "ks_smooth", "ks_covariances", "ks_residual",
           "ks_release", "ks_sync", "ks_destroy", "ks_last_error", "ks_max_n", "ks_max_m",
           "ks_profile_read", "ks_smooth_static", "ks_smooth_batch", "ks_generate",
           "ks_server_create", "ks_server_submit", "ks_server_submit_synthetic",
           "ks_server_covariances", "ks_server_wait", "ks_server_result", "ks_server_release",
           "ks_server_stats", "ks_server_destroy", "ks_measure_fma_rate", "ks_smooth_var",
           "ks_covariances_var", "ks_generate_steps", "ks_gn_default_options",
           "ks_gauss_newton", "ks_pendulum_linearize")
PHASES = ("whiten", "level", "backsub", "refine", "selinv", "copy", "batch")


class ks_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("mem_budget", ctypes.c_size_t),
                ("sync", ctypes.c_int), ("profile", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


class ks_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("phase_launches", ctypes.c_uint64 * 7),
                ("phase_ms", ctypes.c_double * 7), ("calls", ctypes.c_uint64)]


class ks_problem(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("n", ctypes.c_int), ("m", ctypes.c_void_p),
                ("F", ctypes.c_void_p), ("H", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("K", ctypes.c_void_p), ("G", ctypes.c_void_p), ("o", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("u_out", ctypes.c_void_p), ("cov_out", ctypes.c_void_p),
                ("time_invariant", ctypes.c_uint)]


class ks_server_options(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("keep_factors", ctypes.c_int)]


class ks_request_info(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("info", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("k", ctypes.c_int64), ("n", ctypes.c_int)]


class ks_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("bytes_budget", ctypes.c_size_t), ("shared_launches", ctypes.c_int64),
                ("max_requests_per_launch", ctypes.c_int64)]


class ks_gn_options(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("lambda0", ctypes.c_double), ("ftol", ctypes.c_double),
                ("xtol", ctypes.c_double)]


class ks_gn_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("accepted", ctypes.c_int), ("converged", ctypes.c_int),
                ("objective0", ctypes.c_double), ("objective", ctypes.c_double),
                ("lambda_", ctypes.c_double)]


class ks_pendulum(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double), ("o", ctypes.c_void_p)]


LINEARIZE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class KsError(RuntimeError):
    def __init__(self, status: int, message: str, info: int = -1):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}"
                         + (f" (info={info})" if info >= 0 else ""))
        self.status = status
        self.info = info


_lock = threading.Lock()
_lib = None


def load():
    """Loads libks.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                               "g.build()'` first (there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.ks_default_options.argtypes = [ctypes.POINTER(ks_options)]
        lib.ks_default_options.restype = None
        lib.ks_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ks_options)]
        lib.ks_create.restype = I
        lib.ks_smooth.argtypes = [P, I64, I, P, P, P, P, P, P, P, P, P, ctypes.POINTER(P),
                                  ctypes.POINTER(I64)]
        lib.ks_smooth.restype = I
        lib.ks_covariances.argtypes = [P, P, P, P]
        lib.ks_covariances.restype = I
        lib.ks_residual.argtypes = [P, P, ctypes.POINTER(ctypes.c_double)]
        lib.ks_residual.restype = I
        lib.ks_release.argtypes = [P, P]
        lib.ks_release.restype = I
        lib.ks_sync.argtypes = [P, ctypes.POINTER(I64)]
        lib.ks_sync.restype = I
        lib.ks_destroy.argtypes = [P]
        lib.ks_destroy.restype = I
        lib.ks_last_error.argtypes = [P]
        lib.ks_last_error.restype = ctypes.c_char_p
        lib.ks_max_n.argtypes = [P]
        lib.ks_max_n.restype = I
        lib.ks_max_m.argtypes = [P, I]
        lib.ks_max_m.restype = I
        lib.ks_profile_read.argtypes = [P, ctypes.POINTER(ks_profile), I]
        lib.ks_profile_read.restype = I
        lib.ks_smooth_static.argtypes = [I, P, I64, I, I, P, P, P, P, P, P, P, P, P,
                                         ctypes.POINTER(I64), ctypes.c_char_p, ctypes.c_size_t]
        lib.ks_smooth_static.restype = I
        lib.ks_smooth_batch.argtypes = [P, I, ctypes.POINTER(ks_problem), ctypes.POINTER(I),
                                        ctypes.POINTER(I64)]
        lib.ks_smooth_batch.restype = I
        lib.ks_generate.argtypes = [P, I64, I, I, ctypes.c_uint64, ctypes.c_double, P, P, P, P, P, P]
        lib.ks_generate.restype = I
        lib.ks_generate_steps.argtypes = [P, I64, I, I, ctypes.c_uint64, ctypes.c_double, P, P, P,
                                          P, P, P]
        lib.ks_generate_steps.restype = I
        lib.ks_gn_default_options.argtypes = [ctypes.POINTER(ks_gn_options)]
        lib.ks_gn_default_options.restype = None
        lib.ks_gauss_newton.argtypes = [P, I64, I, I, LINEARIZE_FN, P, P, P, P,
                                        ctypes.POINTER(ks_gn_options), ctypes.POINTER(ks_gn_report)]
        lib.ks_gauss_newton.restype = I
        lib.ks_pendulum_linearize.argtypes = [P, I64, I, I, P, P, P, P, P, P]
        lib.ks_pendulum_linearize.restype = ctypes.c_int
        lib.ks_server_create.argtypes = [P, ctypes.POINTER(ks_server_options), ctypes.POINTER(P)]
        lib.ks_server_create.restype = I
        lib.ks_server_submit.argtypes = [P, ctypes.POINTER(ks_problem), ctypes.POINTER(I64)]
        lib.ks_server_submit.restype = I
        lib.ks_server_submit_synthetic.argtypes = [P, I64, I, I, ctypes.c_uint64, I, ctypes.POINTER(I64)]
        lib.ks_server_submit_synthetic.restype = I
        lib.ks_server_covariances.argtypes = [P, I64, P, ctypes.POINTER(I64)]
        lib.ks_server_covariances.restype = I
        lib.ks_server_wait.argtypes = [P, I64, ctypes.c_double, ctypes.POINTER(ks_request_info)]
        lib.ks_server_wait.restype = I
        lib.ks_server_result.argtypes = [P, I64, P, P]
        lib.ks_server_result.restype = I
        lib.ks_server_release.argtypes = [P, I64]
        lib.ks_server_release.restype = I
        lib.ks_server_stats.argtypes = [P, ctypes.POINTER(ks_server_counters)]
        lib.ks_server_stats.restype = I
        lib.ks_server_destroy.argtypes = [P]
        lib.ks_server_destroy.restype = I
        lib.ks_measure_fma_rate.argtypes = [I, I, ctypes.POINTER(ctypes.c_double)]
        lib.ks_measure_fma_rate.restype = I
        lib.ks_smooth_var.argtypes = [P, I64, P, P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(P),
                                      ctypes.POINTER(I64)]
        lib.ks_smooth_var.restype = I
        lib.ks_covariances_var.argtypes = [P, P, P]
        lib.ks_covariances_var.restype = I
        _lib = lib
        return lib


def ptr(a):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, st, info=-1):
    if st != KS_OK:
        raise KsError(st, ks_last_error(ctx), info)


def ks_default_options() -> ks_options:
    o = ks_options()
    load().ks_default_options(ctypes.byref(o))
    return o


def ks_create(opts: ks_options | None = None):
    ctx = ctypes.c_void_p()
    st = load().ks_create(ctypes.byref(ctx), ctypes.byref(opts) if opts is not None else None)
    if st != KS_OK:
        raise KsError(st, "ks_create failed")
    return ctx


def ks_smooth(ctx, k, n, m, F, H, c, K, G, o, C, u_out, keep=False, check=True, reuse=None):
    """Returns (status, handle or None, info).  With check=True a failure raises KsError.
    ``reuse``: a handle from an earlier call whose memory the library may reuse (keep=True)."""
    h = ctypes.c_void_p(reuse.value if reuse is not None else None)
    info = ctypes.c_int64(-1)
    st = load().ks_smooth(ctx, int(k), int(n), ptr(m), ptr(F), ptr(H), ptr(c), ptr(K), ptr(G),
                          ptr(o), ptr(C), ptr(u_out), ctypes.byref(h) if keep else None,
                          ctypes.byref(info))
    if check:
        _check(ctx, st, info.value)
    return st, (h if keep and h.value else None), info.value


def ks_covariances(ctx, h, cov_out, cross_out=None, check=True):
    st = load().ks_covariances(ctx, h, ptr(cov_out), ptr(cross_out))
    if check:
        _check(ctx, st)
    return st


def ks_residual(ctx, h) -> float:
    v = ctypes.c_double(0.0)
    _check(ctx, load().ks_residual(ctx, h, ctypes.byref(v)))
    return v.value


def ks_release(ctx, h):
    return load().ks_release(ctx, h)


def ks_sync(ctx):
    info = ctypes.c_int64(-1)
    st = load().ks_sync(ctx, ctypes.byref(info))
    return st, info.value


def ks_destroy(ctx):
    return load().ks_destroy(ctx)


def ks_last_error(ctx) -> str:
    return load().ks_last_error(ctx).decode()


def ks_max_n(ctx) -> int:
    return load().ks_max_n(ctx)


def ks_max_m(ctx, n) -> int:
    return load().ks_max_m(ctx, int(n))


def ks_profile_read(ctx, reset=False) -> dict:
    """Launch counts and per-phase GPU milliseconds of a ctx (see include/ks.h)."""
    pr = ks_profile()
    _check(ctx, load().ks_profile_read(ctx, ctypes.byref(pr), 1 if reset else 0))
    return {"launches": int(pr.launches), "calls": int(pr.calls),
            "phase_launches": {PHASES[i]: int(pr.phase_launches[i]) for i in range(7)},
            "phase_ms": {PHASES[i]: float(pr.phase_ms[i]) for i in range(7)}}


def ks_smooth_static(device, stream, k, n, m, F, H, c, K, G, o, C, u_out, cov_out=None):
    """The allocation-free entry point (device arrays only; see include/ks.h).
    Returns (status, info, message); never raises for a library status."""
    info = ctypes.c_int64(-1)
    buf = ctypes.create_string_buffer(512)
    st = load().ks_smooth_static(int(device), stream, int(k), int(n), int(m), ptr(F), ptr(H),
                                 ptr(c), ptr(K), ptr(G), ptr(o), ptr(C), ptr(u_out),
                                 ptr(cov_out), ctypes.byref(info), buf, len(buf))
    return st, info.value, buf.value.decode()


def _problem_struct(p, keep):
    m = p["m"]
    keep.append(m)
    return ks_problem(int(p["k"]), int(p["n"]), ptr(m), ptr(p.get("F")), ptr(p.get("H")),
                      ptr(p.get("c")), ptr(p.get("K")), ptr(p.get("G")), ptr(p.get("o")),
                      ptr(p.get("C")), ptr(p["u_out"]), ptr(p.get("cov_out")),
                      int(p.get("time_invariant", 0)))


def ks_generate(ctx, k, n, m, seed, f_scale, F, H, K, G, C, o):
    st = load().ks_generate(ctx, int(k), int(n), int(m), int(seed), float(f_scale), ptr(F), ptr(H),
                            ptr(K), ptr(G), ptr(C), ptr(o))
    _check(ctx, st)


def ks_generate_steps(ctx, k, n, m, seed, f_scale, F, H, K, G, C, o):
    st = load().ks_generate_steps(ctx, int(k), int(n), int(m), int(seed), float(f_scale), ptr(F),
                                  ptr(H), ptr(K), ptr(G), ptr(C), ptr(o))
    _check(ctx, st)


def ks_server_create(ctx, mem_budget=0, max_active=0, keep_factors=False):
    o = ks_server_options(int(mem_budget), int(max_active), 1 if keep_factors else 0)
    srv = ctypes.c_void_p()
    st = load().ks_server_create(ctx, ctypes.byref(o), ctypes.byref(srv))
    if st != KS_OK:
        raise KsError(st, ks_last_error(ctx))
    return srv


def ks_server_submit(srv, problem) -> int:
    keep = []
    s = _problem_struct(problem, keep)
    rid = ctypes.c_int64(0)
    st = load().ks_server_submit(srv, ctypes.byref(s), ctypes.byref(rid))
    if st != KS_OK:
        raise KsError(st, "ks_server_submit failed")
    return rid.value


def ks_server_submit_synthetic(srv, k, n, m, seed, want_cov=False) -> int:
    rid = ctypes.c_int64(0)
    st = load().ks_server_submit_synthetic(srv, int(k), int(n), int(m), int(seed),
                                           1 if want_cov else 0, ctypes.byref(rid))
    if st != KS_OK:
        raise KsError(st, "ks_server_submit_synthetic failed")
    return rid.value


def ks_server_covariances(srv, rid, cov_out=None) -> int:
    fid = ctypes.c_int64(0)
    st = load().ks_server_covariances(srv, int(rid), ptr(cov_out), ctypes.byref(fid))
    if st != KS_OK:
        raise KsError(st, "ks_server_covariances failed")
    return fid.value


def ks_server_wait(srv, rid, timeout_ms=-1.0) -> dict:
    info = ks_request_info()
    st = load().ks_server_wait(srv, int(rid), float(timeout_ms), ctypes.byref(info))
    return {"status": st, "done": bool(info.done), "request_status": info.status,
            "info": info.info, "queue_ms": info.queue_ms, "latency_ms": info.latency_ms,
            "k": info.k, "n": info.n}


def ks_server_result(srv, rid, u_out=None, cov_out=None):
    st = load().ks_server_result(srv, int(rid), ptr(u_out), ptr(cov_out))
    if st != KS_OK:
        raise KsError(st, "ks_server_result failed")


def ks_server_release(srv, rid):
    return load().ks_server_release(srv, int(rid))


def ks_server_stats(srv) -> dict:
    c = ks_server_counters()
    load().ks_server_stats(srv, ctypes.byref(c))
    return {f: getattr(c, f) for f, _ in ks_server_counters._fields_}


def ks_server_destroy(srv):
    return load().ks_server_destroy(srv)


def ks_smooth_batch(ctx, problems, check=True):
    """problems: list of dicts with k, n, m and the arrays of ks_smooth plus u_out / cov_out.
    Returns (status, per-problem statuses, per-problem infos)."""
    arr = (ks_problem * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        arr[i] = _problem_struct(p, keep)
    st_arr = (ctypes.c_int * len(problems))()
    info_arr = (ctypes.c_int64 * len(problems))()
    st = load().ks_smooth_batch(ctx, len(problems), arr, st_arr, info_arr)
    if check and st != KS_OK:
        bad = [i for i in range(len(problems)) if st_arr[i] != KS_OK]
        raise KsError(st, ks_last_error(ctx) + f" (problems {bad[:8]})",
                      info_arr[bad[0]] if bad else -1)
    return st, list(st_arr), list(info_arr)


def ks_measure_fma_rate(device, precision) -> float:
    """Measured FMA rate of the device in TFLOP/s (FP64 for KS_FP64, FP32 otherwise)."""
    v = ctypes.c_double(0.0)
    st = load().ks_measure_fma_rate(int(device), int(precision), ctypes.byref(v))
    if st != KS_OK:
        raise KsError(st, "ks_measure_fma_rate failed")
    return v.value


def ks_smooth_var(ctx, k, nd, l, m, F, H, c, K, G, o, C, u_out, keep=False, check=True):
    """Variable state dimensions (see include/ks.h).  nd, l, m: int32 host arrays.
    Returns (status, handle or None, info)."""
    import numpy as np
    nd = np.ascontiguousarray(nd, dtype=np.int32)
    lv = np.ascontiguousarray(l if l is not None and len(l) else np.zeros(1), dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    h = ctypes.c_void_p(None)
    info = ctypes.c_int64(-1)
    st = load().ks_smooth_var(ctx, int(k), ptr(nd), ptr(lv), ptr(m), ptr(F), ptr(H), ptr(c),
                              ptr(K), ptr(G), ptr(o), ptr(C), ptr(u_out),
                              ctypes.byref(h) if keep else None, ctypes.byref(info))
    if check:
        _check(ctx, st, info.value)
    return st, (h if keep and h.value else None), info.value


def ks_covariances_var(ctx, h, cov_out, check=True):
    st = load().ks_covariances_var(ctx, h, ptr(cov_out))
    if check:
        _check(ctx, st)
    return st


def ks_gn_default_options() -> ks_gn_options:
    o = ks_gn_options()
    load().ks_gn_default_options(ctypes.byref(o))
    return o


def pendulum_linearizer():
    """The library's built-in pendulum linearization as a ks_linearize_fn pointer."""
    return ctypes.cast(load().ks_pendulum_linearize, LINEARIZE_FN)


def ks_gauss_newton(ctx, k, n, m, fn, user, K, C, u, opts=None, check=True):
    """Levenberg-Marquardt smoothing (see include/ks.h).  fn: a LINEARIZE_FN (e.g.
    pendulum_linearizer()); user: a ctypes object passed by reference (e.g. ks_pendulum).
    Returns (status, report dict)."""
    rep = ks_gn_report()
    uptr = ctypes.addressof(user) if user is not None else None
    st = load().ks_gauss_newton(ctx, int(k), int(n), int(m), fn, uptr, ptr(K), ptr(C), ptr(u),
                                ctypes.byref(opts) if opts is not None else None, ctypes.byref(rep))
    if check:
        _check(ctx, st)
    return st, {"iterations": rep.iterations, "accepted": rep.accepted,
                "converged": bool(rep.converged), "objective0": rep.objective0,
                "objective": rep.objective, "lambda": rep.lambda_}
