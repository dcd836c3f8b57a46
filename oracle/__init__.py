"""CPU oracle for the Kalman smoother -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import this package.  The product path (``paper_2502_11686_gb300``) never imports it and
shares no code with it.

``smooth`` calls ``ks_oracle.c``: a plain sequential FP64 Paige-Saunders block QR of the
whitened least-squares matrix U A (Section 2 and Section 3 of Gargir & Toledo), back
substitution, and Algorithm 1 (block SelInv for (R^T R)^{-1}) with I = {j+1}.  See the C
file's header for the precise definitions and indexing.

Every function here is pinned by ``tests/test_oracle_pins.py`` against things the paper and
the mathematics fix (dense least squares on tiny inputs, normal equations, the scalar
random-walk steady state, exact recovery, the RTS smoother, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "ARG", 2: "NOT_SPD", 3: "SINGULAR", 4: "OOM"}


class OracleError(RuntimeError):
    def __init__(self, code: int, info: int):
        super().__init__(f"oracle failed: {STATUS.get(code, code)} at index {info}")
        self.code = code
        self.info = info


def build(force: bool = False) -> str:
    """Compile ks_oracle.c into liboracle.so next to it (plain gcc, no vendor libraries)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """ctypes handle of a compiled oracle at ``path`` (tests also load planted-mistake copies)."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_smooth.restype = ctypes.c_int
    lib.oracle_smooth.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P, P,
                                  P, P, P, P, P]
    lib.oracle_smooth_var.restype = ctypes.c_int
    lib.oracle_smooth_var.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_LIB_PATH)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def smooth(prob, covariances: bool = True, cross: bool = False, lib=None):
    """Smoothed states (and covariances) of a problem.

    ``prob`` has attributes k, n, m (int32[k]) and FP64 arrays F, H, c (or None), K, G, o, C in
    the packed layout of ``paper_2502_11686_gb300.inputs.Problem``.
    Returns a dict with ``u`` [k,n], ``cov`` [k,n,n] (or None), ``cross`` [k-1,n,n] (or None)
    and ``resid2`` (the minimal objective value).
    """
    lib = lib or _load()
    k, n = int(prob.k), int(prob.n)
    m = np.ascontiguousarray(prob.m, dtype=np.int32)
    F, H, c, K = _f64(prob.F), _f64(prob.H), _f64(prob.c), _f64(prob.K)
    G, o, C = _f64(prob.G), _f64(prob.o), _f64(prob.C)
    u = np.zeros((k, n))
    cov = np.zeros((k, n, n)) if covariances else None
    crs = np.zeros((max(k - 1, 1), n, n)) if cross else None
    resid = ctypes.c_double(0.0)
    info = ctypes.c_int64(-1)
    st = lib.oracle_smooth(k, n, _ptr(m), _ptr(F), _ptr(H), _ptr(c), _ptr(K), _ptr(G), _ptr(o),
                           _ptr(C), _ptr(u), _ptr(cov), _ptr(crs), ctypes.byref(resid),
                           ctypes.byref(info))
    if st != 0:
        raise OracleError(st, info.value)
    return {"u": u, "cov": cov, "cross": (crs[: k - 1] if cross else None),
            "resid2": resid.value}


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def smooth_var(prob, covariances: bool = True, lib=None):
    """Smoothed states (and covariances) of a problem whose state dimension varies per step
    (``paper_2502_11686_gb300.inputs.VarProblem``: per-step n_i, evolution rows l_i, packed
    arrays).  Returns ``u`` packed [sum n_i], ``cov`` packed [sum n_i^2] (or None) and
    ``resid2``."""
    lib = lib or _load()
    k = int(prob.k)
    nd, m = _i32(prob.nd), _i32(prob.m)
    lv = _i32(prob.l) if k > 1 else _i32(np.zeros(1))
    F, H, c, K = _f64(prob.F), _f64(prob.H), _f64(prob.c), _f64(prob.K)
    G, o, C = _f64(prob.G), _f64(prob.o), _f64(prob.C)
    u = np.zeros(int(nd.astype(np.int64).sum()))
    cov = np.zeros(int((nd.astype(np.int64) ** 2).sum())) if covariances else None
    resid = ctypes.c_double(0.0)
    info = ctypes.c_int64(-1)
    st = lib.oracle_smooth_var(k, _ptr(nd), _ptr(lv), _ptr(m), _ptr(F), _ptr(H), _ptr(c), _ptr(K),
                               _ptr(G), _ptr(o), _ptr(C), _ptr(u), _ptr(cov), ctypes.byref(resid),
                               ctypes.byref(info))
    if st != 0:
        raise OracleError(st, info.value)
    return {"u": u, "cov": cov, "resid2": resid.value}
