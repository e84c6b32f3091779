"""FP64 CPU oracle for ADMM LP decoding (and the appendix's dual subgradient
decoder) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library (``liblpdec``)
never loads it, and it shares no code with the CUDA path.

The arithmetic lives in ``admm_oracle.c`` (plain C, double precision, written
from Algorithms 1 and 2 of the paper); this module compiles it with gcc and
wraps it with ctypes.  ctypes releases the GIL during foreign calls, so
``decode`` splits a batch of frames over a thread pool.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "admm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile admm_oracle.c into liboracle.so (gcc, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                                   "-fno-fast-math", "-ffp-contract=off",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_project.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_project_bisect.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_project_many.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int]
        lib.oracle_decode.argtypes = [
            ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int, dp,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
            dp, u8p, i32p, u8p, u8p, dp]
        lib.oracle_lp_max.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_decode_dual.argtypes = [
            ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
            dp, u8p, i32p, u8p]
        for f in (lib.oracle_project, lib.oracle_project_bisect, lib.oracle_project_many,
                  lib.oracle_decode, lib.oracle_lp_max, lib.oracle_decode_dual):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def project(u, bisect: bool = False) -> np.ndarray:
    """Pi_PP(u) for one vector (Algorithm 2), or by bisection when ``bisect``."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    z = np.empty_like(u)
    fn = lib.oracle_project_bisect if bisect else lib.oracle_project
    if fn(len(u), _ptr(u, ctypes.c_double), _ptr(z, ctypes.c_double)) != 0:
        raise ValueError("degree out of range")
    return z


def project_many(v: np.ndarray, bisect: bool = False) -> np.ndarray:
    """Row-wise projection of a [count x d] array."""
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    count, d = v.shape
    z = np.empty_like(v)
    if lib.oracle_project_many(d, count, _ptr(v, ctypes.c_double), _ptr(z, ctypes.c_double),
                               1 if bisect else 0) != 0:
        raise ValueError("degree out of range")
    return z


def lp_max(c) -> np.ndarray:
    """argmax_{z in PP_d} c^T z (Algorithm 3 of the appendix)."""
    lib = _load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    z = np.empty_like(c)
    if lib.oracle_lp_max(len(c), _ptr(c, ctypes.c_double), _ptr(z, ctypes.c_double)) != 0:
        raise ValueError("degree out of range")
    return z


def decode_dual(row_ptr, col_idx, n: int, gamma, mu: float = 1.0, max_iter: int = 1000,
                threads: int | None = None) -> dict:
    """Dual subgradient ascent of the appendix on every frame of ``gamma``."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    gamma = np.ascontiguousarray(np.atleast_2d(gamma), dtype=np.float64)
    F = gamma.shape[0]
    m = len(row_ptr) - 1
    x = np.zeros((F, n), dtype=np.float64)
    bits = np.zeros((F, n), dtype=np.uint8)
    iters = np.zeros(F, dtype=np.int32)
    cert = np.zeros(F, dtype=np.uint8)
    threads = max(1, min(threads or default_threads(), F))

    def run(lo: int, hi: int) -> int:
        return lib.oracle_decode_dual(
            n, m, _ptr(row_ptr, ctypes.c_int32), _ptr(col_idx, ctypes.c_int32), lo, hi,
            _ptr(gamma, ctypes.c_double), mu, max_iter, _ptr(x, ctypes.c_double), _ptr(bits, ctypes.c_uint8),
            _ptr(iters, ctypes.c_int32), _ptr(cert, ctypes.c_uint8))

    edges = np.linspace(0, F, threads + 1).astype(int)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        rc = list(ex.map(lambda t: run(int(edges[t]), int(edges[t + 1])), range(threads)))
    if any(rc):
        raise ValueError("oracle_decode_dual rejected its arguments")
    return {"x": x, "bits": bits, "iters": iters, "cert": cert}


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def decode(row_ptr, col_idx, n: int, gamma, mu: float = 3.0, rho: float = 1.9,
           eps: float = 1e-5, max_iter: int = 200, cert_tol: float = 1e-2,
           threads: int | None = None) -> dict:
    """Algorithm 1 on every frame of ``gamma`` ([frames x n]).

    Returns a dict with x (float64), bits (uint8), iters (int32),
    converged (uint8), cert (uint8), and rp, rd (float64): the primal and dual
    residuals of Section 3.3 after each frame's last iteration.
    """
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    gamma = np.ascontiguousarray(np.atleast_2d(gamma), dtype=np.float64)
    F = gamma.shape[0]
    m = len(row_ptr) - 1
    if gamma.shape[1] != n:
        raise ValueError("gamma must be [frames x n]")
    x = np.zeros((F, n), dtype=np.float64)
    bits = np.zeros((F, n), dtype=np.uint8)
    iters = np.zeros(F, dtype=np.int32)
    conv = np.zeros(F, dtype=np.uint8)
    cert = np.zeros(F, dtype=np.uint8)
    resid = np.zeros((F, 2), dtype=np.float64)
    threads = max(1, min(threads or default_threads(), F))

    def run(lo: int, hi: int) -> int:
        return lib.oracle_decode(
            n, m, _ptr(row_ptr, ctypes.c_int32), _ptr(col_idx, ctypes.c_int32), lo, hi,
            _ptr(gamma, ctypes.c_double), mu, rho, eps, max_iter, cert_tol,
            _ptr(x, ctypes.c_double), _ptr(bits, ctypes.c_uint8), _ptr(iters, ctypes.c_int32),
            _ptr(conv, ctypes.c_uint8), _ptr(cert, ctypes.c_uint8), _ptr(resid, ctypes.c_double))

    if threads == 1:
        rc = [run(0, F)]
    else:
        edges = np.linspace(0, F, threads + 1).astype(int)
        with ThreadPoolExecutor(max_workers=threads) as ex:
            rc = list(ex.map(lambda t: run(int(edges[t]), int(edges[t + 1])), range(threads)))
    if any(rc):
        raise ValueError("oracle_decode rejected its arguments")
    return {"x": x, "bits": bits, "iters": iters, "converged": conv, "cert": cert,
            "rp": resid[:, 0].copy(), "rd": resid[:, 1].copy()}
