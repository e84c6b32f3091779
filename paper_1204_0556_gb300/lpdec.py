"""Python binding of liblpdec (ctypes; argument marshalling only).

The functions named ``lpdec_*`` mirror the C-ABI of ``include/lpdec.h`` one to
one.  The helpers below them (``Code``, ``decode``, ``decode_host``,
``project``) take torch tensors for device memory and streams and call those
same entry points; every step of decoding runs in the CUDA library.  There is
no CPU fallback: if liblpdec.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblpdec.so")

LPDEC_OK = 0
LPDEC_EINVAL = -1
LPDEC_ENOMEM = -2
LPDEC_ECUDA = -3
LPDEC_ETIMEOUT = -4
LPDEC_EBUSY = -5
LPDEC_ECLOSED = -6
LPDEC_FRAME_BAD_LLR = -1
LPDEC_FRAME_ABANDONED = -2

STATE_F32, STATE_BF16, STATE_F16, STATE_Q16 = 0, 1, 2, 3
SCHED_AUTO, SCHED_STREAMED, SCHED_RESIDENT = 0, 1, 2
_DTYPES = {"f32": STATE_F32, "fp32": STATE_F32, "bf16": STATE_BF16, "f16": STATE_F16, "fp16": STATE_F16,
           "q16": STATE_Q16}
_SCHEDS = {"auto": SCHED_AUTO, "streamed": SCHED_STREAMED, "resident": SCHED_RESIDENT}

# Every symbol include/lpdec.h declares (checked by the CPU test suite).
EXPORTED = [
    "lpdec_params_default", "lpdec_last_error", "lpdec_version",
    "lpdec_code_create", "lpdec_code_info", "lpdec_code_destroy",
    "lpdec_decode", "lpdec_decode_host", "lpdec_project", "lpdec_decode_noalloc",
    "lpdec_decode_mixed",
    "lpdec_server_create", "lpdec_server_add_code", "lpdec_server_submit", "lpdec_server_poll",
    "lpdec_server_stats", "lpdec_server_destroy", "lpdec_autotune", "lpdec_set_tile", "lpdec_server_counters",
    "lpdec_mixed_plan_create", "lpdec_mixed_plan_decode", "lpdec_mixed_plan_destroy",
    "lpdec_decode_dual", "lpdec_dual_set_tile", "lpdec_set_streamed_tile", "lpdec_get_tile",
    "lpdec_release_memory", "lpdec_set_wait_limit",
]


class LpdecError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"liblpdec status {status}: {msg}")
        self.status = status


class lpdec_params(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("state_dtype", ctypes.c_int32),
        ("cert_tol", ctypes.c_double),
        ("schedule", ctypes.c_int32),
        ("iters_per_launch", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_i32p = ctypes.POINTER(ctypes.c_int32)


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load liblpdec.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"liblpdec.so not found at {p}; run paper_1204_0556_gb300.build.build() first")
        lib = ctypes.CDLL(p)
        P = ctypes.POINTER(lpdec_params)
        sig = {
            "lpdec_params_default": (None, [P]),
            "lpdec_last_error": (ctypes.c_char_p, []),
            "lpdec_version": (ctypes.c_char_p, []),
            "lpdec_code_create": (ctypes.c_int, [_i32, _i32, _i32p, _i32p, _i32p, _i32p, _i32p, ctypes.POINTER(_vp)]),
            "lpdec_code_info": (ctypes.c_int, [_vp, _i32p, _i32p, ctypes.POINTER(_i64), _i32p, _i32p]),
            "lpdec_code_destroy": (ctypes.c_int, [_vp]),
            "lpdec_decode": (ctypes.c_int, [_vp, _i32, _vp, P, _vp, _vp, _vp, _vp, _vp]),
            "lpdec_decode_host": (ctypes.c_int, [_vp, _i32, _vp, P, _vp, _vp, _vp, _vp, _vp]),
            "lpdec_project": (ctypes.c_int, [_i32, _i64, _vp, _vp, _vp]),
            "lpdec_decode_noalloc": (ctypes.c_int, [_vp, _i32, _vp, P, _vp, _vp, _vp, _vp, _vp]),
            "lpdec_decode_mixed": (ctypes.c_int, [ctypes.POINTER(_vp), _i32, _i32, _i32p, _vp, P, _vp, _vp, _vp,
                                                  _vp, _vp]),
        }
        u64p = ctypes.POINTER(ctypes.c_uint64)
        dp = ctypes.POINTER(ctypes.c_double)
        sig.update({
            "lpdec_server_create": (ctypes.c_int, [ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
            "lpdec_server_add_code": (ctypes.c_int, [_vp, _vp, _i32p]),
            "lpdec_server_submit": (ctypes.c_int, [_vp, _i32, _i32, _vp, P, u64p]),
            "lpdec_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _i32, _vp, _vp, _vp, _vp]),
            "lpdec_server_stats": (ctypes.c_int, [_vp, dp, dp, dp, ctypes.POINTER(_i64)]),
            "lpdec_server_destroy": (ctypes.c_int, [_vp]),
            "lpdec_server_counters": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), dp, dp]),
            "lpdec_autotune": (ctypes.c_int, [_vp, P, _i32, _vp, _vp, _i32p, _i32p, dp]),
            "lpdec_set_tile": (ctypes.c_int, [_vp, _i32, _i32, _i32]),
            "lpdec_mixed_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i32, _i32, _i32p, P,
                                                       ctypes.POINTER(_vp)]),
            "lpdec_mixed_plan_decode": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
            "lpdec_mixed_plan_destroy": (ctypes.c_int, [_vp]),
            "lpdec_decode_dual": (ctypes.c_int, [_vp, _i32, _vp, ctypes.c_double, _i32, _vp, _vp, _vp, _vp, _vp]),
            "lpdec_dual_set_tile": (ctypes.c_int, [_vp, _i32, _i32]),
            "lpdec_set_streamed_tile": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32]),
            "lpdec_get_tile": (ctypes.c_int, [_vp, _i32, _i32, _i32p, _i32p, _i32p]),
            "lpdec_release_memory": (ctypes.c_int, []),
            "lpdec_set_wait_limit": (ctypes.c_int, [_i64]),
        })
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int) -> None:
    if status != LPDEC_OK:
        raise LpdecError(status, load().lpdec_last_error().decode())


# ---- thin C-ABI mirrors -------------------------------------------------------

def lpdec_params_default() -> lpdec_params:
    p = lpdec_params()
    load().lpdec_params_default(ctypes.byref(p))
    return p


def lpdec_last_error() -> str:
    return load().lpdec_last_error().decode()


def lpdec_version() -> str:
    return load().lpdec_version().decode()


def _i32arr(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def lpdec_code_create(n, m, row_ptr, col_idx, col_ptr, row_idx, edge_perm) -> int:
    arrs = [_i32arr(a) for a in (row_ptr, col_idx, col_ptr, row_idx, edge_perm)]
    out = _vp()
    _check(load().lpdec_code_create(n, m, *[a.ctypes.data_as(_i32p) for a in arrs], ctypes.byref(out)))
    return out.value


def lpdec_code_info(handle: int) -> dict:
    n, m, mx, kr = _i32(), _i32(), _i32(), _i32()
    E = _i64()
    _check(load().lpdec_code_info(handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(E),
                                  ctypes.byref(mx), ctypes.byref(kr)))
    return {"n": n.value, "m": m.value, "E": E.value, "max_dc": mx.value, "k_rank": kr.value}


def lpdec_code_destroy(handle: int) -> None:
    _check(load().lpdec_code_destroy(handle))


def lpdec_decode(handle, n_frames, llr_ptr, params, x_ptr, bits_ptr, iters_ptr, cert_ptr, stream_ptr) -> None:
    _check(load().lpdec_decode(handle, n_frames, llr_ptr, ctypes.byref(params), x_ptr, bits_ptr, iters_ptr,
                               cert_ptr, stream_ptr))


def lpdec_decode_host(handle, n_frames, llr_ptr, params, x_ptr, bits_ptr, iters_ptr, cert_ptr, stream_ptr) -> None:
    _check(load().lpdec_decode_host(handle, n_frames, llr_ptr, ctypes.byref(params), x_ptr, bits_ptr, iters_ptr,
                                    cert_ptr, stream_ptr))


def lpdec_decode_noalloc(handle, n_frames, llr_ptr, params, x_ptr, bits_ptr, iters_ptr, cert_ptr,
                         stream_ptr) -> None:
    """lpdec_decode with scratch in the library's fixed device array: no allocation
    during the call (for callers that cannot allocate device memory as they run)."""
    _check(load().lpdec_decode_noalloc(handle, n_frames, llr_ptr, ctypes.byref(params), x_ptr, bits_ptr,
                                       iters_ptr, cert_ptr, stream_ptr))


def lpdec_decode_mixed(handles, n_frames, frame_code, llr_ptr, params, x_ptr, bits_ptr, iters_ptr, cert_ptr,
                       stream_ptr) -> None:
    arr = (_vp * len(handles))(*handles)
    fc = _i32arr(frame_code)
    _check(load().lpdec_decode_mixed(arr, len(handles), n_frames, fc.ctypes.data_as(_i32p), llr_ptr,
                                     ctypes.byref(params), x_ptr, bits_ptr, iters_ptr, cert_ptr, stream_ptr))


def lpdec_server_create(budget_bytes: int, stream_ptr: int = 0) -> int:
    out = _vp()
    _check(load().lpdec_server_create(budget_bytes, stream_ptr, ctypes.byref(out)))
    return out.value


def lpdec_server_add_code(server: int, code_handle: int) -> int:
    cid = _i32()
    _check(load().lpdec_server_add_code(server, code_handle, ctypes.byref(cid)))
    return cid.value


def lpdec_server_submit(server: int, code_id: int, n_frames: int, llr_ptr: int, params) -> int:
    rid = ctypes.c_uint64()
    _check(load().lpdec_server_submit(server, code_id, n_frames, llr_ptr, ctypes.byref(params), ctypes.byref(rid)))
    return rid.value


def lpdec_server_poll(server: int, request_id: int, timeout_ms: int, x_ptr, bits_ptr, iters_ptr, cert_ptr) -> int:
    """Returns the status (LPDEC_OK or LPDEC_ETIMEOUT); other errors raise."""
    st = load().lpdec_server_poll(server, request_id, timeout_ms, x_ptr, bits_ptr, iters_ptr, cert_ptr)
    if st not in (LPDEC_OK, LPDEC_ETIMEOUT):
        _check(st)
    return st


def lpdec_server_stats(server: int) -> dict:
    p50, p99, bps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    fr = _i64()
    _check(load().lpdec_server_stats(server, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(bps),
                                     ctypes.byref(fr)))
    return {"p50_ms": p50.value, "p99_ms": p99.value, "bits_per_s": bps.value, "frames": fr.value}


def lpdec_server_counters(server: int) -> dict:
    r = _i64()
    w, g = ctypes.c_double(), ctypes.c_double()
    _check(load().lpdec_server_counters(server, ctypes.byref(r), ctypes.byref(w), ctypes.byref(g)))
    return {"rounds": r.value, "round_wall_ms": w.value, "round_gpu_ms": g.value}


def lpdec_server_destroy(server: int) -> None:
    _check(load().lpdec_server_destroy(server))


def lpdec_autotune(handle: int, params, n_frames: int, llr_ptr: int, stream_ptr: int) -> dict:
    gt, g = _i32(), _i32()
    ms = ctypes.c_double()
    _check(load().lpdec_autotune(handle, ctypes.byref(params), n_frames, llr_ptr, stream_ptr, ctypes.byref(gt),
                                 ctypes.byref(g), ctypes.byref(ms)))
    ring = 0
    if params.schedule == SCHED_STREAMED:
        ring = lpdec_get_tile(handle, params.state_dtype, SCHED_STREAMED)["ring_slots"]
    return {"group_threads": gt.value, "groups": g.value, "ring_slots": ring, "ms_per_frame": ms.value}


def lpdec_set_tile(handle: int, state_dtype: int, group_threads: int, groups: int) -> None:
    _check(load().lpdec_set_tile(handle, state_dtype, group_threads, groups))


def lpdec_set_streamed_tile(handle: int, state_dtype: int, group_threads: int, groups: int,
                            ring_slots: int = 0) -> None:
    _check(load().lpdec_set_streamed_tile(handle, state_dtype, group_threads, groups, ring_slots))


def lpdec_release_memory() -> None:
    _check(load().lpdec_release_memory())


def lpdec_set_wait_limit(clocks: int) -> None:
    """Limit (SM clocks) of a STREAMED launch's first wait on a copy or a ring
    slot; clocks <= 0 restores the default (2^31)."""
    _check(load().lpdec_set_wait_limit(int(clocks)))


def lpdec_get_tile(handle: int, state_dtype: int, schedule: int) -> dict:
    gt, g, r = _i32(), _i32(), _i32()
    _check(load().lpdec_get_tile(handle, state_dtype, schedule, ctypes.byref(gt), ctypes.byref(g), ctypes.byref(r)))
    return {"group_threads": gt.value, "groups": g.value, "ring_slots": r.value}


def lpdec_mixed_plan_create(handles, frame_code, params) -> int:
    arr = (_vp * len(handles))(*handles)
    fc = _i32arr(frame_code)
    out = _vp()
    _check(load().lpdec_mixed_plan_create(arr, len(handles), len(fc), fc.ctypes.data_as(_i32p), ctypes.byref(params),
                                          ctypes.byref(out)))
    return out.value


def lpdec_mixed_plan_decode(plan, llr_ptr, x_ptr, bits_ptr, iters_ptr, cert_ptr, stream_ptr) -> None:
    _check(load().lpdec_mixed_plan_decode(plan, llr_ptr, x_ptr, bits_ptr, iters_ptr, cert_ptr, stream_ptr))


def lpdec_mixed_plan_destroy(plan) -> None:
    _check(load().lpdec_mixed_plan_destroy(plan))


def lpdec_project(d, count, v_ptr, z_ptr, stream_ptr) -> None:
    _check(load().lpdec_project(d, count, v_ptr, z_ptr, stream_ptr))


def lpdec_decode_dual(handle, n_frames, llr_ptr, mu, max_iter, x_ptr, bits_ptr, iters_ptr, cert_ptr,
                      stream_ptr) -> None:
    _check(load().lpdec_decode_dual(handle, n_frames, llr_ptr, float(mu), int(max_iter), x_ptr, bits_ptr,
                                    iters_ptr, cert_ptr, stream_ptr))


def lpdec_dual_set_tile(handle: int, group_threads: int, groups: int) -> None:
    _check(load().lpdec_dual_set_tile(handle, group_threads, groups))


# ---- convenience layer (torch tensors) ---------------------------------------

def make_params(mu=3.0, rho=1.9, eps=1e-5, max_iter=1000, state="f32", cert_tol=1e-2,
                schedule="auto", iters_per_launch=1) -> lpdec_params:
    p = lpdec_params_default()
    p.mu, p.rho, p.eps, p.max_iter = float(mu), float(rho), float(eps), int(max_iter)
    p.state_dtype = _DTYPES[state] if isinstance(state, str) else int(state)
    p.cert_tol = float(cert_tol)
    p.schedule = _SCHEDS[schedule] if isinstance(schedule, str) else int(schedule)
    p.iters_per_launch = int(iters_per_launch)
    return p


class Code:
    """A parity-check matrix uploaded to the current CUDA device."""

    def __init__(self, code):
        self.src = code
        self.handle = lpdec_code_create(code.n, code.m, code.row_ptr, code.col_idx, code.col_ptr,
                                        code.row_idx, code.edge_perm)
        self.info = lpdec_code_info(self.handle)
        self.n, self.m = code.n, code.m

    def close(self):
        if self.handle:
            lpdec_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def decode(code: Code, llr, params: lpdec_params | None = None, stream=None, out: dict | None = None) -> dict:
    """Decode a [frames x n] float32 CUDA tensor; returns CUDA tensors x, bits, iters, cert."""
    import torch

    if not (llr.is_cuda and llr.dtype == torch.float32 and llr.is_contiguous()):
        raise ValueError("llr must be a contiguous float32 CUDA tensor")
    F = llr.shape[0]
    if llr.shape[1] != code.n:
        raise ValueError("llr must be [frames x n]")
    params = params or make_params()
    if out is None:
        out = {
            "x": torch.empty((F, code.n), dtype=torch.float32, device=llr.device),
            "bits": torch.empty((F, code.n), dtype=torch.uint8, device=llr.device),
            "iters": torch.empty((F,), dtype=torch.int32, device=llr.device),
            "cert": torch.empty((F,), dtype=torch.uint8, device=llr.device),
        }
    lpdec_decode(code.handle, F, llr.data_ptr(), params, out["x"].data_ptr(), out["bits"].data_ptr(),
                 out["iters"].data_ptr(), out["cert"].data_ptr(), _stream_ptr(stream))
    return out


def decode_host(code: Code, llr: np.ndarray, params: lpdec_params | None = None, stream=None,
                out: dict | None = None) -> dict:
    """Decode host LLRs (numpy float32 [frames x n]); copies happen inside the call."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    F = llr.shape[0]
    params = params or make_params()
    if out is None:
        out = {"x": np.empty((F, code.n), np.float32), "bits": np.empty((F, code.n), np.uint8),
               "iters": np.empty(F, np.int32), "cert": np.empty(F, np.uint8)}
    lpdec_decode_host(code.handle, F, llr.ctypes.data, params, out["x"].ctypes.data, out["bits"].ctypes.data,
                      out["iters"].ctypes.data, out["cert"].ctypes.data, _stream_ptr(stream))
    return out


def decode_mixed(codes: list, frame_code, llr, params: lpdec_params | None = None, stream=None,
                 out: dict | None = None) -> dict:
    """Decode a packed batch of frames of several codes in one persistent launch.

    ``llr`` is a 1-D float32 CUDA tensor with the frames back to back in frame
    order; ``frame_code`` (host ints) gives each frame's index into ``codes``."""
    import torch

    fc = np.ascontiguousarray(frame_code, dtype=np.int32)
    F = len(fc)
    total = int(sum(codes[c].n for c in fc))
    if not (llr.is_cuda and llr.dtype == torch.float32 and llr.is_contiguous() and llr.numel() == total):
        raise ValueError("llr must be a contiguous float32 CUDA tensor of sum(n) elements")
    params = params or make_params()
    if out is None:
        out = {"x": torch.empty(total, dtype=torch.float32, device=llr.device),
               "bits": torch.empty(total, dtype=torch.uint8, device=llr.device),
               "iters": torch.empty(F, dtype=torch.int32, device=llr.device),
               "cert": torch.empty(F, dtype=torch.uint8, device=llr.device)}
    lpdec_decode_mixed([c.handle for c in codes], F, fc, llr.data_ptr(), params, out["x"].data_ptr(),
                       out["bits"].data_ptr(), out["iters"].data_ptr(), out["cert"].data_ptr(), _stream_ptr(stream))
    return out


class Server:
    """Continuous-batching decode server (thin wrapper over lpdec_server_*)."""

    def __init__(self, budget_bytes: int = 8 << 30, stream=None):
        self.handle = lpdec_server_create(budget_bytes, 0 if stream is None else int(stream.cuda_stream))
        self.codes = []

    def add_code(self, code: Code) -> int:
        self.codes.append(code)
        return lpdec_server_add_code(self.handle, code.handle)

    def submit(self, code_id: int, llr: np.ndarray, params: lpdec_params) -> int:
        llr = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float32)
        return lpdec_server_submit(self.handle, code_id, llr.shape[0], llr.ctypes.data, params)

    def poll(self, request_id: int, code_id: int, n_frames: int = 1, timeout_ms: int = -1):
        n = self.codes[code_id].n
        out = {"x": np.empty((n_frames, n), np.float32), "bits": np.empty((n_frames, n), np.uint8),
               "iters": np.empty(n_frames, np.int32), "cert": np.empty(n_frames, np.uint8)}
        st = lpdec_server_poll(self.handle, request_id, timeout_ms, out["x"].ctypes.data, out["bits"].ctypes.data,
                               out["iters"].ctypes.data, out["cert"].ctypes.data)
        return out if st == LPDEC_OK else None

    def stats(self) -> dict:
        return lpdec_server_stats(self.handle)

    def counters(self) -> dict:
        return lpdec_server_counters(self.handle)

    def close(self):
        if self.handle:
            lpdec_server_destroy(self.handle)
            self.handle = None


def decode_dual(code: Code, llr, mu: float = 0.25, max_iter: int = 5000, stream=None,
                out: dict | None = None) -> dict:
    """Dual subgradient decoding (appendix) of a [frames x n] float32 CUDA
    tensor; returns CUDA tensors x, bits, iters, cert."""
    import torch

    if not (llr.is_cuda and llr.dtype == torch.float32 and llr.is_contiguous()):
        raise ValueError("llr must be a contiguous float32 CUDA tensor")
    F = llr.shape[0]
    if llr.shape[1] != code.n:
        raise ValueError("llr must be [frames x n]")
    if out is None:
        out = {
            "x": torch.empty((F, code.n), dtype=torch.float32, device=llr.device),
            "bits": torch.empty((F, code.n), dtype=torch.uint8, device=llr.device),
            "iters": torch.empty((F,), dtype=torch.int32, device=llr.device),
            "cert": torch.empty((F,), dtype=torch.uint8, device=llr.device),
        }
    lpdec_decode_dual(code.handle, F, llr.data_ptr(), mu, max_iter, out["x"].data_ptr(), out["bits"].data_ptr(),
                      out["iters"].data_ptr(), out["cert"].data_ptr(), _stream_ptr(stream))
    return out


def project(v, stream=None):
    """Row-wise projection onto PP_d of a [count x d] float32 CUDA tensor."""
    import torch

    if not (v.is_cuda and v.dtype == torch.float32 and v.is_contiguous() and v.dim() == 2):
        raise ValueError("v must be a contiguous [count x d] float32 CUDA tensor")
    z = torch.empty_like(v)
    lpdec_project(v.shape[1], v.shape[0], v.data_ptr(), z.data_ptr(), _stream_ptr(stream))
    return z
