"""ctypes binding of the C ABI in include/sosfilt.h (argument marshalling only).

Every function keeps the C name and argument order; pointers are passed as
integers (``tensor.data_ptr()``), streams as the raw cudaStream_t handle.
Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import buildlib as _build

_lock = threading.Lock()
_lib = None

SOS_OK = 0
SOS_FLAG_CHECK_STABLE = 1
SOS_FLAG_CARRY_ONLY = 2
SOS_FLAG_SECTION_PIPELINE = 4
SOS_FLAG_REPLAN = 8
SOS_FLAG_DOUBLE_FLOAT = 16


def SOS_FLAG_WS_CTAS(n: int) -> int:  # noqa: N802 - the C macro's name
    return (int(n) & 15) << 8


SOS_MAX_SECTIONS = 8

STATUS_NAMES = {
    0: "SOS_OK", -1: "SOS_ERR_ARG", -2: "SOS_ERR_UNSTABLE", -3: "SOS_ERR_CUDA",
    -4: "SOS_ERR_TIMEOUT", -5: "SOS_ERR_WORKSPACE", -6: "SOS_ERR_UNSUPPORTED", -7: "SOS_ERR_COEF",
}


class SosError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class sos_tuning(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("algo", ctypes.c_int32), ("flags", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded library.  Raises if it has not been built (call
    ``paper_2607_14054_gb300.build.build()`` / ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"CUDA library not built: {path} is missing; run "
                                   "paper_2607_14054_gb300.build.build() first")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        tp = ctypes.POINTER(sos_tuning)
        lib.sos_abi_version.argtypes = []
        lib.sos_abi_version.restype = i32
        lib.sos_status_str.argtypes = [ctypes.c_int]
        lib.sos_status_str.restype = ctypes.c_char_p
        lib.sos_workspace_size.argtypes = [i32, i32, vp, tp]
        lib.sos_workspace_size.restype = sz
        lib.sos_workspace_init.argtypes = [vp, sz, vp]
        lib.sos_workspace_init.restype = ctypes.c_int
        lib.sos_filter.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, sz, tp, vp]
        lib.sos_filter.restype = ctypes.c_int
        lib.sos_prepare.argtypes = [vp, vp, i32, i32, vp, vp, vp, sz, tp, vp]
        lib.sos_prepare.restype = ctypes.c_int
        lib.sos_apply.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, sz, tp, vp]
        lib.sos_apply.restype = ctypes.c_int
        for fn in (lib.sos_apply_pipeline, lib.sos_apply_carried):
            fn.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, sz, tp, vp]
            fn.restype = ctypes.c_int
        lib.sos_filter_static.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, tp, vp,
                                          ctypes.POINTER(ctypes.c_int32)]
        lib.sos_filter_static.restype = ctypes.c_int
        lib.sos_apply_baseline.argtypes = [i32, vp, i32, i32, vp, vp, vp, vp, i64, vp, sz, tp, vp]
        lib.sos_apply_baseline.restype = ctypes.c_int
        lib.sos_filtfilt.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, sz, tp, vp]
        lib.sos_filtfilt.restype = ctypes.c_int
        lib.sos_stream.argtypes = [vp, vp, vp, vp, i32, i32, i64, ctypes.c_uint32, vp, sz, tp,
                                   vp]
        lib.sos_stream.restype = ctypes.c_int
        lib.sos_filter_host_sizes.argtypes = [i32, i32, vp, i64, tp, vp, vp, vp]
        lib.sos_filter_host_sizes.restype = ctypes.c_int
        lib.sos_filter_host.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, sz, vp, sz,
                                        i64, tp, vp]
        lib.sos_filter_host.restype = ctypes.c_int
        lib.sos_device_status.argtypes = [vp, vp]
        lib.sos_device_status.restype = ctypes.c_int
        lib.sos_backward_workspace_size.argtypes = [i32, i32, vp, tp]
        lib.sos_backward_workspace_size.restype = sz
        lib.sos_filter_backward.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                            vp, sz, tp, vp]
        lib.sos_filter_backward.restype = ctypes.c_int
        lib.sos_plan_query.argtypes = [vp, i32, i32, vp, vp, vp]
        lib.sos_plan_query.restype = ctypes.c_int
        lib.sos_plan_extended.argtypes = [vp, i32, i32, vp, vp]
        lib.sos_plan_extended.restype = ctypes.c_int
        lib.sos_workspace_set_wait_limit.argtypes = [vp, ctypes.c_uint32, vp]
        lib.sos_workspace_set_wait_limit.restype = ctypes.c_int
        lib.sos_plan_recomputed.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), vp]
        lib.sos_plan_recomputed.restype = ctypes.c_int
        _lib = lib
        return lib


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, sos_tuning):
        return ctypes.byref(t)
    n, w, a, f = (list(t) + [0, 0, 0, 0])[:4]
    return ctypes.byref(sos_tuning(int(n), int(w), int(a), int(f)))


def sos_workspace_size(n_channels: int, kmax: int, lengths_host_ptr: int, tuning=None) -> int:
    return int(load().sos_workspace_size(n_channels, kmax, ctypes.c_void_p(lengths_host_ptr),
                                         _tuning(tuning)))


def sos_workspace_init(ws_ptr: int, ws_bytes: int, stream: int) -> int:
    return int(load().sos_workspace_init(ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream)))


def sos_filter(x, sos, K, n_channels, kmax, lengths, lengths_host, zi, y, zf, ws, ws_bytes,
               tuning, stream) -> int:
    """All pointer arguments are integers (0 for NULL)."""
    V = ctypes.c_void_p
    return int(load().sos_filter(V(x), V(sos), V(K), n_channels, kmax, V(lengths), V(lengths_host),
                                 V(zi or None), V(y), V(zf or None), V(ws), ws_bytes,
                                 _tuning(tuning), V(stream)))


def sos_filter_host_sizes(n_channels, kmax, lengths_host, block, tuning):
    """(status, workspace bytes, staging bytes, block used)."""
    ws = ctypes.c_size_t(0)
    stg = ctypes.c_size_t(0)
    blk = ctypes.c_int64(0)
    st = int(load().sos_filter_host_sizes(n_channels, kmax, ctypes.c_void_p(lengths_host),
                                          int(block), _tuning(tuning), ctypes.byref(ws),
                                          ctypes.byref(stg), ctypes.byref(blk)))
    return st, ws.value, stg.value, blk.value


def sos_filter_host(x_host, sos, K, n_channels, kmax, lengths, lengths_host, zi, y_host, zf, ws,
                    ws_bytes, staging, staging_bytes, block, tuning, stream) -> int:
    """All pointer arguments are integers (0 for NULL); x_host, y_host host."""
    V = ctypes.c_void_p
    return int(load().sos_filter_host(V(x_host), V(sos), V(K), n_channels, kmax, V(lengths),
                                      V(lengths_host), V(zi or None), V(y_host), V(zf or None),
                                      V(ws), ws_bytes, V(staging), staging_bytes, int(block),
                                      _tuning(tuning), V(stream)))


def sos_prepare(sos, K, n_channels, kmax, lengths, lengths_host, ws, ws_bytes, tuning,
                stream) -> int:
    V = ctypes.c_void_p
    return int(load().sos_prepare(V(sos), V(K), n_channels, kmax, V(lengths), V(lengths_host),
                                  V(ws), ws_bytes, _tuning(tuning), V(stream)))


def sos_apply(x, n_channels, kmax, lengths_host, zi, y, zf, ws, ws_bytes, tuning, stream) -> int:
    V = ctypes.c_void_p
    return int(load().sos_apply(V(x), n_channels, kmax, V(lengths_host), V(zi or None), V(y),
                                V(zf or None), V(ws), ws_bytes, _tuning(tuning), V(stream)))


def sos_apply_part(part: str, x, n_channels, kmax, lengths_host, zi, y, zf, ws, ws_bytes,
                   tuning, stream) -> int:
    """part: "pipeline" or "carried"; pointer arguments are integers."""
    V = ctypes.c_void_p
    fn = load().sos_apply_pipeline if part == "pipeline" else load().sos_apply_carried
    return int(fn(V(x), n_channels, kmax, V(lengths_host), V(zi or None), V(y), V(zf or None),
                  V(ws), ws_bytes, _tuning(tuning), V(stream)))


def sos_filter_static(x, sos, K, n_channels, kmax, lengths, lengths_host, zi, y, zf, tuning,
                      stream, want_status: bool = True):
    """Returns (status, device_status or None)."""
    V = ctypes.c_void_p
    ds = ctypes.c_int32(0)
    st = int(load().sos_filter_static(V(x), V(sos), V(K), n_channels, kmax, V(lengths),
                                      V(lengths_host), V(zi or None), V(y), V(zf or None),
                                      _tuning(tuning), V(stream),
                                      ctypes.byref(ds) if want_status else None))
    return st, (int(ds.value) if want_status else None)


def sos_apply_baseline(algorithm, x, n_channels, kmax, lengths_host, zi, y, zf, seg_len, ws,
                       ws_bytes, tuning, stream) -> int:
    """algorithm 0 = scalar, 1 = block filtering; pointers as integers."""
    V = ctypes.c_void_p
    return int(load().sos_apply_baseline(int(algorithm), V(x), n_channels, kmax, V(lengths_host),
                                         V(zi or None), V(y), V(zf or None), int(seg_len), V(ws),
                                         ws_bytes, _tuning(tuning), V(stream)))


def sos_filtfilt(x, sos, K, n_channels, kmax, lengths, lengths_host, y, tmp, ws, ws_bytes, tuning,
                 stream) -> int:
    """All pointer arguments are integers."""
    V = ctypes.c_void_p
    return int(load().sos_filtfilt(V(x), V(sos), V(K), n_channels, kmax, V(lengths),
                                   V(lengths_host), V(y), V(tmp), V(ws), ws_bytes, _tuning(tuning),
                                   V(stream)))


SOS_STREAM_FOREIGN_STATE = 1


def sos_stream(x, y, zi, zf, n_channels, kmax, chunk, flags, ws, ws_bytes, tuning,
               stream) -> int:
    """All pointer arguments are integers (0 for NULL)."""
    V = ctypes.c_void_p
    return int(load().sos_stream(V(x), V(y), V(zi or None), V(zf or None), n_channels, kmax,
                                 int(chunk), int(flags), V(ws), ws_bytes, _tuning(tuning),
                                 V(stream)))


def sos_device_status(ws_ptr: int, stream: int) -> int:
    return int(load().sos_device_status(ctypes.c_void_p(ws_ptr), ctypes.c_void_p(stream)))


def sos_backward_workspace_size(n_channels: int, kmax: int, lengths_host_ptr: int,
                                tuning=None) -> int:
    return int(load().sos_backward_workspace_size(n_channels, kmax,
                                                  ctypes.c_void_p(lengths_host_ptr),
                                                  _tuning(tuning)))


def sos_filter_backward(x, sos, K, n_channels, kmax, lengths, lengths_host, zi, grad_y, grad_zf,
                        grad_x, grad_sos, grad_zi, ws, ws_bytes, tuning, stream) -> int:
    """All pointer arguments are integers (0 for NULL)."""
    V = ctypes.c_void_p
    return int(load().sos_filter_backward(V(x), V(sos), V(K), n_channels, kmax, V(lengths),
                                          V(lengths_host), V(zi or None), V(grad_y),
                                          V(grad_zf or None), V(grad_x), V(grad_sos),
                                          V(grad_zi or None), V(ws), ws_bytes, _tuning(tuning),
                                          V(stream)))


def sos_plan_query(ws_ptr: int, first: int, count: int, horizon_ptr: int, tiles_ptr: int,
                   stream: int) -> int:
    """Host pointers are integers (0 for NULL)."""
    V = ctypes.c_void_p
    return int(load().sos_plan_query(V(ws_ptr), first, count, V(horizon_ptr or None),
                                     V(tiles_ptr or None), V(stream)))


def sos_plan_extended(ws_ptr: int, first: int, count: int, extended_ptr: int,
                      stream: int) -> int:
    """Host pointer as an integer."""
    V = ctypes.c_void_p
    return int(load().sos_plan_extended(V(ws_ptr), first, count, V(extended_ptr), V(stream)))


def sos_workspace_set_wait_limit(ws_ptr: int, limit: int, stream: int) -> int:
    return int(load().sos_workspace_set_wait_limit(ctypes.c_void_p(ws_ptr), int(limit),
                                                   ctypes.c_void_p(stream)))


def sos_plan_recomputed(ws_ptr: int, stream: int):
    """Returns (status, channels recomputed by the latest plan)."""
    n = ctypes.c_int32(0)
    st = int(load().sos_plan_recomputed(ctypes.c_void_p(ws_ptr), ctypes.byref(n),
                                        ctypes.c_void_p(stream)))
    return st, int(n.value)


def sos_status_str(status: int) -> str:
    return load().sos_status_str(status).decode()


def sos_abi_version() -> int:
    return int(load().sos_abi_version())
