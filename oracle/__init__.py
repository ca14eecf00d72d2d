"""FP64 CPU oracle for cascaded biquad filtering.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2607_14054_gb300``) never imports, links or executes it, and the two
share no code.

The oracle is the plain definition of the result, written out sample by
sample in FP64 (paper Sec. II, Eq. general_cascaded_equation and
Eq. complex_second_order; Sec. III shows that solving the banded
block-Toeplitz system of Eq. recursive_equation_block_form by forward
substitution is exactly this recurrence).  The paper's method is exact and
direct, so its result is this definition up to rounding order.

The heavy loops live in ``sosfilt_oracle.c`` (plain C, built by :func:`build`
with gcc, OpenMP over independent channels).  This module is a ctypes wrapper
plus the small helpers the pins need.

Pins (tests/test_oracle_pins.py) tie it to things other than itself: the
closed-form biquad impulse response from its poles, the cascade impulse
response as a convolution of section responses, the DFT of a long impulse
response against H(e^jw), a dense solve of the paper's Toeplitz system and of
its stride-N permuted block form on tiny inputs, zero-input and step-input
closed forms, scipy.signal.sosfilt, and a dot-product plus finite-difference
check of the adjoint.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sosfilt_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags: no -march, no intrinsics)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lp = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_sosfilt.argtypes = [dp, dp, ip, ctypes.c_int32, ctypes.c_int32, lp, dp, dp, dp]
    lib.oracle_sosfilt.restype = ctypes.c_int
    lib.oracle_sosfilt_adjoint.argtypes = [dp, dp, ip, ctypes.c_int32, ctypes.c_int32, lp,
                                           dp, dp, dp, dp, dp, dp]
    lib.oracle_sosfilt_adjoint.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _prep(x, sos, K, lengths, zi):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    sos = np.ascontiguousarray(sos, dtype=np.float64)
    if sos.ndim == 2:
        sos = sos[None]
    C, kmax, six = sos.shape
    assert six == 6
    if lengths is None:
        lengths = np.array([x.size], dtype=np.int64)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64).reshape(-1)
    assert lengths.size == C, (lengths.size, C)
    assert int(lengths.sum()) == x.size
    if K is None:
        K = np.full(C, kmax, dtype=np.int32)
    K = np.ascontiguousarray(K, dtype=np.int32).reshape(-1)
    if zi is not None:
        zi = np.ascontiguousarray(zi, dtype=np.float64).reshape(C, kmax, 2)
    return x, sos, K, lengths, zi, C, kmax


class Oracle:
    """The oracle bound to one compiled library (the default one, or a test's
    deliberately broken copy)."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(path)

    def num_threads(self) -> int:
        return int(self.lib.oracle_num_threads())

    def sosfilt(self, x, sos, K=None, lengths=None, zi=None):
        """Cascade filter, FP64.  Returns (y, zf) with y packed like x and
        zf shaped [C, kmax, 2].

        x: packed samples of all channels (any float dtype; promoted exactly).
        sos: [C, kmax, 6] or [kmax, 6] rows (b0, b1, b2, a0, a1, a2).
        K: sections used per channel (default kmax).  lengths: per channel.
        zi: [C, kmax, 2] transposed-direct-form-II initial state (None = 0).
        """
        x, sos, K, lengths, zi, C, kmax = _prep(x, sos, K, lengths, zi)
        y = np.empty_like(x)
        zf = np.empty((C, kmax, 2), dtype=np.float64)
        rc = self.lib.oracle_sosfilt(_ptr(x, ctypes.c_double), _ptr(sos, ctypes.c_double),
                                     _ptr(K, ctypes.c_int32), C, kmax,
                                     _ptr(lengths, ctypes.c_int64), _ptr(zi, ctypes.c_double),
                                     _ptr(y, ctypes.c_double), _ptr(zf, ctypes.c_double))
        if rc != 0:
            raise ValueError("oracle_sosfilt: bad arguments")
        return y, zf

    def sosfilt_adjoint(self, x, sos, g_y, K=None, lengths=None, zi=None, g_zf=None):
        """Reverse-mode gradients of L(y, zf) given g_y = dL/dy, g_zf = dL/dzf.
        Returns (g_x, g_sos, g_zi); g_sos covers the raw rows including a0."""
        x, sos, K, lengths, zi, C, kmax = _prep(x, sos, K, lengths, zi)
        g_y = np.ascontiguousarray(g_y, dtype=np.float64).reshape(-1)
        assert g_y.size == x.size
        if g_zf is not None:
            g_zf = np.ascontiguousarray(g_zf, dtype=np.float64).reshape(C, kmax, 2)
        g_x = np.empty_like(x)
        g_sos = np.empty((C, kmax, 6), dtype=np.float64)
        g_zi = np.empty((C, kmax, 2), dtype=np.float64)
        rc = self.lib.oracle_sosfilt_adjoint(
            _ptr(x, ctypes.c_double), _ptr(sos, ctypes.c_double), _ptr(K, ctypes.c_int32),
            C, kmax, _ptr(lengths, ctypes.c_int64), _ptr(zi, ctypes.c_double),
            _ptr(g_y, ctypes.c_double), _ptr(g_zf, ctypes.c_double),
            _ptr(g_x, ctypes.c_double), _ptr(g_sos, ctypes.c_double), _ptr(g_zi, ctypes.c_double))
        if rc != 0:
            raise ValueError("oracle_sosfilt_adjoint: bad arguments")
        return g_x, g_sos, g_zi


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
        return _lib


def num_threads() -> int:
    return default().num_threads()


def sosfilt(x, sos, K=None, lengths=None, zi=None):
    """See :meth:`Oracle.sosfilt`."""
    return default().sosfilt(x, sos, K, lengths, zi)


def sosfiltfilt(x, sos, K=None, lengths=None):
    """Zero-phase forward-backward filtering, written out as its definition:
    the cascade from zero state over each channel, the result reversed in
    time, the cascade again, reversed back (y = R H R H x).  FP64."""
    x = np.asarray(x, dtype=np.float64)
    sos = np.asarray(sos, dtype=np.float64)
    if sos.ndim == 2:
        sos = sos[None]
    C = sos.shape[0]
    lengths = np.array([x.size]) if lengths is None else np.asarray(lengths, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lengths)])

    def rev(v):
        out = np.empty_like(v)
        for c in range(C):
            out[off[c]:off[c + 1]] = v[off[c]:off[c + 1]][::-1]
        return out
    y1, _ = sosfilt(x, sos, K=K, lengths=lengths)
    y2, _ = sosfilt(rev(y1), sos, K=K, lengths=lengths)
    return rev(y2)


def sosfilt_adjoint(x, sos, g_y, K=None, lengths=None, zi=None, g_zf=None):
    """See :meth:`Oracle.sosfilt_adjoint`."""
    return default().sosfilt_adjoint(x, sos, g_y, K, lengths, zi, g_zf)


def rel_l2_per_channel(y_test, y_ref, lengths):
    """Relative L2 error per channel, FP64: ||y_test - y_ref|| / ||y_ref||.
    (A channel whose reference is all zero reports the absolute norm.)"""
    y_test = np.asarray(y_test, dtype=np.float64).reshape(-1)
    y_ref = np.asarray(y_ref, dtype=np.float64).reshape(-1)
    out = []
    o = 0
    for n in np.asarray(lengths, dtype=np.int64).reshape(-1):
        n = int(n)
        d = np.linalg.norm(y_test[o:o + n] - y_ref[o:o + n])
        r = np.linalg.norm(y_ref[o:o + n])
        out.append(d / r if r > 0 else d)
        o += n
    return np.array(out)
