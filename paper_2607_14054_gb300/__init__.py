"""Cascaded biquad (second-order-section) filtering on GB300 (sm_103a).

The compute runs in the hand-written CUDA kernels of ``libsosfilt.so`` behind
the C ABI of ``include/sosfilt.h``; this package only marshals PyTorch
tensors (device memory and the current stream) into those calls.  There is
no CPU fallback: without the compiled library and a CUDA device every entry
point raises.

    y, zf = sosfilt(x, sos)                        # one channel
    y, zf = sosfilt(x, sos, K=K, lengths=lengths, zi=zi)   # packed batch

``SosFilter`` keeps the workspace and the device copy of the lengths for
repeated calls with the same shapes (and is what CUDA-graph capture uses).
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import _abi
from ._abi import SosError, sos_tuning  # noqa: F401

__all__ = ["SosFilter", "SosHostFilter", "SosStream", "sosfilt", "sosfilt_host", "sosfiltfilt", "sosfilt_diff", "SosFilterFunction", "SosError",
           "sos_tuning", "build"]


def build(force: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force)


def _check_device(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (this library has no CPU path)")


class SosFilter:
    """A reusable plan: channel lengths, section count and tuning fixed;
    signals, coefficients and states passed per call."""

    def __init__(self, lengths: Sequence[int] | torch.Tensor, kmax: int,
                 tuning: Optional[Sequence[int]] = None, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("sosfilt needs a CUDA device")
        _abi.load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        lh = torch.as_tensor(lengths, dtype=torch.int64).reshape(-1).cpu().contiguous()
        if lh.numel() < 1:
            raise ValueError("at least one channel")
        if int(lh.min()) < 0:
            raise ValueError("negative length")
        self.lengths_host = lh
        self.lengths = lh.to(self.device)
        self.n_channels = int(lh.numel())
        self.kmax = int(kmax)
        self.total = int(lh.sum())
        self.tuning = tuple(tuning) if tuning is not None else (0, 0, 0, 0)
        nbytes = _abi.sos_workspace_size(self.n_channels, self.kmax, lh.data_ptr(), self.tuning)
        if nbytes == 0:
            raise ValueError("unsupported sizes or tuning %r" % (self.tuning,))
        self.ws_bytes = nbytes
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = _abi.sos_workspace_init(self.workspace.data_ptr(), nbytes, stream)
        if st != 0:
            raise SosError(st, "sos_workspace_init")

    def __call__(self, x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                 zi: Optional[torch.Tensor] = None, y: Optional[torch.Tensor] = None,
                 zf: Optional[torch.Tensor] = None, want_zf: bool = True):
        C, kmax = self.n_channels, self.kmax
        _check_device(x, "x")
        if x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != self.total:
            raise ValueError("x must be contiguous float32 with sum(lengths) elements")
        sos = sos.reshape(C, kmax, 6)
        if sos.dtype != torch.float64 or not sos.is_contiguous() or sos.device != x.device:
            raise ValueError("sos must be contiguous float64 [C, kmax, 6] on x's device")
        if K is None:
            K = torch.full((C,), kmax, dtype=torch.int32, device=x.device)
        if K.dtype != torch.int32 or not K.is_contiguous() or K.numel() != C:
            raise ValueError("K must be contiguous int32 [C]")
        if zi is not None:
            zi = zi.reshape(C, kmax, 2)
            if zi.dtype != torch.float32 or not zi.is_contiguous():
                raise ValueError("zi must be contiguous float32 [C, kmax, 2]")
        if y is None:
            y = torch.empty_like(x)
        if zf is None and want_zf:
            zf = torch.empty((C, kmax, 2), dtype=torch.float32, device=x.device)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_filter(x.data_ptr(), sos.data_ptr(), K.data_ptr(), C, kmax,
                             self.lengths.data_ptr(), self.lengths_host.data_ptr(),
                             zi.data_ptr() if zi is not None else 0, y.data_ptr(),
                             zf.data_ptr() if zf is not None else 0, self.workspace.data_ptr(),
                             self.ws_bytes, self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_filter")
        return y, zf

    def prepare(self, sos: torch.Tensor, K: Optional[torch.Tensor] = None):
        """Enqueue only the plan kernel (coefficient tables) for these sos/K."""
        C, kmax = self.n_channels, self.kmax
        sos = sos.reshape(C, kmax, 6)
        if K is None:
            K = torch.full((C,), kmax, dtype=torch.int32, device=sos.device)
        self._keep = (sos, K)
        stream = torch.cuda.current_stream(sos.device).cuda_stream
        st = _abi.sos_prepare(sos.data_ptr(), K.data_ptr(), C, kmax, self.lengths.data_ptr(),
                              self.lengths_host.data_ptr(), self.workspace.data_ptr(),
                              self.ws_bytes, self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_prepare")

    def apply(self, x: torch.Tensor, y: torch.Tensor, zi: Optional[torch.Tensor] = None,
              zf: Optional[torch.Tensor] = None):
        """Enqueue only the filtering kernel, using the tables of the last
        prepare() on this plan."""
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_apply(x.data_ptr(), self.n_channels, self.kmax, self.lengths_host.data_ptr(),
                            zi.data_ptr() if zi is not None else 0, y.data_ptr(),
                            zf.data_ptr() if zf is not None else 0, self.workspace.data_ptr(),
                            self.ws_bytes, self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_apply")
        return y, zf

    def backward(self, x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor],
                 zi: Optional[torch.Tensor], grad_y: torch.Tensor,
                 grad_zf: Optional[torch.Tensor] = None, want_zi: bool = True):
        """dL/dx, dL/dsos (float64, w.r.t. the rows as given) and dL/dzi from
        dL/dy and dL/dzf, by the library's adjoint kernels."""
        C, kmax = self.n_channels, self.kmax
        sos = sos.reshape(C, kmax, 6).contiguous()
        if K is None:
            K = torch.full((C,), kmax, dtype=torch.int32, device=x.device)
        if not hasattr(self, "_bws"):
            nb = _abi.sos_backward_workspace_size(C, kmax, self.lengths_host.data_ptr(),
                                                  self.tuning)
            if nb == 0:
                raise ValueError("unsupported sizes for the backward pass")
            self._bws_bytes = nb
            self._bws = torch.zeros(nb, dtype=torch.uint8, device=self.device)
        grad_y = grad_y.contiguous()
        if grad_y.dtype != torch.float32 or grad_y.numel() != self.total:
            raise ValueError("grad_y must be float32 with sum(lengths) elements")
        gx = torch.empty_like(grad_y)
        gsos = torch.empty((C, kmax, 6), dtype=torch.float64, device=x.device)
        gzi = torch.empty((C, kmax, 2), dtype=torch.float32, device=x.device) if want_zi else None
        gzf = grad_zf.reshape(C, kmax, 2).contiguous() if grad_zf is not None else None
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_filter_backward(x.data_ptr(), sos.data_ptr(), K.data_ptr(), C, kmax,
                                      self.lengths.data_ptr(), self.lengths_host.data_ptr(),
                                      zi.data_ptr() if zi is not None else 0, grad_y.data_ptr(),
                                      gzf.data_ptr() if gzf is not None else 0, gx.data_ptr(),
                                      gsos.data_ptr(), gzi.data_ptr() if gzi is not None else 0,
                                      self._bws.data_ptr(), self._bws_bytes, self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_filter_backward")
        return gx, gsos, gzi

    def backward_status(self) -> int:
        """Device-side status of the latest backward call (synchronises)."""
        stream = torch.cuda.current_stream(self.device).cuda_stream
        return _abi.sos_device_status(self._bws.data_ptr(), stream)

    def plan_info(self):
        """(horizon, tiles) per channel from the latest prepare: int32 host
        tensors; horizon -1 marks channels whose state is carried by the
        look-back."""
        h = torch.empty(self.n_channels, dtype=torch.int32)
        t = torch.empty(self.n_channels, dtype=torch.int32)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = _abi.sos_plan_query(self.workspace.data_ptr(), 0, self.n_channels, h.data_ptr(),
                                 t.data_ptr(), stream)
        if st != 0:
            raise SosError(st, "sos_plan_query")
        return h, t

    def plan_extended(self):
        """Per channel, 1 where some section is ill-conditioned for FP32 and
        the default kernel runs its lane scan in extended precision (int32
        host tensor, from the latest prepare)."""
        e = torch.empty(self.n_channels, dtype=torch.int32)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = _abi.sos_plan_extended(self.workspace.data_ptr(), 0, self.n_channels, e.data_ptr(),
                                    stream)
        if st != 0:
            raise SosError(st, "sos_plan_extended")
        return e

    def filtfilt(self, x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                 y: Optional[torch.Tensor] = None, tmp: Optional[torch.Tensor] = None):
        """Zero-phase filtering, y = R H R H x (sos_filtfilt)."""
        C, kmax = self.n_channels, self.kmax
        _check_device(x, "x")
        if x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != self.total:
            raise ValueError("x must be contiguous float32 with sum(lengths) elements")
        sos = sos.reshape(C, kmax, 6).contiguous()
        if K is None:
            K = torch.full((C,), kmax, dtype=torch.int32, device=x.device)
        y = torch.empty_like(x) if y is None else y
        tmp = torch.empty_like(x) if tmp is None else tmp
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_filtfilt(x.data_ptr(), sos.data_ptr(), K.data_ptr(), C, kmax,
                               self.lengths.data_ptr(), self.lengths_host.data_ptr(), y.data_ptr(),
                               tmp.data_ptr(), self.workspace.data_ptr(), self.ws_bytes, self.tuning,
                               stream)
        if st != 0:
            raise SosError(st, "sos_filtfilt")
        return y

    def apply_baseline(self, algorithm: str, x: torch.Tensor, y: torch.Tensor, seg_len: int,
                       zi: Optional[torch.Tensor] = None, zf: Optional[torch.Tensor] = None):
        """The comparison algorithms on this plan's tables: "scalar" or
        "block" filtering (sos_apply_baseline), segments of seg_len."""
        algo = {"scalar": 0, "block": 1}[algorithm]
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_apply_baseline(algo, x.data_ptr(), self.n_channels, self.kmax,
                                     self.lengths_host.data_ptr(),
                                     zi.data_ptr() if zi is not None else 0, y.data_ptr(),
                                     zf.data_ptr() if zf is not None else 0,
                                     seg_len, self.workspace.data_ptr(), self.ws_bytes,
                                     self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_apply_baseline")
        return y, zf

    def plan_recomputed(self) -> int:
        """Channels whose tables the latest prepare() recomputed (0: all came
        from the plan cache); synchronises the current stream."""
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st, n = _abi.sos_plan_recomputed(self.workspace.data_ptr(), stream)
        if st != 0:
            raise SosError(st, "sos_plan_recomputed")
        return n

    def apply_part(self, part: str, x: torch.Tensor, y: torch.Tensor,
                   zi: Optional[torch.Tensor] = None, zf: Optional[torch.Tensor] = None):
        """One of the two launches of apply(): "pipeline" or "carried"."""
        stream = torch.cuda.current_stream(x.device).cuda_stream
        st = _abi.sos_apply_part(part, x.data_ptr(), self.n_channels, self.kmax,
                                 self.lengths_host.data_ptr(),
                                 zi.data_ptr() if zi is not None else 0, y.data_ptr(),
                                 zf.data_ptr() if zf is not None else 0, self.workspace.data_ptr(),
                                 self.ws_bytes, self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_apply_" + part)
        return y, zf

    def device_status(self) -> int:
        """Synchronises the current stream and returns the device-side status
        of the latest call (0 = OK)."""
        stream = torch.cuda.current_stream(self.device).cuda_stream
        return _abi.sos_device_status(self.workspace.data_ptr(), stream)


class SosStream:
    """Block-by-block filtering of C channels (the low-latency streaming
    mode): each call filters the next ``chunk`` samples of every channel in
    one kernel launch, carrying the state on the device from call to call.

        st = SosStream(sos, chunk)                 # sos [C, K, 6] float64, CUDA
        for block in blocks:                       # block: [C, chunk] float32
            y = st(block)
    """

    def __init__(self, sos: torch.Tensor, chunk: int, K: Optional[torch.Tensor] = None,
                 zi: Optional[torch.Tensor] = None, tuning: Optional[Sequence[int]] = None):
        _check_device(sos, "sos")
        sos = sos if sos.dim() == 3 else sos.unsqueeze(0)
        self.n_channels, self.kmax = int(sos.shape[0]), int(sos.shape[1])
        self.chunk = int(chunk)
        if self.chunk < 1:
            raise ValueError("chunk must be positive")
        if tuning is None:
            # latency: short groups (N = 16) unless the blocks are long
            n = 16 if self.chunk <= (1 << 14) else 32
            tuning = (n, 8, 1, 0)
        self.plan = SosFilter([self.chunk] * self.n_channels, self.kmax, tuning=tuning,
                              device=sos.device)
        self.sos = sos.contiguous()
        self.K = (K if K is not None else
                  torch.full((self.n_channels,), self.kmax, dtype=torch.int32, device=sos.device))
        self.plan.prepare(self.sos, self.K)
        # the state alternates between two buffers: each block reads one and
        # writes the other (different warps of a channel read and write it)
        self._bufs = [torch.zeros((self.n_channels, self.kmax, 2), dtype=torch.float32,
                                  device=sos.device) for _ in range(2)]
        self._cur = 0
        # a caller's initial state (not one this filter left): the next block
        # waits for its response to die out before cutting segments
        self._foreign = zi is not None
        if zi is not None:
            self.state.copy_(zi.reshape(self.n_channels, self.kmax, 2))

    @property
    def state(self) -> torch.Tensor:
        """The state after the latest block (before the next one)."""
        return self._bufs[self._cur]

    def __call__(self, x: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        _check_device(x, "x")
        if x.dtype != torch.float32 or not x.is_contiguous() or \
                x.numel() != self.n_channels * self.chunk:
            raise ValueError("x must be contiguous float32 [C, chunk]")
        if y is None:
            y = torch.empty_like(x)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        zi, zf = self._bufs[self._cur], self._bufs[1 - self._cur]
        flags = _abi.SOS_STREAM_FOREIGN_STATE if self._foreign else 0
        st = _abi.sos_stream(x.data_ptr(), y.data_ptr(), zi.data_ptr(), zf.data_ptr(),
                             self.n_channels, self.kmax, self.chunk, flags,
                             self.plan.workspace.data_ptr(), self.plan.ws_bytes, self.plan.tuning,
                             stream)
        if st != 0:
            raise SosError(st, "sos_stream")
        self._foreign = False
        self._cur = 1 - self._cur
        return y

    def reset(self, zi: Optional[torch.Tensor] = None) -> None:
        self._foreign = zi is not None
        if zi is None:
            self.state.zero_()
        else:
            self.state.copy_(zi.reshape(self.n_channels, self.kmax, 2))


_plans = {}


def sosfilt(x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
            lengths=None, zi: Optional[torch.Tensor] = None, tuning=None, check: bool = False):
    """Filter x (float32, CUDA, packed channels) through the cascade ``sos``
    (float64 [C, kmax, 6] or [kmax, 6]).  Returns (y, zf).  ``tuning="auto"``
    picks (N, W, solver) for these shapes by measurement (``autotune``)."""
    _check_device(x, "x")
    if sos.dim() == 2:
        sos = sos.unsqueeze(0)
    C, kmax = int(sos.shape[0]), int(sos.shape[1])
    if lengths is None:
        if C != 1:
            raise ValueError("lengths are required for more than one channel")
        lengths = [x.numel()]
    if isinstance(tuning, str):
        if tuning != "auto":
            raise ValueError("tuning must be a 4-tuple, None or 'auto'")
        from .autotune import autotune
        tuning = autotune(x, sos, K, lengths, zi)
    lh = tuple(int(v) for v in torch.as_tensor(lengths).reshape(-1).tolist())
    key = (x.device, lh, kmax, tuple(tuning) if tuning is not None else None)
    plan = _plans.get(key)
    if plan is None:
        plan = SosFilter(lh, kmax, tuning=tuning, device=x.device)
        if len(_plans) > 16:
            _plans.clear()
        _plans[key] = plan
    y, zf = plan(x.contiguous(), sos.contiguous(), K, zi)
    if check:
        st = plan.device_status()
        if st != 0:
            raise SosError(st, "sos_filter (device)")
    return y, zf


class SosHostFilter:
    """sos_filter from host memory to host memory (``sos_filter_host``): the
    signal is cut into blocks whose copy in, filtering and copy out overlap.
    Keeps the device workspace and staging buffers for repeated calls with
    the same channel lengths."""

    def __init__(self, lengths: Sequence[int] | torch.Tensor, kmax: int,
                 tuning: Optional[Sequence[int]] = None, block: int = 0, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("sosfilt needs a CUDA device")
        _abi.load()
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        lh = torch.as_tensor(lengths, dtype=torch.int64).reshape(-1).cpu().contiguous()
        if lh.numel() < 1 or int(lh.min()) < 0:
            raise ValueError("lengths must be one or more non-negative counts")
        self.lengths_host = lh
        self.lengths = lh.to(self.device)
        self.n_channels = int(lh.numel())
        self.kmax = int(kmax)
        self.total = int(lh.sum())
        self.tuning = tuple(tuning) if tuning is not None else (0, 0, 0, 0)
        st, ws, stg, blk = _abi.sos_filter_host_sizes(self.n_channels, self.kmax, lh.data_ptr(),
                                                      block, self.tuning)
        if st != 0:
            raise SosError(st, "sos_filter_host_sizes")
        self.block = blk
        self.ws_bytes, self.staging_bytes = ws, stg
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.staging = torch.empty(stg, dtype=torch.uint8, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = _abi.sos_workspace_init(self.workspace.data_ptr(), ws, stream)
        if st != 0:
            raise SosError(st, "sos_workspace_init")

    def __call__(self, x_host: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                 zi: Optional[torch.Tensor] = None, y_host: Optional[torch.Tensor] = None,
                 zf: Optional[torch.Tensor] = None, want_zf: bool = True):
        """x_host: float32 host tensor (pinned for the copies to overlap);
        sos, K, zi on the device.  Returns (y_host, zf); y_host is complete
        once the current stream has finished the call."""
        C, kmax = self.n_channels, self.kmax
        if x_host.is_cuda or x_host.dtype != torch.float32 or not x_host.is_contiguous() or \
                x_host.numel() != self.total:
            raise ValueError("x_host must be a contiguous float32 host tensor of sum(lengths)")
        sos = sos.reshape(C, kmax, 6)
        if sos.dtype != torch.float64 or not sos.is_contiguous() or sos.device != self.device:
            raise ValueError("sos must be contiguous float64 [C, kmax, 6] on the plan's device")
        if K is None:
            K = torch.full((C,), kmax, dtype=torch.int32, device=self.device)
        if zi is not None:
            zi = zi.reshape(C, kmax, 2)
            if zi.dtype != torch.float32 or not zi.is_contiguous() or zi.device != self.device:
                raise ValueError("zi must be contiguous float32 [C, kmax, 2] on the device")
        if y_host is None:
            y_host = torch.empty(self.total, dtype=torch.float32, pin_memory=True)
        if y_host.is_cuda or y_host.numel() != self.total or not y_host.is_contiguous():
            raise ValueError("y_host must be a contiguous float32 host tensor of sum(lengths)")
        if zf is None and want_zf:
            zf = torch.empty((C, kmax, 2), dtype=torch.float32, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        st = _abi.sos_filter_host(x_host.data_ptr(), sos.data_ptr(), K.data_ptr(), C, kmax,
                                  self.lengths.data_ptr(), self.lengths_host.data_ptr(),
                                  zi.data_ptr() if zi is not None else 0, y_host.data_ptr(),
                                  zf.data_ptr() if zf is not None else 0,
                                  self.workspace.data_ptr(), self.ws_bytes,
                                  self.staging.data_ptr(), self.staging_bytes, self.block,
                                  self.tuning, stream)
        if st != 0:
            raise SosError(st, "sos_filter_host")
        return y_host, zf


_host_plans = {}


def sosfilt_host(x_host: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                 lengths=None, zi: Optional[torch.Tensor] = None,
                 y_host: Optional[torch.Tensor] = None, tuning=None, block: int = 0):
    """``sosfilt`` for a signal in host memory (``sos_filter_host``): x_host
    float32 on the host (pinned), sos/K/zi on the CUDA device.  Returns
    (y_host, zf) after synchronising the current stream, so y_host is ready."""
    if sos.dim() == 2:
        sos = sos.unsqueeze(0)
    _check_device(sos, "sos")
    C, kmax = int(sos.shape[0]), int(sos.shape[1])
    if lengths is None:
        if C != 1:
            raise ValueError("lengths are required for more than one channel")
        lengths = [x_host.numel()]
    lh = tuple(int(v) for v in torch.as_tensor(lengths).reshape(-1).tolist())
    key = (sos.device, lh, kmax, tuple(tuning) if tuning is not None else None, int(block))
    plan = _host_plans.get(key)
    if plan is None:
        plan = SosHostFilter(lh, kmax, tuning=tuning, block=block, device=sos.device)
        if len(_host_plans) > 8:
            _host_plans.clear()
        _host_plans[key] = plan
    y_host, zf = plan(x_host.contiguous(), sos.contiguous(), K, zi, y_host=y_host)
    torch.cuda.current_stream(sos.device).synchronize()
    return y_host, zf


class SosFilterFunction(torch.autograd.Function):
    """y, zf = sosfilt(x, sos, zi) with gradients for x, sos and zi from the
    library's adjoint kernels (``SosFilter.backward``)."""

    @staticmethod
    def forward(ctx, x, sos, zi, plan, K):
        y, zf = plan(x.contiguous(), sos.contiguous(), K,
                     zi.contiguous() if zi is not None else None)
        ctx.plan = plan
        ctx.K = K
        ctx.save_for_backward(x, sos, zi if zi is not None else torch.empty(0))
        ctx.has_zi = zi is not None
        return y, zf

    @staticmethod
    def backward(ctx, grad_y, grad_zf):
        x, sos, zi = ctx.saved_tensors
        zi = zi if ctx.has_zi else None
        if grad_y is None:
            grad_y = torch.zeros_like(x)
        gx, gsos, gzi = ctx.plan.backward(x, sos, ctx.K, zi, grad_y, grad_zf,
                                          want_zi=ctx.has_zi)
        return gx, gsos.reshape(sos.shape), (gzi.reshape(zi.shape) if ctx.has_zi else None), \
            None, None


def sosfiltfilt(x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                lengths=None, tuning=None) -> torch.Tensor:
    """Zero-phase forward-backward filtering of x (float32, CUDA, packed
    channels): the cascade applied forward, then to the time-reversed result,
    reversed back (no edge padding)."""
    _check_device(x, "x")
    sos3 = sos if sos.dim() == 3 else sos.unsqueeze(0)
    C, kmax = int(sos3.shape[0]), int(sos3.shape[1])
    if lengths is None:
        if C != 1:
            raise ValueError("lengths are required for more than one channel")
        lengths = [x.numel()]
    lh = tuple(int(v) for v in torch.as_tensor(lengths).reshape(-1).tolist())
    key = (x.device, lh, kmax, tuple(tuning) if tuning is not None else None)
    plan = _plans.get(key)
    if plan is None:
        plan = SosFilter(lh, kmax, tuning=tuning, device=x.device)
        if len(_plans) > 16:
            _plans.clear()
        _plans[key] = plan
    return plan.filtfilt(x.contiguous(), sos3.contiguous(), K)


def sosfilt_diff(x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
                 lengths=None, zi: Optional[torch.Tensor] = None, tuning=None):
    """Differentiable ``sosfilt``: (y, zf) with autograd through x, sos and zi."""
    _check_device(x, "x")
    sos3 = sos if sos.dim() == 3 else sos.unsqueeze(0)
    C, kmax = int(sos3.shape[0]), int(sos3.shape[1])
    if lengths is None:
        if C != 1:
            raise ValueError("lengths are required for more than one channel")
        lengths = [x.numel()]
    lh = tuple(int(v) for v in torch.as_tensor(lengths).reshape(-1).tolist())
    key = (x.device, lh, kmax, tuple(tuning) if tuning is not None else None)
    plan = _plans.get(key)
    if plan is None:
        plan = SosFilter(lh, kmax, tuning=tuning, device=x.device)
        if len(_plans) > 16:
            _plans.clear()
        _plans[key] = plan
    if K is None:
        K = torch.full((C,), kmax, dtype=torch.int32, device=x.device)
    if zi is not None:
        zi = zi.reshape(C, kmax, 2)
    return SosFilterFunction.apply(x, sos3, zi, plan, K)
