"""Per-shape choice of the kernel tuning (N, W, solver, kernel) by measurement.

The sequential depth of a section grows with N (PH: N, cyclic reduction:
log2 N) while the lane scan's cost per sample shrinks with it, and which one
wins depends on the shape of the call (the paper's depth-versus-N trade-off,
Sec. VIII).  ``autotune`` times every supported candidate on the caller's own
shapes and coefficients with CUDA events and returns the fastest; results are
cached in memory, keyed by (max K, length bucket, channel-count bucket,
precision class), and optionally in a JSON file (``SOSFILT_TUNE_CACHE``).

The precision class is whether the plan carries any channel's state by the
look-back (poles near the unit circle): only then does W, the look-back
kernel's tile width, matter, so only then are several W tried.  And whether
some section is ill-conditioned for FP32 (``SosFilter.plan_extended``): only
the PH warp-segment kernel gives those sections extended precision, so then
neither the section pipeline nor cyclic reduction is a candidate, nor N = 64.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import torch

# (N, W) pairs compiled into the library
SUPPORTED_NW = [(16, 8), (16, 16), (32, 4), (32, 7), (32, 8), (32, 16), (64, 3), (64, 4), (64, 7),
                (64, 8)]
ALGOS = (1, 2)  # PH, cyclic reduction
DEFAULT = (32, 8, 1, 0)

_cache: Dict[Tuple, Tuple[int, int, int, int]] = {}
_lock = threading.Lock()


def shape_key(lengths: Sequence[int], kmax: int, carried: bool, extended: bool = False) -> Tuple:
    """(max K, length bucket, channel-count bucket, precision class)."""
    n = len(lengths)
    total = sum(int(v) for v in lengths)
    mean = total / max(n, 1)
    lb = int(round(math.log2(mean))) if mean >= 1 else 0
    cb = int(round(math.log2(n))) if n >= 1 else 0
    cls = "carried" if carried else "horizon"
    return (int(kmax), lb, cb, cls + "+ext" if extended else cls)


SECTION_PIPELINE = 4  # SOS_FLAG_SECTION_PIPELINE


def ws_ctas(n: int) -> int:
    """SOS_FLAG_WS_CTAS(n): CTAs per SM of the warp-segment launch."""
    return (n & 15) << 8


# flags for the channels within their memory horizon: the warp-segment kernel
# at the most CTAs per SM that fit and at fewer (longer-running warps, for
# calls whose segments fill the GPU about once), and the section pipeline
KERNELS = {16: (0, ws_ctas(2), SECTION_PIPELINE),
           32: (0, ws_ctas(2), SECTION_PIPELINE),
           64: (0, ws_ctas(2), SECTION_PIPELINE)}


def candidates(carried: bool, extended: bool = False) -> List[Tuple[int, int, int, int]]:
    """Tunings to try: every N with both solvers and each kernel choice for
    the channels within their memory horizon; several W only when some
    channel is carried by the look-back (W sizes the look-back tiles); PH on
    the warp-segment kernel with N <= 32 only when some section is
    ill-conditioned."""
    out = []
    # ill-conditioned sections: N <= 32 (the in-lane FP32 runs are N samples
    # long; at N = 64 some precision-stress channels exceed the FP32 bound)
    for n in ((16, 32) if extended else (16, 32, 64)):
        ws = sorted({w for (nn, w) in SUPPORTED_NW if nn == n}) if carried else \
            [8 if (n, 8) in SUPPORTED_NW else min(w for (nn, w) in SUPPORTED_NW if nn == n)]
        for w in ws:
            for a in ((1,) if extended else ALGOS):
                for f in KERNELS[n]:
                    if extended and f & SECTION_PIPELINE:
                        continue
                    out.append((n, w, a, f))
    return out


def _cache_file() -> Optional[str]:
    return os.environ.get("SOSFILT_TUNE_CACHE") or None


def _load_file(path: str) -> None:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return
    for k, v in data.items():
        _cache[tuple(json.loads(k))] = tuple(v)


def _save_file(path: str) -> None:
    data = {json.dumps(list(k)): list(v) for k, v in _cache.items()}
    tmp = path + ".tmp"
    try:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(data, f)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_apply(plan, x, y, zi, zf, sos, K, reps: int) -> float:
    """Best of `reps` timed calls as a caller makes them: prepare (its plan
    cache holding the tables after the first) and apply."""
    plan.prepare(sos, K)
    plan.apply(x, y, zi, zf)  # warm-up (also first-launch attribute setup)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.prepare(sos, K)
        plan.apply(x, y, zi, zf)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune(x: torch.Tensor, sos: torch.Tensor, K: Optional[torch.Tensor] = None,
             lengths=None, zi: Optional[torch.Tensor] = None, reps: int = 5,
             use_cache: bool = True, report: Optional[list] = None) -> Tuple[int, int, int, int]:
    """Fastest (N, W, algo, flags) for this call's shapes, by measurement."""
    from . import SosFilter
    sos = sos if sos.dim() == 3 else sos.unsqueeze(0)
    C, kmax = int(sos.shape[0]), int(sos.shape[1])
    if lengths is None:
        lengths = [x.numel()]
    lh = [int(v) for v in torch.as_tensor(lengths).reshape(-1).tolist()]
    if K is None:
        K = torch.full((C,), kmax, dtype=torch.int32, device=x.device)
    # precision class from the default plan
    probe = SosFilter(lh, kmax, tuning=DEFAULT, device=x.device)
    probe.prepare(sos.contiguous(), K)
    hz, _ = probe.plan_info()
    carried = bool((hz < 0).any())
    extended = bool(probe.plan_extended().any())
    key = shape_key(lh, kmax, carried, extended)
    path = _cache_file()
    with _lock:
        if use_cache and path and not _cache:
            _load_file(path)
        if use_cache and key in _cache:
            return _cache[key]
    y = torch.empty_like(x)
    zf = torch.empty((C, kmax, 2), dtype=torch.float32, device=x.device)
    best, best_t = DEFAULT, float("inf")
    for cand in candidates(carried, extended):
        plan = SosFilter(lh, kmax, tuning=cand, device=x.device)
        t = _time_apply(plan, x, y, zi, zf, sos.contiguous(), K, reps)
        if report is not None:
            report.append((cand, t))
        if t < best_t:
            best, best_t = cand, t
    with _lock:
        _cache[key] = best
        if path:
            _save_file(path)
    return best


def clear_cache() -> None:
    with _lock:
        _cache.clear()


def cached(key: Tuple) -> Optional[Tuple[int, int, int, int]]:
    return _cache.get(key)


def seed_cache(entries: Iterable[Tuple[Tuple, Tuple[int, int, int, int]]]) -> None:
    with _lock:
        for k, v in entries:
            _cache[tuple(k)] = tuple(v)
