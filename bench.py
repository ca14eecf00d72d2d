#!/usr/bin/env python3
"""Benchmark of the cascaded-biquad hot path on GB300.

One step = one full call of the C ABI's sos_filter on the 16th-order (K = 8)
Butterworth band-pass workload, 2^24 FP32 samples i.i.d. N(0, 1), one
channel, zero initial state, inputs resident in HBM: sos_prepare (the plan
kernel; the coefficients are unchanged from the previous step, so its plan
cache keeps the tables after comparing them on the device) then sos_apply
(the kernel for channels within their memory horizon -- warp segments or the
section pipeline -- launched early behind the plan, then the look-back
kernel, which finds no carried channel here, launched early behind that),
replayed as one CUDA graph.  The same step with the plan recomputed every
time is reported beside it.  The tuning (N, W, solver, kernel) is chosen by
the library's autotuner before the timed region.
Prints one JSON line (rank 0), with the low-pass (K = 1, 8192 samples:
latency), batched (4096 channels), differentiation (forward + backward,
256 x 2^16) and precision-stress (64 x 2^26, poles at radius 0.999..0.9999)
workloads as extra fields, and the oracle parity of every one of them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun, one process per GPU): the single long signal does not
shard without a state exchange, so each rank filters its own replica of the
workload (weak scaling, no data-path collective); a barrier and a max over
ranks bracket the timing.

The L2 cache (126.5 MiB on GB300) is flushed between timed steps by writing a
256 MiB buffer, outside the timed events.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def fma_per_sample(K: int) -> int:
    # the method's own count: 6 block FMAs per sample per section
    # (paper Table overall_complexity, dominant term 6/L per lane-sample) plus
    # one multiply for the split-off gain (Sec. II, Eq. simple_second_order)
    return 6 * K + 1


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is under load."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "utilization.gpu")

    def __init__(self, gpu_index: int, out_path: str | None):
        self.gpu = gpu_index
        self.out_path = out_path
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.out_path:
            with open(self.out_path, "w") as f:
                f.write(self.FIELDS + "\n")
                for _, l in self.lines:
                    f.write(l + "\n")
        rows = []
        for _, l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]),
                             "hw": parts[5], "hwt": parts[6], "swt": parts[7], "pcap": parts[8],
                             "util": float(parts[9])})
            except ValueError:
                continue
        load = [r for r in rows if r["util"] > 0] or rows
        if not load:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["max"] for r in load), "reasons": sorted(reasons),
                "samples": len(load)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        # one process per GPU over NCCL; gloo where there is no GPU (the
        # host-side logic of the multi-rank path)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def reduce_max(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ParityJob:
    """One workload's outputs to check against the oracle in the cpu_baseline
    leg: every channel in full (relative L2 per channel, run in chunks of
    channels so that host memory stays bounded) and, with `windows`, also
    that many equal windows of each channel, each against the oracle's output
    over the same span (computed from the channel's start)."""

    def __init__(self, name, x, sos, K, lengths, zi, y, tol, windows=0, chunk=256,
                 channels=None):
        self.name, self.x, self.sos, self.K = name, x, sos, K
        self.lengths, self.zi, self.y, self.tol = lengths, zi, y, tol
        self.windows, self.chunk = windows, chunk
        self.channels = channels  # None: all; else the channel indices checked

    def run(self):
        import numpy as np
        import oracle
        L = np.asarray(self.lengths, dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(L)])
        sos = self.sos.cpu().numpy()
        K = np.asarray(self.K.cpu() if hasattr(self.K, "cpu") else self.K)
        zi = self.zi.cpu().double().numpy() if self.zi is not None else None
        chans = np.arange(len(L)) if self.channels is None else np.asarray(self.channels)
        errs, wins = [], []
        for i0 in range(0, len(chans), self.chunk):
            cs = chans[i0:i0 + self.chunk]
            xs = np.concatenate([self.x[int(off[c]):int(off[c + 1])].cpu().double().numpy()
                                 for c in cs])
            ys = np.concatenate([self.y[int(off[c]):int(off[c + 1])].cpu().double().numpy()
                                 for c in cs])
            ref, _ = oracle.sosfilt(xs, sos[cs], K=K[cs], lengths=L[cs],
                                    zi=zi[cs] if zi is not None else None)
            o = np.concatenate([[0], np.cumsum(L[cs])])
            for j in range(len(cs)):
                r, g = ref[o[j]:o[j + 1]], ys[o[j]:o[j + 1]]
                nr = np.linalg.norm(r)
                errs.append(float(np.linalg.norm(g - r) / nr) if nr > 0 else 0.0)
                if self.windows:
                    w = len(r) // self.windows
                    wins.append(max(float(np.linalg.norm(g[k * w:(k + 1) * w] - r[k * w:(k + 1) * w])
                                          / np.linalg.norm(r[k * w:(k + 1) * w]))
                                    for k in range(self.windows)))
        errs = np.array(errs)
        out = {"rel_l2": float(errs.max()), "rel_l2_median": float(np.median(errs)),
               "tolerance": self.tol, "channels": int(len(chans)),
               "samples": int(L[chans].sum()), "within_tolerance": int((errs <= self.tol).sum())}
        if self.windows:
            wins = np.array(wins)
            out.update({"windows_per_channel": self.windows, "worst_window_rel_l2": float(wins.max()),
                        "within_tolerance_every_window": int(((errs <= self.tol) &
                                                              (wins <= self.tol)).sum())})
        return out


def oracle_baseline(wl, target_seconds: float = 10.0, jobs=()):
    """Times the FP64 oracle (as it stands) on the host cores: whole-signal
    passes of the workload, repeated until ~target_seconds of CPU work.  Then
    runs the parity jobs: the GPU path's outputs on the benchmarked workloads
    against the oracle, per channel."""
    import oracle
    x = wl.x.detach().cpu().double().numpy()
    sos = wl.sos.cpu().numpy()
    K = wl.K.cpu().numpy()
    lengths = wl.lengths.numpy()
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.sosfilt(x, sos, K=K, lengths=lengths)
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_seconds or reps >= 50:
            break
    samples = x.size * reps
    threads = min(oracle.num_threads(), wl.n_channels)
    parity = {}
    t1 = time.perf_counter()
    for job in jobs:
        parity[job.name] = job.run()
    return {"value": samples / el / 1e9, "unit": "Gsamples/s", "cores": int(threads),
            "kind": "oracle",
            "sample": f"{reps} full passes of the {x.size}-sample workload ({el:.1f} s); "
                      f"FP64 sample-by-sample cascade, one thread per channel",
            "seconds": el, "parity": parity, "parity_seconds": time.perf_counter() - t1}


def run_reference(args):
    rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return 0
    from synth import workloads
    wl = workloads.plain_bandpass16(n=1 << 24, device="cpu")
    import oracle
    x = wl.x.double().numpy()
    sos = wl.sos.numpy()
    # each step is a bounded sample of the workload: the first 2^21 samples
    # (causal: these outputs equal the full run's first 2^21)
    n = 1 << 21
    xs = x[:n]
    for _ in range(max(args.warmup, 0)):
        oracle.sosfilt(xs, sos)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sosfilt(xs, sos)
    el = time.perf_counter() - t0
    value = n * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": "Gsamples/s K=8 FP32 (batched/plain) and % roofline at "
        "rel-L2<=1e-5 vs FP64", "value": value, "unit": "Gsamples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "samples_per_step": n, "channels": 1, "sections": 8},
        "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} samples of the 2^24-sample signal per step"},
        "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def copy_rates(x, stream, reps: int = 10):
    """The box's own pinned host <-> device copy rates (GB/s) for buffers the
    size of the step's input and output: each direction timed alone, and both
    at once on two streams ("both": bytes of one direction over the time of
    the pair), with CUDA events.  The pair bounds an end-to-end pass that
    moves the input in and the output out once while overlapping them."""
    import torch
    xh = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
    yh = torch.empty(x.numel(), dtype=torch.float32, pin_memory=True)
    xd = torch.empty_like(x)
    yd = torch.empty_like(x)
    nbytes = 4 * x.numel()
    side = torch.cuda.Stream()
    out = {}

    def both():
        side.wait_stream(torch.cuda.current_stream())
        xd.copy_(xh, non_blocking=True)
        with torch.cuda.stream(side):
            yh.copy_(yd, non_blocking=True)
        torch.cuda.current_stream().wait_stream(side)
    for name, fn in (("h2d", lambda: xd.copy_(xh, non_blocking=True)),
                     ("d2h", lambda: yh.copy_(xd, non_blocking=True)), ("both", both)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    return out


def end_to_end(P, x, sos, stream, samples, world, args, tuning):
    """Same metric through the public API with host buffers: pinned host
    input -> sos_filter_host (blocks copied in, filtered and copied out on
    overlapping streams) -> pinned host output, every step; the output
    checked against the device path's once."""
    import torch
    xh = torch.empty(samples, dtype=torch.float32, pin_memory=True)
    xh.copy_(x)
    yh = torch.empty(samples, dtype=torch.float32, pin_memory=True)
    plan = P.SosHostFilter([samples], sos.shape[-2], tuning=tuning, device=x.device)
    e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        plan(xh, sos, y_host=yh)
    torch.cuda.synchronize()
    yd, _ = P.sosfilt(x, sos, tuning=tuning)
    torch.cuda.synchronize()
    ref = yd.cpu()
    agree = float((yh - ref).norm() / ref.norm())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        plan(xh, sos, y_host=yh)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps
    e2e_ms = reduce_max(e2e_ms, world)
    e2e_value = samples * world / (e2e_ms * 1e-3) / 1e9
    return e2e_value, e2e_ms, {"block": plan.block, "blocks": -(-samples // plan.block),
                               "rel_l2_vs_device_path": agree}



# the kernel for channels within their memory horizon: its committed ncu
# summary and the sources it is built from
_COMMON_SOURCES = ["pipe_section.cuh", "sos_pipe.cuh", "sos_async.cuh", "sos_kernels.cuh",
                   "sos_common.cuh"]
KERNEL_PROFILES = {
    "sos_warpseg_kernel": ("sos_warpseg_kernel_bp16_2e24.json", ["warpseg.cu"] + _COMMON_SOURCES),
    "sos_pipe_kernel": ("sos_pipe_kernel_bp16_2e24.json", ["pipe.cu"] + _COMMON_SOURCES),
}


def horizon_kernel(tuning) -> str:
    return "sos_pipe_kernel" if int(tuning[3]) & 4 else "sos_warpseg_kernel"


def source_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_PROFILES[kernel][1]:
        with open(os.path.join(ROOT, "paper_2607_14054_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, samples: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary,
    scaled to this workload's samples; None when the kernel's sources changed
    since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", KERNEL_PROFILES[kernel][0])) as f:
            prof = json.load(f)
    except (OSError, ValueError):
        return None
    if prof.get("source_hash") != source_hash(kernel):
        return None
    return prof["dram_bytes_per_launch"] * samples / prof["samples"]


def graph_of(fn):
    """fn() captured as one CUDA graph (after a warm-up call on the capture
    stream)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def replay_ms(g, steps: int, flush=None):
    """Mean milliseconds per replay of g, CUDA events on the current stream
    around each replay (flush written before each one, outside the events)."""
    import torch
    stream = torch.cuda.current_stream()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        evs[i][0].record(stream)
        g.replay()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(e[0].elapsed_time(e[1]) for e in evs) / steps


def lowpass_leg(P, dev, steps: int = 50):
    """2nd-order Butterworth low-pass on 8,192 samples (K = 1): the latency
    of one whole call (prepare + apply, one graph replay; inputs resident,
    small enough to stay in L2 between calls, as a real-time caller's
    would)."""
    import torch
    from synth import workloads
    wl = workloads.plain_lowpass(device=dev)
    plan = P.SosFilter(wl.lengths, 1, device=dev)
    y = torch.empty_like(wl.x)
    zf = torch.empty(1, 1, 2, device=dev)

    def call():
        plan(wl.x, wl.sos, wl.K, None, y=y, zf=zf)
    g = graph_of(call)
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    ms = replay_ms(g, steps)
    # the streaming mode: the same 8,192 samples as one block of a stream
    # (one launch, tables prepared once), timed per launch
    st = P.SosStream(wl.sos, wl.total)
    ys = torch.empty_like(wl.x)
    x2 = wl.x.view(1, -1)
    gs = graph_of(lambda: st(x2, ys.view(1, -1)))
    ms_s = replay_ms(gs, steps)
    st.reset()
    st(x2, ys.view(1, -1))  # one block from zero state, for the parity check
    # audio-like: 64 channels of the 16th-order band-pass, 256-sample blocks
    bp = workloads.plain_bandpass16(n=16)
    sos64 = bp.sos.to(dev).expand(64, -1, -1).contiguous()
    st64 = P.SosStream(sos64, 256)
    xb = torch.randn(64, 256, device=dev)
    yb = torch.empty_like(xb)
    gb = graph_of(lambda: st64(xb, yb))
    ms_b = replay_ms(gb, steps)
    return {"workload": wl.name, "samples": wl.total, "latency_us": ms_s * 1e3,
            "value": wl.total / (ms_s * 1e-3) / 1e9, "unit": "Gsamples/s",
            "step": "sos_stream: the signal as one block of a stream (one launch, tables "
                    "prepared once, the block cut into warm-up segments within the filter's "
                    "memory horizon, one warp each), one CUDA-graph replay",
            "latency_us_sos_filter": ms * 1e3,
            "sos_filter_step": "sos_filter (prepare + apply), one CUDA-graph replay",
            "stream_64ch_bp16_256": {"latency_us": ms_b * 1e3,
                                     "value": 64 * 256 / (ms_b * 1e-3) / 1e9,
                                     "unit": "Gsamples/s",
                                     "step": "sos_stream, 64 channels x 256-sample blocks of the "
                                             "16th-order band-pass, one launch per block"}}, \
        [ParityJob("lowpass", wl.x, wl.sos.cpu(), wl.K.cpu(), wl.lengths.numpy(), None, y, 1e-5),
         ParityJob("lowpass_stream", wl.x, wl.sos.cpu(), wl.K.cpu(), wl.lengths.numpy(), None,
                   ys, 1e-5)]


def batched_leg(P, dev, world, sms, sm_max, hbm_gbs, steps: int = 5, rank: int = 0):
    """4096 channels, lengths U[2^10, 2^20], K U{1..8}, random sections,
    nonzero zi: one prepare + apply per step, captured as one CUDA graph and
    replayed, inputs resident (8.5 GB, far beyond L2).  With several ranks the
    channels are sharded by cost (contiguous ranges, no collective): each rank
    filters its own range, the time is the slowest rank's, the value the whole
    batch over it (strong scaling)."""
    import torch
    from synth import workloads
    from paper_2607_14054_gb300 import shard
    from paper_2607_14054_gb300.autotune import autotune
    full = workloads.batched(device=dev)
    lh = full.lengths.tolist()
    parts = shard.partition_by_cost(shard.channel_costs(lh, full.K.tolist()), world)
    c0, c1 = parts[rank]
    xs, ss, ks, ls, zs = shard.shard(full.x, full.sos, full.K, lh, full.zi, c0, c1)
    xs, ss, ks, zs = xs.contiguous(), ss.contiguous(), ks.contiguous(), zs.contiguous()
    tuning = autotune(xs, ss, ks, ls, zs)
    plan = P.SosFilter(ls, full.kmax, tuning=tuning, device=dev)
    y = torch.empty_like(xs)
    zf = torch.empty(c1 - c0, full.kmax, 2, device=dev)

    def call():
        plan(xs, ss, ks, zs, y=y, zf=zf)
    call()
    g = graph_of(call)
    g.replay()
    torch.cuda.synchronize()
    ms = reduce_max(replay_ms(g, steps), world)
    if plan.device_status() != 0:
        raise RuntimeError("batched leg: device status")
    ext = plan.plan_extended()
    total = full.total
    lens = full.lengths.double()
    fma = float((lens * (6 * full.K.cpu().double() + 1)).sum())
    t_hbm = 8.0 * total / (hbm_gbs * 1e9)
    t_alu = fma / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    roof = total / max(t_hbm, t_alu) / 1e9  # one GPU
    value = total / (ms * 1e-3) / 1e9       # the whole batch over the slowest rank
    return {"workload": full.name, "channels": full.n_channels, "samples": total,
            "value": value, "unit": "Gsamples/s", "ms_per_step": ms,
            "roofline_gsamples_per_s": roof, "frac_of_roofline": value / world / roof,
            "bound": "hbm" if t_hbm >= t_alu else "alu", "tuning": list(tuning),
            "sharding": {"ranks": world, "scaling": "strong",
                         "channels_per_rank": [b - a for a, b in parts],
                         "how": "contiguous channel ranges balanced by len (6K + 1), "
                                "no collective"},
            "precision_classes": {str(v): int((ext == v).sum()) for v in range(4)},
            "step": "sos_filter (prepare + apply), one CUDA-graph replay"}, \
        ([ParityJob("batched", full.x, full.sos.cpu(), full.K.cpu(), full.lengths.numpy(), full.zi,
                    y, 1e-5)] if world == 1 else [])


def stress_leg(P, dev, world, sms, sm_max, hbm_gbs, steps: int = 3):
    """Precision stress: 64 x 2^26 samples, K = 8, poles at radius
    0.999..0.9999 (long memory horizons, per-channel segments), autotuned
    (untimed), one prepare + apply per step.  Parity: every channel in full
    and in 8 windows, each against the oracle run from the channel's start."""
    import torch
    from synth import workloads
    wl = workloads.precision_stress(device=dev)
    from paper_2607_14054_gb300.autotune import autotune
    tuning = autotune(wl.x, wl.sos, wl.K, wl.lengths, wl.zi)
    plan = P.SosFilter(wl.lengths, wl.kmax, tuning=tuning, device=dev)
    y = torch.empty_like(wl.x)
    zf = torch.empty(wl.n_channels, wl.kmax, 2, device=dev)
    plan(wl.x, wl.sos, wl.K, None, y=y, zf=zf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan(wl.x, wl.sos, wl.K, None, y=y, zf=zf)
    e1.record()
    torch.cuda.synchronize()
    if plan.device_status() != 0:
        raise RuntimeError("stress leg: device status")
    ms = reduce_max(e0.elapsed_time(e1) / steps, world)
    hz, segs = plan.plan_info()
    ext = plan.plan_extended()
    total = wl.total
    fma = 49.0 * total
    t_hbm = 8.0 * total / (hbm_gbs * 1e9)
    t_alu = fma / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    roof = total / max(t_hbm, t_alu) / 1e9
    value = total * world / (ms * 1e-3) / 1e9
    return {"workload": wl.name, "channels": wl.n_channels, "samples": total,
            "value": value, "unit": "Gsamples/s", "ms_per_step": ms,
            "roofline_gsamples_per_s": roof, "frac_of_roofline": value / world / roof,
            "carried_channels": int((hz < 0).sum()), "min_segments_per_channel": int(segs.min()),
            "precision_classes": {str(v): int((ext == v).sum()) for v in range(4)},
            "tuning": list(plan.tuning), "step": "sos_filter (prepare + apply)"}, \
        [ParityJob("stress", wl.x, wl.sos.cpu(), wl.K.cpu(), wl.lengths.numpy(), None, y, 1e-3,
                   windows=8, chunk=8)]


# backward FMAs per sample and section, the count of the method's adjoint:
# 6 to recompute the section's input (forward), 6 for the adjoint run
# (all-pole and FIR parts of the transposed recurrence), 5 for the
# coefficient sums; bytes per sample: x and dL/dy read, dL/dx written
BWD_FMA_PER_SECTION = 17
BWD_BYTES_PER_SAMPLE = 12


def backward_leg(P, dev, world, sms, sm_max, hbm_gbs, steps: int = 5):
    """256 x 2^16, K = 8: forward + backward through the autograd Function;
    the backward launch alone is also timed for its roofline."""
    import torch
    from synth import workloads
    wl = workloads.differentiation(device=dev)
    xg = wl.x.clone().requires_grad_(True)
    sg = wl.sos.clone().requires_grad_(True)
    zg = wl.zi.clone().requires_grad_(True)
    tgt = torch.zeros_like(wl.x)

    def fb():
        y, zf = P.sosfilt_diff(xg, sg, wl.K, lengths=wl.lengths, zi=zg)
        loss = ((y - tgt) ** 2).mean()
        loss.backward()

    for _ in range(2):
        fb()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fb()
    e1.record()
    torch.cuda.synchronize()
    ms = reduce_max(e0.elapsed_time(e1) / steps, world)
    # the library's backward call alone (plan, adjoint kernel, finalize)
    plan = P.SosFilter(wl.lengths, wl.kmax, device=dev)
    gy = torch.randn_like(wl.x)
    plan.backward(wl.x, wl.sos, wl.K, wl.zi, gy)

    def bwd():
        plan.backward(wl.x, wl.sos, wl.K, wl.zi, gy)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    for _ in range(steps):
        bwd()
    b1.record()
    torch.cuda.synchronize()
    ms_b = reduce_max(b0.elapsed_time(b1) / steps, world)
    total = wl.total
    fmas = BWD_FMA_PER_SECTION * float((wl.lengths.double() * wl.K.cpu().double()).sum())
    t_alu = fmas / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    t_hbm = BWD_BYTES_PER_SAMPLE * total / (hbm_gbs * 1e9)
    roof = total / max(t_alu, t_hbm) / 1e9
    vb = total * world / (ms_b * 1e-3) / 1e9
    return {"workload": wl.name, "samples": total,
            "value": total * world / (ms * 1e-3) / 1e9, "unit": "Gsamples/s",
            "ms_per_step": ms, "step": "forward + MSE + backward (dL/dx, dL/dsos, dL/dzi)",
            "backward_call": {"ms": ms_b, "value": vb, "unit": "Gsamples/s",
                              "roofline_gsamples_per_s": roof, "frac_of_roofline": vb / world / roof,
                              "bound": "alu" if t_alu >= t_hbm else "hbm",
                              "fma_per_sample_section": BWD_FMA_PER_SECTION}}


def compare_leg(P, dev, sms, sm_max, hbm_gbs, steps: int = 5):
    """The paper's algorithm comparison (Sec. VIII) on this GPU: the scalar
    recursion, block filtering, PH and cyclic reduction on one 2^24-sample
    channel of Butterworth band-pass cascades of K = 1, 2, 4, 8 sections, all
    on the same segmentation by memory horizon; each algorithm at its best
    segment length / tuning.  Gsamples/s and the fraction of the FP32
    roofline (6K + 1 FMAs per sample against the FMA peak, or 8 bytes per
    sample against HBM)."""
    import torch
    from synth import filters, rng
    n = 1 << 24
    x = rng.normal(2, rng.STREAM_SIGNAL, n, device=dev, dtype=torch.float32)
    y = torch.empty_like(x)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = []
    for K in (1, 2, 4, 8):
        sos = torch.from_numpy(filters.butter_bandpass(K, 0.1, 0.2))[None].contiguous().to(dev)
        Kt = torch.full((1,), K, dtype=torch.int32, device=dev)
        roof = min(hbm_gbs * 1e9 / 8.0, sms * FP32_LANES_PER_SM * sm_max * 1e6 / (6 * K + 1)) / 1e9
        row = {"K": K, "roofline_gsamples_per_s": roof}
        for name, tunings in (("PH", [(16, 8, 1, 0), (32, 8, 1, 0), (32, 8, 1, 768),
                                      (64, 8, 1, 0), (32, 8, 1, 4), (64, 8, 1, 4)]),
                              ("CR", [(16, 8, 2, 0), (32, 8, 2, 0), (32, 8, 2, 768),
                                      (64, 8, 2, 0), (32, 8, 2, 4), (64, 8, 2, 4)])):
            best = None
            for t in tunings:
                plan = P.SosFilter([n], K, tuning=t, device=dev)
                plan.prepare(sos, Kt)
                g = graph_of(lambda: plan.apply(x, y))
                ms = replay_ms(g, steps, flush)
                if best is None or ms < best[0]:
                    best = (ms, t)
            row[name] = {"value": n / (best[0] * 1e-3) / 1e9, "tuning": list(best[1])}
        plan = P.SosFilter([n], K, tuning=(32, 8, 1, 0), device=dev)
        plan.prepare(sos, Kt)
        for name in ("scalar", "block"):
            best = None
            for sl in (256, 1024, 4096, 16384, 65536):
                g = graph_of(lambda: plan.apply_baseline(name, x, y, sl))
                ms = replay_ms(g, steps, flush)
                if best is None or ms < best[0]:
                    best = (ms, sl)
            row[name] = {"value": n / (best[0] * 1e-3) / 1e9, "seg_len": best[1]}
        for name in ("scalar", "block", "PH", "CR"):
            row[name]["frac_of_roofline"] = row[name]["value"] / roof
        out.append(row)
    return {"workload": "butter_bp(K)_0.1-0.2_1x16777216", "rows": out,
            "note": "apply only (tables prepared once), L2 flushed between steps"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tuning", default="", help="N,W (e.g. 32,8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling)")
    ap.add_argument("--clock-seconds", type=float, default=2.0)
    ap.add_argument("--clocks-out", default="")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the low-pass, batched, differentiation and stress legs")
    ap.add_argument("--leg", default="", choices=["", "backward", "batched", "stress", "compare"],
                    help="run only this extra leg and print its figures (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2607_14054_gb300 as P
    from synth import workloads
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))

    if args.leg:
        fn = {"backward": lambda: backward_leg(P, dev, world, sms, sm_max, hbm_gbs, args.steps),
              "batched": lambda: batched_leg(P, dev, world, sms, sm_max, hbm_gbs, args.steps,
                                             rank)[0],
              "stress": lambda: stress_leg(P, dev, world, sms, sm_max, hbm_gbs, args.steps)[0],
              "compare": lambda: compare_leg(P, dev, sms, sm_max, hbm_gbs, args.steps)}
        line = {"leg": args.leg, **fn[args.leg]()}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0

    wl = workloads.plain_bandpass16(n=1 << 24, device=dev)
    Kmax = wl.kmax
    if args.tuning:
        tuning = (tuple(int(v) for v in args.tuning.split(",")) + (0, 0, 0, 0))[:4]
    else:
        from paper_2607_14054_gb300.autotune import autotune
        tuning = autotune(wl.x, wl.sos, wl.K, wl.lengths, None)
    plan = P.SosFilter(wl.lengths, Kmax, tuning=tuning, device=dev)
    # the same tuning with the plan cache off: every step recomputes the
    # tables (the cost of a call whose coefficients changed)
    tr = list(tuning) + [0] * (4 - len(tuning))
    plan_re = P.SosFilter(wl.lengths, Kmax, tuning=(tr[0], tr[1], tr[2], tr[3] | 8), device=dev)
    x = wl.x
    sos = wl.sos
    K = wl.K
    y = torch.empty_like(x)
    zf = torch.empty(wl.n_channels, Kmax, 2, dtype=torch.float32, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        plan.prepare(sos, K)
        plan.apply(x, y, None, zf)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    # the step as one captured CUDA graph: sos_prepare (the plan kernel; the
    # coefficients are those of the previous step, so the plan cache keeps the
    # tables after checking them on the device), then sos_apply (the horizon
    # kernel launched early behind the plan, the look-back kernel launched
    # early behind it); the same step with the cache off, each half, and the
    # horizon kernel alone are captured too and timed in loops of their own
    g_step = graph_of(step)
    g_replan = graph_of(lambda: (plan_re.prepare(sos, K), plan_re.apply(x, y, None, zf)))
    g_prep = graph_of(lambda: plan.prepare(sos, K))
    g_prep_re = graph_of(lambda: plan_re.prepare(sos, K))
    g_apply = graph_of(lambda: plan.apply(x, y, None, zf))
    g_pipe = graph_of(lambda: plan.apply_part("pipeline", x, y, None, zf))
    st = plan.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")
    if plan.plan_recomputed() != 0:
        raise RuntimeError("the plan cache did not keep the tables")

    stream = torch.cuda.current_stream(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        g_step.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    ms_per_step = reduce_max(sum(step_ms) / len(step_ms), world)
    ms_pipe = reduce_max(replay_ms(g_pipe, args.steps, flush), world)
    ms_prep = replay_ms(g_prep, args.steps, flush)
    ms_prep_re = replay_ms(g_prep_re, args.steps, flush)
    ms_apply = reduce_max(replay_ms(g_apply, args.steps, flush), world)
    ms_replan = reduce_max(replay_ms(g_replan, args.steps, flush), world)
    samples = wl.total
    value = samples * world / (ms_per_step * 1e-3) / 1e9

    # sustained loop with clock sampling (same steps, untimed)
    clocks = None
    if args.clock_seconds > 0:
        sampler = ClockSampler(local, args.clocks_out or None)
        sampler.start()
        time.sleep(0.3)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < args.clock_seconds:
            for _ in range(50):
                flush.zero_()
                g_step.replay()
            torch.cuda.synchronize()
        clocks = sampler.stop()

    # end to end through the public API: pinned host input -> device ->
    # filter -> host output, every step; beside it the box's own pinned copy
    # rates, whose sum of both directions bounds it
    e2e = None
    if not args.no_e2e:
        e2e_value, e2e_ms, e2e_info = end_to_end(P, x, sos, stream, samples, world, args,
                                                 plan.tuning)
        rates = copy_rates(x, stream)
        copy_ms = 4 * samples / (rates["h2d"] * 1e9) * 1e3 + 4 * samples / (rates["d2h"] * 1e9) * 1e3
        serial_bound = samples / (copy_ms * 1e-3) / 1e9
        copy_bound = samples / (4 * samples / (rates["both"] * 1e9)) / 1e9
        e2e = {"value": e2e_value, "unit": "Gsamples/s", "h2d_bytes_per_step": 4 * samples,
               "d2h_bytes_per_step": 4 * samples, "ms_per_step": e2e_ms,
               "api": "paper_2607_14054_gb300.SosHostFilter (sos_filter_host; pinned host "
                      "buffers)", **e2e_info,
               "copy_gbs": {"h2d": rates["h2d"], "d2h": rates["d2h"],
                            "both_at_once_per_direction": rates["both"]},
               "copy_bound_gsamples_per_s": copy_bound,
               "frac_of_copy_bound": e2e_value / world / copy_bound,
               "serial_copy_bound_gsamples_per_s": serial_bound,
               "copy_bound_note": "input copied in and output copied out once per step, both "
                                  "directions at once, at the box's measured pinned rates; "
                                  "the serial bound has them one after the other"}

    jobs = [ParityJob("bandpass16", x, sos.cpu(), K.cpu(), wl.lengths.numpy(), None, y, 1e-5)]

    fmas = fma_per_sample(8)
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = 2.0 * fmas * samples / (ms_pipe * 1e-3) / 1e12
    kname = horizon_kernel(plan.tuning)
    traffic = profiled_traffic(kname, samples)
    roof_samples = min(hbm_gbs * 1e9 / 8.0, sms * FP32_LANES_PER_SM * sm_max * 1e6 / fmas) / 1e9

    lowpass = batched = backward = stress = None
    if not args.no_extra:
        lowpass, j = lowpass_leg(P, dev)
        jobs += j
        batched, j = batched_leg(P, dev, world, sms, sm_max, hbm_gbs, rank=rank)
        jobs += j
        backward = backward_leg(P, dev, world, sms, sm_max, hbm_gbs)
        stress, j = stress_leg(P, dev, world, sms, sm_max, hbm_gbs)
        jobs += j

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(workloads.plain_bandpass16(n=1 << 24, device="cpu"), jobs=jobs)

    line = {
        "metric": "Gsamples/s K=8 FP32 (batched/plain) and % roofline at rel-L2<=1e-5 vs FP64",
        "value": value,
        "unit": "Gsamples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "samples": samples, "channels": 1, "sections": 8,
                   "parallelism": f"replicas{world}", "l2": "flushed between steps (256 MiB write)",
                   "tuning": list(plan.tuning),
                   "tuning_source": "--tuning" if args.tuning else "autotuner (untimed setup)",
                   "step": "sos_filter on a new signal with the same filter: sos_prepare (plan "
                           "kernel; the plan cache keeps the tables after comparing the "
                           "coefficients on the device) + sos_apply (horizon kernel launched "
                           "early behind the plan, look-back kernel early behind that), one "
                           "CUDA-graph replay",
                   "headline": "ms_per_step (plan cache on)",
                   "breakdown": "ms_prepare, ms_apply, ms_horizon_kernel, ms_step_replan, "
                                "ms_prepare_replan: each replayed alone in a loop of its own",
                   "ms_prepare": ms_prep, "ms_apply": ms_apply,
                   "ms_step_replan": ms_replan, "ms_prepare_replan": ms_prep_re,
                   "value_replan": samples * world / (ms_replan * 1e-3) / 1e9,
                   "horizon_kernel": kname, "ms_horizon_kernel": ms_pipe,
                   "roofline_gsamples_per_s": roof_samples,
                   "frac_of_sample_roofline": value / world / roof_samples,
                   "wall_s_timed": t_wall},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": kname, "flops_per_sample": 2 * fmas,
                     "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                    f"{sm_max:.0f} MHz ({src} max clock)"},
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "lowpass": lowpass,
        "batched": batched,
        "backward": backward,
        "stress": stress,
        "clocks": clocks,
        "parity": cpu["parity"] if cpu else None,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
