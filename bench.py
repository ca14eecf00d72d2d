#!/usr/bin/env python3
"""Benchmark of the cascaded-biquad hot path on GB300.

One step = one full call of the C ABI's sos_filter on the 16th-order (K = 8)
Butterworth band-pass workload, 2^24 FP32 samples i.i.d. N(0, 1), one
channel, zero initial state, inputs resident in HBM: sos_prepare (plan and
dispatch order, one kernel) then sos_apply (the kernel for channels within
their memory horizon -- warp segments or the section pipeline -- launched
early behind the plan, then the look-back kernel, which finds no carried
channel here, launched early behind that), replayed as one CUDA graph.  The
tuning (N, W, solver, kernel) is chosen by the library's autotuner before the
timed region.
Prints one JSON line (rank 0), with the batched (4096 channels),
differentiation (forward + backward, 256 x 2^16) and precision-stress
(64 x 2^26, poles at radius 0.999..0.9999) workloads as extra fields.

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


def oracle_baseline(wl, target_seconds: float = 10.0, checks=()):
    """Times the FP64 oracle (as it stands) on the host cores: whole-signal
    passes of the workload, repeated until ~target_seconds of CPU work.  Also
    runs it on each check (name, x prefix, sos rows, zi rows or None, GPU
    output prefix, tolerance[, factor]): the relative L2 error of the GPU path
    against the oracle on causal prefixes of the benchmarked workloads.  With a
    factor, the same filter run sample by sample in FP32 (scipy's sosfilt on
    float32 data: what FP32 arithmetic itself gives on that channel) is
    measured beside it, and the channel also counts as within
    max(tolerance, factor x that error)."""
    import numpy as np
    import oracle
    parity = {}
    for chk in checks:
        name, xs, sos_c, zi_c, yg, tol = chk[:6]
        factor = chk[6] if len(chk) > 6 else None
        zi_o = None if zi_c is None else zi_c.double().numpy().reshape(1, -1, 2)
        ref, _ = oracle.sosfilt(xs.double().numpy(), sos_c.numpy(), zi=zi_o)
        nref = np.linalg.norm(ref)
        err = float(np.linalg.norm(yg.double().numpy() - ref) / nref)
        prev = parity.get(name)
        if prev is None:
            prev = parity[name] = {"rel_l2": 0.0, "tolerance": tol, "channels": 0,
                                   "samples": 0, "within_tolerance": 0}
            if factor is not None:
                prev.update({"fp32_sequential_rel_l2": 0.0, "fp32_factor": factor,
                             "within_fp32_bound": 0, "worst_error_over_bound": 0.0})
        prev["rel_l2"] = max(prev["rel_l2"], err)
        prev["channels"] += 1
        prev["samples"] += int(xs.numel())
        prev["within_tolerance"] += int(err <= tol)
        if factor is not None:
            import scipy.signal
            zi32 = None if zi_c is None else zi_c.numpy().astype(np.float32)
            x32 = xs.numpy().astype(np.float32)
            s32 = sos_c.numpy().astype(np.float32)
            y32 = (scipy.signal.sosfilt(s32, x32) if zi32 is None
                   else scipy.signal.sosfilt(s32, x32, zi=zi32)[0])
            e32 = float(np.linalg.norm(y32.astype(np.float64) - ref) / nref)
            prev["fp32_sequential_rel_l2"] = max(prev["fp32_sequential_rel_l2"], e32)
            bound = max(tol, factor * e32)
            prev["within_fp32_bound"] += int(err <= bound)
            prev["worst_error_over_bound"] = max(prev["worst_error_over_bound"], err / bound)
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
    return {"value": samples / el / 1e9, "unit": "Gsamples/s", "cores": int(threads),
            "kind": "oracle",
            "sample": f"{reps} full passes of the {x.size}-sample workload ({el:.1f} s); "
                      f"FP64 sample-by-sample cascade, one thread per channel",
            "seconds": el, "parity": parity}


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


def end_to_end(P, x, sos, stream, samples, world, args, tuning):
    """Same metric through the public API with host buffers: pinned host
    input -> device -> sosfilt -> host output, every step."""
    import torch
    xh = torch.empty(samples, dtype=torch.float32, pin_memory=True)
    xh.copy_(x)
    yh = torch.empty(samples, dtype=torch.float32, pin_memory=True)
    xd = torch.empty_like(x)
    e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        xd.copy_(xh, non_blocking=True)
        step_e2e_y = P.sosfilt(xd, sos, tuning=tuning)
        yh.copy_(step_e2e_y[0], non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        xd.copy_(xh, non_blocking=True)
        yd, zfd = P.sosfilt(xd, sos, tuning=tuning)
        yh.copy_(yd, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps
    e2e_ms = reduce_max(e2e_ms, world)
    e2e_value = samples * world / (e2e_ms * 1e-3) / 1e9
    return e2e_value, e2e_ms



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


def batched_leg(P, dev, world, sms, sm_max, hbm_gbs, steps: int = 5):
    """4096 channels, lengths U[2^10, 2^20], K U{1..8}, random sections,
    nonzero zi: one prepare + apply per step, inputs resident."""
    import torch
    from synth import workloads
    from paper_2607_14054_gb300.autotune import autotune
    wl = workloads.batched(device=dev)
    tuning = autotune(wl.x, wl.sos, wl.K, wl.lengths, wl.zi)
    plan = P.SosFilter(wl.lengths, wl.kmax, tuning=tuning, device=dev)
    y = torch.empty_like(wl.x)
    zf = torch.empty(wl.n_channels, wl.kmax, 2, device=dev)
    for _ in range(2):
        plan(wl.x, wl.sos, wl.K, wl.zi, y=y, zf=zf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan(wl.x, wl.sos, wl.K, wl.zi, y=y, zf=zf)
    e1.record()
    torch.cuda.synchronize()
    if plan.device_status() != 0:
        raise RuntimeError("batched leg: device status")
    ms = reduce_max(e0.elapsed_time(e1) / steps, world)
    total = wl.total
    lens = wl.lengths.double()
    fma = float((lens * (6 * wl.K.cpu().double() + 1)).sum())
    t_hbm = 8.0 * total / (hbm_gbs * 1e9)
    t_alu = fma / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    roof = total / max(t_hbm, t_alu) / 1e9
    value = total * world / (ms * 1e-3) / 1e9
    off = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(wl.lengths, 0)])
    checks = []
    for c in range(0, wl.n_channels, 64):
        a = int(off[c])
        n = min(int(wl.lengths[c]), 1 << 16)
        k = int(wl.K[c])
        checks.append(("batched", wl.x[a:a + n].cpu(), wl.sos[c, :k].cpu(),
                       wl.zi[c, :k].cpu(), y[a:a + n].cpu(), 1e-5))
    return {"workload": wl.name, "channels": wl.n_channels, "samples": total,
            "value": value, "unit": "Gsamples/s", "ms_per_step": ms,
            "roofline_gsamples_per_s": roof, "frac_of_roofline": value / world / roof,
            "bound": "hbm" if t_hbm >= t_alu else "alu", "tuning": list(tuning),
            "step": "sos_filter (prepare + apply)"}, checks


# the precision-stress channels' bound relative to the sample-by-sample FP32
# recursion's own error (the block method rounds at more places: the lane
# scan, the fold, the particular and the re-run)
STRESS_FP32_FACTOR = 8.0


def stress_leg(P, dev, world, sms, sm_max, hbm_gbs, steps: int = 3):
    """Precision stress: 64 x 2^26 samples, K = 8, poles at radius
    0.999..0.9999 (long memory horizons, per-channel segments), autotuned
    (untimed), one prepare + apply per step.  Returns the leg's figures and the first 2^16 outputs of
    every channel (causal prefixes) for the oracle check."""
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
    hz, _ = plan.plan_info()
    ext = plan.plan_extended()
    L = int(wl.lengths[0])
    n = 1 << 16
    checks = [("stress", wl.x[c * L:c * L + n].cpu(), wl.sos[c].cpu(), None,
               y[c * L:c * L + n].cpu(), 1e-3, STRESS_FP32_FACTOR) for c in range(wl.n_channels)]
    total = wl.total
    fma = 49.0 * total
    t_hbm = 8.0 * total / (hbm_gbs * 1e9)
    t_alu = fma / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    roof = total / max(t_hbm, t_alu) / 1e9
    value = total * world / (ms * 1e-3) / 1e9
    return {"workload": wl.name, "channels": wl.n_channels, "samples": total,
            "value": value, "unit": "Gsamples/s", "ms_per_step": ms,
            "roofline_gsamples_per_s": roof, "frac_of_roofline": value / world / roof,
            "carried_channels": int((hz < 0).sum()),
            "extended_precision_channels": int(ext.sum()),
            "tuning": list(plan.tuning), "step": "sos_filter (prepare + apply)"}, checks


def backward_leg(P, dev, world, steps: int = 5):
    """256 x 2^16, K = 8: forward + backward through the autograd Function."""
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
    return {"workload": wl.name, "samples": wl.total,
            "value": wl.total * world / (ms * 1e-3) / 1e9, "unit": "Gsamples/s",
            "ms_per_step": ms, "step": "forward + MSE + backward (dL/dx, dL/dsos, dL/dzi)"}


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
                    help="skip the batched and differentiation legs")
    ap.add_argument("--leg", default="", choices=["", "backward"],
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

    if args.leg == "backward":
        line = {"leg": "backward", **backward_leg(P, dev, world, steps=args.steps)}
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
    # each half of the step is replayed from a captured CUDA graph (one launch
    # each), so the timed region holds no host-side launch gaps
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream(dev).wait_stream(side)
    # the step as one captured CUDA graph: sos_prepare (the plan kernel), then
    # sos_apply (the horizon kernel launched early behind the plan, the
    # look-back kernel launched early behind it); each half and the horizon
    # kernel alone are captured too and timed in loops of their own for the
    # breakdown and the roofline
    g_step, g_prep, g_apply, g_pipe = (torch.cuda.CUDAGraph() for _ in range(4))
    with torch.cuda.graph(g_step):
        plan.prepare(sos, K)
        plan.apply(x, y, None, zf)
    with torch.cuda.graph(g_prep):
        plan.prepare(sos, K)
    with torch.cuda.graph(g_apply):
        plan.apply(x, y, None, zf)
    with torch.cuda.graph(g_pipe):
        plan.apply_part("pipeline", x, y, None, zf)
    torch.cuda.synchronize()

    def step():  # noqa: F811 - the captured form of the same step
        g_step.replay()
    st = plan.device_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

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

    def loop_ms(g):
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            g.replay()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [e[0].elapsed_time(e[1]) for e in evs]
    pipe_ms = loop_ms(g_pipe)
    prep_ms = loop_ms(g_prep)
    apply_ms = loop_ms(g_apply)
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    ms_per_step = sum(step_ms) / len(step_ms)
    ms_apply = sum(apply_ms) / len(apply_ms)
    ms_pipe = reduce_max(sum(pipe_ms) / len(pipe_ms), world)
    ms_per_step = reduce_max(ms_per_step, world)
    ms_apply = reduce_max(ms_apply, world)
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
                step()
            torch.cuda.synchronize()
        clocks = sampler.stop()

    # end to end through the public API: pinned host input -> device ->
    # filter -> host output, every step
    e2e_value, e2e_ms = None, None
    if not args.no_e2e:
        e2e_value, e2e_ms = end_to_end(P, x, sos, stream, samples, world, args, plan.tuning)

    # causal prefix of the output for the oracle check of the cpu_baseline leg
    checks = [("bandpass16", x[:1 << 20].cpu(), sos[0].cpu(), None, y[:1 << 20].cpu(), 1e-5)]

    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    fmas = fma_per_sample(8)
    achieved = 2.0 * fmas * samples / (ms_pipe * 1e-3) / 1e12
    kname = horizon_kernel(plan.tuning)
    traffic = profiled_traffic(kname, samples)
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    roof_samples = min(hbm_gbs * 1e9 / 8.0, sms * FP32_LANES_PER_SM * sm_max * 1e6 / fmas) / 1e9

    batched = backward = stress = None
    if not args.no_extra:
        batched, c_b = batched_leg(P, dev, world, sms, sm_max, hbm_gbs)
        backward = backward_leg(P, dev, world)
        stress, c_s = stress_leg(P, dev, world, sms, sm_max, hbm_gbs)
        checks += c_b + c_s

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(workloads.plain_bandpass16(n=1 << 24, device="cpu"), checks=checks)

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
                   "step": "sos_prepare + sos_apply (one CUDA-graph replay: plan kernel, "
                           "horizon kernel launched early behind it, look-back kernel "
                           "launched early behind that)",
                   "breakdown": "ms_prepare, ms_apply, ms_horizon_kernel: each part "
                                "replayed alone in a loop of its own",
                   "ms_prepare": sum(prep_ms) / len(prep_ms), "ms_apply": ms_apply,
                   "horizon_kernel": kname, "ms_horizon_kernel": ms_pipe,
                   "roofline_gsamples_per_s": roof_samples,
                   "frac_of_sample_roofline": value / world / roof_samples,
                   "wall_s_timed": t_wall},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": kname, "flops_per_sample": 2 * fmas,
                     "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                    f"{sm_max:.0f} MHz ({src} max clock)"},
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": "Gsamples/s", "h2d_bytes_per_step": 4 * samples,
            "d2h_bytes_per_step": 4 * samples, "ms_per_step": e2e_ms,
            "api": "paper_2607_14054_gb300.sosfilt (pinned host buffers)"},
        "gpu_launches": 3 * args.steps,
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
