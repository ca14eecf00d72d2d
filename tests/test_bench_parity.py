"""The bench's oracle-parity aggregation (cpu_baseline leg), on the CPU:
per-check relative L2 against the oracle, counts within tolerance, and the
optional bound relative to the sample-by-sample FP32 recursion."""
import numpy as np
import torch

import bench
import oracle
from synth import workloads


def test_parity_aggregation_and_fp32_bound():
    wl = workloads.plain_lowpass(n=4096)
    x, sos = wl.x, wl.sos[0]
    ref, _ = oracle.sosfilt(x.double().numpy(), sos.numpy())
    exact = torch.from_numpy(ref.astype(np.float32))
    off = torch.from_numpy((ref * 1.01).astype(np.float32))  # 1e-2 relative
    checks = [("a", x, sos, None, exact, 1e-5), ("a", x, sos, None, off, 1e-5),
              ("b", x, sos, None, off, 1e-3, 8.0), ("b", x, sos, None, exact, 1e-3, 8.0)]
    out = bench.oracle_baseline(wl, target_seconds=0.01, checks=checks)
    assert out["kind"] == "oracle" and out["value"] > 0
    a, b = out["parity"]["a"], out["parity"]["b"]
    assert a["channels"] == 2 and a["samples"] == 2 * 4096
    assert a["within_tolerance"] == 1 and abs(a["rel_l2"] - 1e-2) < 1e-5
    assert "within_fp32_bound" not in a
    # the FP32 recursion is far below 1e-3 on this filter, so the bound is the
    # tolerance itself: the 1e-2 output is 10x over it, the exact one within
    assert b["fp32_factor"] == 8.0 and 0 < b["fp32_sequential_rel_l2"] < 1e-5
    assert b["within_fp32_bound"] == 1 and b["within_tolerance"] == 1
    assert abs(b["worst_error_over_bound"] - 10.0) < 1e-2
