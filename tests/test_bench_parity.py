"""The bench's oracle-parity jobs (cpu_baseline leg), on the CPU: per-channel
relative L2 against the oracle over whole channels and windows, counts within
tolerance."""
import numpy as np
import torch

import bench
import oracle
from synth import workloads


def test_parity_jobs_whole_channels_and_windows():
    wl = workloads.batched(n_channels=5, min_len=3000, max_len=9000, seed=9)
    ref, _ = oracle.sosfilt(wl.x.double().numpy(), wl.sos.numpy(), K=wl.K.numpy(),
                            lengths=wl.lengths.numpy(), zi=wl.zi.double().numpy())
    exact = torch.from_numpy(ref.astype(np.float32))
    off = np.concatenate([[0], np.cumsum(wl.lengths.numpy())])
    bad = exact.clone()
    c = 3
    n = int(wl.lengths[c])
    # channel 3: its last fifth 1 % off (whole-channel error below 1 %)
    bad[off[c] + n - n // 5:off[c + 1]] *= 1.01
    jobs = [bench.ParityJob("ok", wl.x, wl.sos, wl.K, wl.lengths.numpy(), wl.zi, exact, 1e-5,
                            windows=5, chunk=2),
            bench.ParityJob("bad", wl.x, wl.sos, wl.K, wl.lengths.numpy(), wl.zi, bad, 1e-3,
                            windows=5, chunk=3),
            bench.ParityJob("some", wl.x, wl.sos, wl.K, wl.lengths.numpy(), wl.zi, bad, 1e-3,
                            channels=[0, 3])]
    out = bench.oracle_baseline(wl, target_seconds=0.01, jobs=jobs)
    assert out["kind"] == "oracle" and out["value"] > 0
    ok, b, some = out["parity"]["ok"], out["parity"]["bad"], out["parity"]["some"]
    assert ok["channels"] == 5 and ok["samples"] == int(wl.lengths.sum())
    assert ok["within_tolerance"] == 5 and ok["within_tolerance_every_window"] == 5
    assert ok["rel_l2"] < 1e-6 and ok["worst_window_rel_l2"] < 1e-6
    # the windows catch what the whole-channel error may average away
    assert b["within_tolerance_every_window"] == 4 and b["within_tolerance"] >= 4
    assert abs(b["worst_window_rel_l2"] - 1e-2) < 1e-4
    assert some["channels"] == 2 and some["rel_l2"] > 1e-4
