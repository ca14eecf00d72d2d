"""GPU parity of the two kernels for channels within their memory horizon
against the FP64 oracle: the warp-segment kernel (default: one warp filters a
whole segment through all K sections) and the section pipeline
(SOS_FLAG_SECTION_PIPELINE: one warp per section).  Ragged lengths around the
group and segment sizes, both solvers, b0 factoring on and off, identity and
empty channels, long-memory channels carried by the look-back in the same
call, and the full-size workloads in the benchmark's launch configuration.

Tolerance as for the forward: relative L2 per channel <= 1e-5 (pole radius
<= 0.995), final states to the same bound against the channel's largest
state value."""
import numpy as np
import pytest
import torch

from synth import rng, workloads
from test_gpu_forward import _lib, check, random_case, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

WS, PIPE = 0, 4  # warp segments (default), SOS_FLAG_SECTION_PIPELINE
WS2 = 2 << 8  # SOS_FLAG_WS_CTAS(2): warp segments, two CTAs per SM


@pytest.mark.parametrize("kernel", [WS, PIPE, WS2])
@pytest.mark.parametrize("N", [16, 32, 64])
@pytest.mark.parametrize("algo", [1, 2])
def test_horizon_kernel_ragged_multichannel(N, algo, kernel):
    G = 32 * N
    lengths = [1, 2, 3, N - 1, N, N + 1, G - 1, G, G + 1, 5 * G + 7, 0, 70_001, 200_000,
               1_000_003]
    args = random_case(600 + N + algo, lengths, 8)
    y_ref, zf_ref = run_oracle(*args)
    y, zf = run_gpu(args, tuning=(N, 8, algo, kernel))
    check(y, zf, y_ref, zf_ref, np.array(lengths), args[2].numpy(), 1e-5)


def test_warpseg_general_mode_identity_empty_and_no_state():
    lengths = [5000, 70000, 3000, 0, 1]
    x, sos, K, L, _ = random_case(610, lengths, 4, b0_zero_channel=1, with_zi=False)
    K[2] = 0
    K[3] = 3
    zi = rng.normal(611, rng.STREAM_STATE, len(lengths) * 4 * 2).view(len(lengths), 4, 2)
    y, zf = run_gpu((x, sos, K, L, None), tuning=(32, 8, 1, WS))
    off = np.concatenate([[0], np.cumsum(lengths)])
    assert np.array_equal(y[off[2]:off[3]], x[off[2]:off[3]].numpy())
    y_ref, zf_ref = run_oracle(x, sos, K, L, None)
    check(y, zf, y_ref, zf_ref, np.array(lengths), K.numpy(), 1e-5)
    # with initial states: the empty channel keeps zi as its final state
    y, zf = run_gpu((x, sos, K, L, zi), tuning=(32, 8, 1, WS))
    k3 = int(K[3])
    assert np.array_equal(zf[3, :k3], zi[3, :k3].numpy())
    y_ref, zf_ref = run_oracle(x, sos, K, L, zi)
    check(y, zf, y_ref, zf_ref, np.array(lengths), K.numpy(), 1e-5)


def test_warpseg_with_long_memory_channels():
    """Channels carried by the look-back and channels run by the warp-segment
    kernel in one call."""
    from synth import filters
    lengths = [300_000, 120_000, 250_000, 90_000]
    C, kmax = len(lengths), 8
    K = np.array([8, 6, 8, 3], dtype=np.int32)
    sos = np.zeros((C, kmax, 6))
    sos[:, :, 0] = 1.0
    sos[:, :, 3] = 1.0
    for c, k in enumerate(K):
        rmin, rmax = (0.999, 0.9999) if c % 2 == 0 else (0.5, 0.95)
        sos[c, :k] = filters.random_sections(640 + c, int(k), rmin, rmax)
    x = rng.normal(641, rng.STREAM_SIGNAL, sum(lengths))
    zi = rng.normal(641, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    args = (x, torch.from_numpy(sos), torch.from_numpy(K), torch.tensor(lengths), zi)
    y, zf = run_gpu(args, tuning=(32, 8, 1, WS))
    y_ref, zf_ref = run_oracle(*args)
    from oracle import rel_l2_per_channel
    err = rel_l2_per_channel(y, y_ref, np.array(lengths))
    assert err[1::2].max() <= 1e-5 and err[0::2].max() <= 1e-3, err


def test_warpseg_repeated_calls_identical_and_graph_replay():
    """The segment hand-out counter resets itself at the end of every launch:
    repeated calls and graph replays give bitwise the same output, whatever
    warp ran which segment."""
    P = _lib()
    lengths = [400_000, 3, 123_457, 65_536]
    x, sos, K, L, zi = random_case(650, lengths, 8)
    plan = P.SosFilter(L, 8, tuning=(32, 8, 2, WS))
    xd, sd, kd, zd = x.cuda(), sos.cuda(), K.cuda(), zi.cuda()
    y1, zf1 = plan(xd, sd, kd, zd)
    y1, zf1 = y1.clone(), zf1.clone()
    for _ in range(3):
        y2, zf2 = plan(xd, sd, kd, zd)
        assert torch.equal(y1, y2) and torch.equal(zf1, zf2)
    y = torch.empty_like(xd)
    zf = torch.empty_like(zf1)
    plan.prepare(sd, kd)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.apply(xd, y, zd, zf)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.apply(xd, y, zd, zf)
    for _ in range(3):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, y1) and torch.equal(zf, zf1)
    assert plan.device_status() == 0


@pytest.mark.parametrize("N,algo,flags", [(32, 1, 0), (16, 2, 0), (64, 1, 0), (32, 1, 3 << 8)])
def test_warpseg_bandpass16_full_size(N, algo, flags):
    wl = workloads.plain_bandpass16(device="cuda")
    args = (wl.x, wl.sos, wl.K, wl.lengths, wl.zi)
    y, zf = run_gpu(args, tuning=(N, 8, algo, flags))
    y_ref, zf_ref = run_oracle(*args)
    err = check(y, zf, y_ref, zf_ref, wl.lengths.numpy(), wl.K.cpu().numpy(), 1e-5)
    print("bandpass16 warp segments", N, algo, flags, "rel-L2", float(err.max()))


def test_warpseg_batched_full_size_sampled_channels():
    wl = workloads.batched(device="cuda")
    y, zf = run_gpu((wl.x, wl.sos, wl.K, wl.lengths, wl.zi), tuning=(32, 8, 1, WS))
    C = wl.n_channels
    pick = sorted(set([0, 1, C - 1] + list(range(7, C, C // 45))))
    off = np.concatenate([[0], np.cumsum(wl.lengths.numpy())])
    xs = torch.cat([wl.x[off[c]:off[c + 1]].cpu() for c in pick])
    ls = wl.lengths[pick]
    y_ref, zf_ref = run_oracle(xs, wl.sos[pick], wl.K[pick], ls, wl.zi[pick])
    ys = np.concatenate([y[off[c]:off[c + 1]] for c in pick])
    err = check(ys, zf[pick], y_ref, zf_ref, ls.numpy(), wl.K[pick].cpu().numpy(), 1e-5)
    print("batched warp segments rel-L2 max", float(err.max()))
