"""GPU parity of the forward cascade (CUDA path through the C ABI) against the
FP64 oracle, element by element, on seeded inputs.

Tolerance: relative L2 error per channel, ||y_gpu - y_oracle|| / ||y_oracle||,
<= 1e-5 for pole radius <= 0.995 and <= 1e-3 for the 0.999..0.9999 stress
workload (the accuracy targets of the method's FP32-bulk / FP64-transition
design); final states are held to the same relative bound against the
channel's largest state value."""
import numpy as np
import pytest
import torch

import oracle
from synth import rng, workloads

pytestmark = pytest.mark.gpu

TUNINGS = [(32, 8), (16, 8), (64, 4), (32, 4), (32, 16), (16, 16), (64, 8), (32, 7), (64, 3)]


def _lib():
    import paper_2607_14054_gb300 as P
    P.build()
    return P


def run_gpu(wl_or_args, tuning=None, zf=True):
    P = _lib()
    x, sos, K, lengths, zi = wl_or_args
    plan = P.SosFilter(lengths, sos.shape[1], tuning=tuning)
    y, zfo = plan(x.cuda(), sos.cuda(), K.cuda(), zi.cuda() if zi is not None else None,
                  want_zf=zf)
    st = plan.device_status()
    assert st == 0, P._abi.STATUS_NAMES.get(st, st)
    return y.cpu().numpy(), (zfo.cpu().numpy() if zfo is not None else None)


def run_oracle(x, sos, K, lengths, zi):
    return oracle.sosfilt(x.cpu().double().numpy(), sos.cpu().numpy(), K=K.cpu().numpy(),
                          lengths=lengths.cpu().numpy(),
                          zi=zi.cpu().double().numpy() if zi is not None else None)


def check(y, zf, y_ref, zf_ref, lengths, K, tol, zf_tol=None):
    err = oracle.rel_l2_per_channel(y, y_ref, lengths)
    assert np.all(np.isfinite(y))
    assert err.max() <= tol, (err.max(), int(err.argmax()))
    if zf is not None:
        zf_tol = tol if zf_tol is None else zf_tol
        for c in range(len(lengths)):
            k = int(K[c])
            if k == 0:
                continue
            ref = zf_ref[c, :k]
            scale = max(np.max(np.abs(ref)), 1e-30)
            d = np.max(np.abs(zf[c, :k] - ref)) / scale
            assert d <= zf_tol * 10, (c, d)
    return err


def random_case(seed, lengths, kmax, rmax=0.95, with_zi=True, b0_zero_channel=None):
    C = len(lengths)
    lengths = torch.tensor(lengths, dtype=torch.int64)
    K = rng.randint(seed, rng.STREAM_SECTIONS, C, 0 if kmax > 1 else 1, kmax).to(torch.int32)
    K[0] = kmax
    sos = workloads._random_bank(seed, C, kmax, 0.3, rmax, K.numpy())
    if b0_zero_channel is not None:
        sos[b0_zero_channel, 0, 0] = 0.0  # first section has no direct path: general mode
    sos = torch.from_numpy(sos)
    # exercise a0 != 1 normalisation
    scale = 0.5 + rng.uniform(seed, rng.STREAM_MISC, C * kmax).reshape(C, kmax, 1).double()
    sos = sos * scale
    x = rng.normal(seed, rng.STREAM_SIGNAL, int(lengths.sum()))
    zi = rng.normal(seed, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2) if with_zi else None
    return x, sos.contiguous(), K, lengths, zi


def test_lowpass_8192_all_tunings():
    wl = workloads.plain_lowpass()
    args = (wl.x, wl.sos, wl.K, wl.lengths, wl.zi)
    y_ref, zf_ref = run_oracle(*args)
    for N, W in TUNINGS:
        y, zf = run_gpu(args, tuning=(N, W, 0, 0))
        check(y, zf, y_ref, zf_ref, wl.lengths.numpy(), wl.K.numpy(), 1e-5)


@pytest.mark.parametrize("N,W", TUNINGS)
def test_ragged_multichannel(N, W):
    T = N * 32 * W
    lengths = [1, 2, 3, N - 1, N, N + 1, 32 * N - 1, 32 * N + 1, T - 1, T, T + 1, 3 * T + 5,
               0, 7 * T + 333]
    args = random_case(100 + N + W, lengths, 8)
    y_ref, zf_ref = run_oracle(*args)
    y, zf = run_gpu(args, tuning=(N, W, 0, 0))
    check(y, zf, y_ref, zf_ref, np.array(lengths), args[2].numpy(), 1e-5)


def test_general_mode_b0_zero_and_no_state():
    lengths = [5000, 70000, 1]
    args = random_case(7, lengths, 4, b0_zero_channel=1, with_zi=False)
    y_ref, zf_ref = run_oracle(*args)
    y, zf = run_gpu(args)
    check(y, zf, y_ref, zf_ref, np.array(lengths), args[2].numpy(), 1e-5)
    y2, zf2 = run_gpu(args, zf=False)
    assert zf2 is None and np.array_equal(y, y2)


def test_identity_channel_and_empty_channel():
    lengths = [3000, 0, 20000]
    x, sos, K, L, zi = random_case(9, lengths, 3)
    K[:] = torch.tensor([0, 2, 3], dtype=torch.int32)
    y, zf = run_gpu((x, sos, K, L, zi))
    assert np.array_equal(y[:3000], x[:3000].numpy())
    assert np.array_equal(zf[1, :2], zi[1, :2].numpy())        # empty channel keeps zi
    assert np.all(zf[0] == 0) and np.all(zf[1, 2:] == 0)
    y_ref, zf_ref = run_oracle(x, sos, K, L, zi)
    check(y, zf, y_ref, zf_ref, np.array(lengths), K.numpy(), 1e-5)


def test_streaming_chunks_match_one_shot():
    """zf of one call fed as zi of the next reproduces the one-shot result."""
    P = _lib()
    wl = workloads.plain_bandpass16(n=300_000)
    x = wl.x.cuda()
    sos = wl.sos.cuda()
    y_full, zf_full = P.sosfilt(x, sos, check=True)
    zi = torch.zeros(1, 8, 2, device="cuda")
    parts = []
    for a, b in [(0, 1), (1, 77777), (77777, 77778), (77778, 300_000)]:
        yp, zi = P.sosfilt(x[a:b].contiguous(), sos, zi=zi, check=True)
        parts.append(yp)
    y_chunks = torch.cat(parts)
    d = (y_chunks - y_full).norm() / y_full.norm()
    assert d.item() <= 2e-6
    assert torch.allclose(zi, zf_full, rtol=1e-4, atol=1e-6)


def test_repeated_calls_are_deterministic_and_graph_capturable():
    P = _lib()
    args = random_case(11, [100_000, 250_000, 4097], 8)
    x, sos, K, L, zi = (a.cuda() if a is not None and a.dtype != torch.int64 else a for a in args)
    plan = P.SosFilter(L, 8)
    y1, zf1 = plan(x, sos, K, zi)
    y2, zf2 = plan(x, sos, K, zi)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2) and torch.equal(zf1, zf2)
    yg = torch.empty_like(x)
    zfg = torch.empty_like(zf1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan(x, sos, K, zi, y=yg, zf=zfg)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan(x, sos, K, zi, y=yg, zf=zfg)
    yg.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(yg, y1) and torch.equal(zfg, zf1)
    assert plan.device_status() == 0


def test_device_side_coefficient_errors():
    P = _lib()
    args = list(random_case(12, [1000, 2000], 2))
    sos = args[1].clone()
    sos[1, 0, 3] = 0.0  # a0 == 0
    plan = P.SosFilter(args[3], 2)
    plan(args[0].cuda(), sos.cuda(), args[2].cuda(), args[4].cuda())
    assert plan.device_status() == -7
    # unstable pole with the stability check on
    sos = args[1].clone()
    sos[0, 0, 3:] = torch.tensor([1.0, -2.0, 1.01], dtype=torch.float64)
    plan = P.SosFilter(args[3], 2, tuning=(0, 0, 0, 1))
    plan(args[0].cuda(), sos.cuda(), args[2].cuda(), args[4].cuda())
    assert plan.device_status() == -2
    # and a clean call afterwards on the same workspace reports OK
    plan(args[0].cuda(), args[1].cuda(), args[2].cuda(), args[4].cuda())
    assert plan.device_status() == 0


def test_bandpass16_full_size():
    """The 16th-order Butterworth band-pass on 2^24 samples, every output
    against the oracle, in the launch configuration the benchmark times."""
    wl = workloads.plain_bandpass16(device="cuda")
    args = (wl.x, wl.sos, wl.K, wl.lengths, wl.zi)
    y, zf = run_gpu(args)
    y_ref, zf_ref = run_oracle(*args)
    err = check(y, zf, y_ref, zf_ref, wl.lengths.numpy(), wl.K.cpu().numpy(), 1e-5)
    print("bandpass16 rel-L2", float(err.max()))


def test_batched_full_size_sampled_channels():
    """4096 channels of uneven length, K in 1..8, nonzero states: the whole
    batch runs in one launch; 48 channels (first, last and spread) are
    checked in full against the oracle."""
    wl = workloads.batched(device="cuda")
    y, zf = run_gpu((wl.x, wl.sos, wl.K, wl.lengths, wl.zi))
    C = wl.n_channels
    pick = sorted(set([0, 1, C - 1] + list(range(5, C, C // 45))))
    off = np.concatenate([[0], np.cumsum(wl.lengths.numpy())])
    xs = torch.cat([wl.x[off[c]:off[c + 1]].cpu() for c in pick])
    ls = wl.lengths[pick]
    y_ref, zf_ref = run_oracle(xs, wl.sos[pick], wl.K[pick], ls, wl.zi[pick])
    ys = np.concatenate([y[off[c]:off[c + 1]] for c in pick])
    err = check(ys, zf[pick], y_ref, zf_ref, ls.numpy(), wl.K[pick].cpu().numpy(), 1e-5)
    print("batched rel-L2 max", float(err.max()), "median", float(np.median(err)))
