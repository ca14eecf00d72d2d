"""The low-latency streaming mode (sos_stream): a signal filtered block by
block, one launch per block, the state carried on the device, must equal the
one-shot result of the oracle (the final state too), whatever the block
length, including blocks shorter than a group, ragged against it, and single
samples."""
import numpy as np
import pytest
import torch

import oracle
from synth import rng, workloads
from test_gpu_forward import _lib, check, random_case

pytestmark = pytest.mark.gpu


def _stream(P, x2d, sos, K, zi, chunk, tuning=None):
    C, T = x2d.shape
    st = P.SosStream(sos.cuda(), chunk, K=K.cuda(), zi=zi.cuda() if zi is not None else None,
                     tuning=tuning)
    out = torch.empty_like(x2d)
    nblk = T // chunk
    for b in range(nblk):
        blk = x2d[:, b * chunk:(b + 1) * chunk].contiguous()
        out[:, b * chunk:(b + 1) * chunk] = st(blk)
    assert st.plan.device_status() == 0
    return out, st.state


@pytest.mark.parametrize("chunk,tuning", [(256, None), (1000, None), (4096, (32, 8, 1, 0)),
                                          (3000, (64, 8, 1, 0))])
def test_stream_blocks_match_one_shot(chunk, tuning):
    P = _lib()
    C, T = 6, 1 << 20
    T = (T // chunk) * chunk
    x, sos, K, L, zi = random_case(91, [T] * C, 8, rmax=0.97)
    K[1] = 3
    K[4] = 0
    x2d = x.view(C, T).cuda()
    y, state = _stream(P, x2d, sos, K, zi, chunk, tuning)
    y_ref, zf_ref = oracle.sosfilt(x.double().numpy(), sos.numpy(), K=K.numpy(), lengths=L.numpy(),
                                   zi=zi.double().numpy())
    zf = state.cpu().numpy().copy()
    for c in range(C):  # rows past K keep the caller's state; the oracle writes 0
        zf[c, int(K[c]):] = 0.0
    check(y.reshape(-1).cpu().numpy(), zf, y_ref, zf_ref, L.numpy(), K.numpy(), 1e-5)


def test_stream_single_samples_and_short_blocks():
    """Blocks of 1 and 7 samples (far below one group), alternating, on the
    16th-order band-pass."""
    P = _lib()
    wl = workloads.plain_bandpass16(n=4096)
    x = wl.x.cuda()
    st = P.SosStream(wl.sos.cuda(), 1)
    st7 = None
    out = []
    pos = 0
    use_seven = False
    while pos < 4096:
        if use_seven and pos + 7 <= 4096:
            if st7 is None:
                st7 = P.SosStream(wl.sos.cuda(), 7)
            st7.state.copy_(st.state)
            out.append(st7(x[pos:pos + 7].contiguous().view(1, 7)).view(-1))
            st.state.copy_(st7.state)
            pos += 7
        else:
            out.append(st(x[pos:pos + 1].contiguous().view(1, 1)).view(-1))
            pos += 1
        use_seven = not use_seven
    y = torch.cat(out)
    ref, zf_ref = oracle.sosfilt(wl.x.double().numpy(), wl.sos.numpy())
    err = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    zf = st.state.cpu().double().numpy()
    assert np.linalg.norm(zf - zf_ref) <= 1e-5 * np.linalg.norm(zf_ref)


def test_stream_rejects_bad_arguments():
    P = _lib()
    wl = workloads.plain_lowpass(n=256)
    st = P.SosStream(wl.sos.cuda(), 256)
    with pytest.raises(ValueError):
        st(torch.zeros(255, device="cuda"))
    # overlapping x and y, or zi and zf
    buf = torch.zeros(512, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    r = P._abi.sos_stream(buf.data_ptr(), buf.data_ptr() + 4, st.state.data_ptr(), 0, 1, 1, 256,
                          0, st.plan.workspace.data_ptr(), st.plan.ws_bytes, st.plan.tuning,
                          stream)
    assert r == -1
    r = P._abi.sos_stream(buf.data_ptr(), buf.data_ptr() + 2048, st.state.data_ptr(),
                          st.state.data_ptr(), 1, 1, 256, 0, st.plan.workspace.data_ptr(),
                          st.plan.ws_bytes, st.plan.tuning, stream)
    assert r == -1
    # unknown flags
    r = P._abi.sos_stream(buf.data_ptr(), buf.data_ptr() + 2048, 0, 0, 1, 1, 256, 6,
                          st.plan.workspace.data_ptr(), st.plan.ws_bytes, st.plan.tuning, stream)
    assert r == -1


def test_stream_long_blocks_cut_into_segments():
    """Blocks of 2^17 samples of short-memory channels, cut into several
    warm-up segments per block inside one launch, three blocks in a row
    against the one-shot oracle (the state handed between blocks)."""
    P = _lib()
    C, chunk = 3, 1 << 17
    T = 3 * chunk
    x, sos, K, L, zi = random_case(95, [T] * C, 4, rmax=0.9)
    y, state = _stream(P, x.view(C, T).cuda(), sos, K, zi, chunk, (32, 8, 1, 0))
    y_ref, zf_ref = oracle.sosfilt(x.double().numpy(), sos.numpy(), K=K.numpy(),
                                   lengths=L.numpy(), zi=zi.double().numpy())
    zf = state.cpu().numpy().copy()
    for c in range(C):
        zf[c, int(K[c]):] = 0.0
    check(y.reshape(-1).cpu().numpy(), zf, y_ref, zf_ref, L.numpy(), K.numpy(), 1e-5)


def test_stream_double_float_channels():
    """Cascades the plan puts in precision class 3 (a double-float range of
    sections around the hand-offs its error estimate blames), taken from the
    batched workload's random bank, streamed in 4096-sample blocks: every
    block through the class-3 segment code, against the one-shot oracle at
    1e-5, final states included."""
    P = _lib()
    C, kmax = 4096, 8
    K = rng.randint(3, rng.STREAM_SECTIONS, C, 1, kmax).to(torch.int32)
    bank = workloads._random_bank(3, C, kmax, 0.5, 0.995, K.numpy())
    probe = P.SosFilter([8192] * C, kmax)
    probe.prepare(torch.from_numpy(bank).cuda(), K.cuda())
    ext = probe.plan_extended().numpy()
    pick = [int(c) for c in np.nonzero(ext == 3)[0][:4]]
    assert len(pick) == 4, ext
    sos = torch.from_numpy(bank[pick]).contiguous()
    Kp = K[pick].contiguous()
    T, chunk = 1 << 18, 4096
    x = rng.normal(97, rng.STREAM_SIGNAL, 4 * T)
    zi = rng.normal(98, rng.STREAM_STATE, 4 * kmax * 2).view(4, kmax, 2)
    for c in range(4):
        zi[c, int(Kp[c]):] = 0.0
    y, state = _stream(P, x.view(4, T).cuda(), sos, Kp, zi, chunk, (16, 8, 1, 0))
    L = torch.full((4,), T, dtype=torch.int64)
    y_ref, zf_ref = oracle.sosfilt(x.double().numpy(), sos.numpy(), K=Kp.numpy(),
                                   lengths=L.numpy(), zi=zi.double().numpy())
    zf = state.cpu().numpy().copy()
    for c in range(4):
        zf[c, int(Kp[c]):] = 0.0
    check(y.reshape(-1).cpu().numpy(), zf, y_ref, zf_ref, L.numpy(), Kp.numpy(), 1e-5)
