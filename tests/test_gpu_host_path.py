"""The host-to-host entry point (sos_filter_host): the signal in pinned host
memory, cut into blocks whose copy in, filtering and copy out overlap, must
equal the one-shot oracle -- including a channel cut into time pieces whose
states are handed on between blocks, groups of whole channels, ragged
lengths, empty channels and the final states."""
import numpy as np
import pytest
import torch

import oracle
from synth import workloads
from test_gpu_forward import _lib, check, random_case

pytestmark = pytest.mark.gpu


def _pinned(t):
    h = torch.empty(t.numel(), dtype=torch.float32, pin_memory=True)
    h.copy_(t.reshape(-1))
    return h


@pytest.mark.parametrize("block,tuning", [(1 << 18, None), (100_000, (32, 8, 1, 4)),
                                          (1 << 20, (16, 8, 1, 0))])
def test_host_path_matches_oracle(block, tuning):
    P = _lib()
    # a channel several blocks long (time pieces, ragged last), short ones
    # grouped, an empty one, a K = 0 one
    lengths = [700_001, 1, 8192, 0, 33_333, 250_000, 5]
    x, sos, K, L, zi = random_case(171, lengths, 6, rmax=0.97)
    K[2] = 0
    xh = _pinned(x)
    plan = P.SosHostFilter(L, 6, tuning=tuning, block=block)
    yh, zf = plan(xh, sos.cuda(), K.cuda(), zi.cuda())
    torch.cuda.synchronize()
    assert plan.block <= max(block, 4) + 3
    y_ref, zf_ref = oracle.sosfilt(x.double().numpy(), sos.numpy(), K=K.numpy(),
                                   lengths=L.numpy(), zi=zi.double().numpy())
    check(yh.numpy(), zf.cpu().numpy(), y_ref, zf_ref, L.numpy(), K.numpy(), 1e-5)


def test_host_path_repeated_calls_and_default_blocks():
    """The band-pass, 2^22 samples, default block (an eighth): two calls in
    a row through sosfilt_host give the oracle's output each time."""
    P = _lib()
    wl = workloads.plain_bandpass16(n=1 << 22)
    xh = _pinned(wl.x)
    ref, _ = oracle.sosfilt(wl.x.double().numpy(), wl.sos.numpy())
    for _ in range(2):
        yh, zf = P.sosfilt_host(xh, wl.sos.cuda())
        err = np.linalg.norm(yh.double().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, err
        yh.zero_()


def test_host_path_rejects_small_buffers():
    P = _lib()
    lengths = torch.tensor([4096], dtype=torch.int64)
    plan = P.SosHostFilter(lengths, 1, block=1024)
    sos = workloads.plain_lowpass(n=4096).sos.cuda()
    xh = torch.zeros(4096, pin_memory=True)
    yh = torch.zeros(4096, pin_memory=True)
    stream = torch.cuda.current_stream().cuda_stream
    r = P._abi.sos_filter_host(xh.data_ptr(), sos.data_ptr(),
                               torch.ones(1, dtype=torch.int32, device="cuda").data_ptr(), 1, 1,
                               plan.lengths.data_ptr(), plan.lengths_host.data_ptr(), 0,
                               yh.data_ptr(), 0, plan.workspace.data_ptr(), plan.ws_bytes,
                               plan.staging.data_ptr(), plan.staging_bytes - 16, plan.block,
                               plan.tuning, stream)
    assert r == -5  # SOS_ERR_WORKSPACE
    with pytest.raises(ValueError):
        plan(xh.cuda(), sos)
