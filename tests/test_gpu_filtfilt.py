"""Zero-phase forward-backward filtering (sos_filtfilt) against the oracle's
definition, y = R H R H x, on ragged packed channels, and its response to a
centred impulse (symmetric, no phase shift)."""
import numpy as np
import pytest
import torch

import oracle
from synth import workloads
from test_gpu_forward import _lib, random_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tuning", [None, (16, 8, 1, 0), (32, 8, 1, 4), (32, 8, 1, 2)])
def test_filtfilt_matches_oracle(tuning):
    P = _lib()
    lengths = [1, 700, 8192, 100_001, 0, 33_333, 400_000]
    x, sos, K, L, zi = random_case(131, lengths, 6, rmax=0.97)
    K[2] = 0
    y = P.sosfiltfilt(x.cuda(), sos.cuda(), K=K.cuda(), lengths=L, tuning=tuning)
    ref = oracle.sosfiltfilt(x.double().numpy(), sos.numpy(), K=K.numpy(), lengths=L.numpy())
    err = oracle.rel_l2_per_channel(y.cpu().numpy(), ref, L.numpy())
    assert err.max() <= 1e-5, (err.max(), int(err.argmax()))


def test_filtfilt_impulse_is_symmetric():
    P = _lib()
    wl = workloads.plain_bandpass16(n=1 << 16)
    x = torch.zeros(1 << 16, device="cuda")
    c = 1 << 15
    x[c] = 1.0
    y = P.sosfiltfilt(x, wl.sos.cuda()).double().cpu().numpy()
    peak = np.abs(y).max()
    assert int(np.abs(y).argmax()) == c
    d = np.abs(y[c - 20000:c][::-1] - y[c + 1:c + 20001]).max()
    assert d <= 1e-5 * peak
