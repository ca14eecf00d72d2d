"""The seeded input generators: SplitMix64 against a pure-Python restatement,
normal moments, and the filter designs against scipy's designs and their
stated properties."""
import math

import numpy as np
import pytest
import torch

from synth import filters, rng, workloads


def test_splitmix_matches_python():
    r = rng.raw_u64(12345, 3, 10, 64)
    for i, v in enumerate(r.tolist()):
        assert (v & ((1 << 64) - 1)) == rng.raw_u64_py(12345, 3, 10 + i)


def test_splitmix_reference_vector():
    # SplitMix64 seeded with 0: the first outputs of the published generator
    # (state += 0x9E3779B97F4A7C15, then the output mix) are
    # 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F.
    out = []
    state = 0
    for _ in range(3):
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        out.append(rng.mix_py(state))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normal_moments():
    z = rng.normal(1, rng.STREAM_SIGNAL, 1 << 20).double()
    assert abs(z.mean().item()) < 5e-3
    assert abs(z.var().item() - 1.0) < 5e-3
    # chunked generation equals one-shot generation
    z2 = torch.cat([rng.normal(1, rng.STREAM_SIGNAL, 1000, start=0),
                    rng.normal(1, rng.STREAM_SIGNAL, 1000, start=1000)])
    assert torch.equal(z2, rng.normal(1, rng.STREAM_SIGNAL, 2000))


def test_butter_designs_match_scipy():
    ss = pytest.importorskip("scipy.signal")
    w = np.linspace(0.001, math.pi - 0.001, 777)
    lp = filters.butter_lowpass2_closed_form(0.1)
    assert np.allclose(lp, ss.butter(2, 0.1, output="sos"), rtol=1e-12, atol=1e-15)
    bp = filters.butter_bandpass(8, 0.1, 0.2)
    ref = ss.butter(8, [0.1, 0.2], btype="bandpass", output="sos")
    assert np.max(np.abs(filters.freqz_sos(bp, w) - filters.freqz_sos(ref, w))) < 1e-10
    # one conjugate pair per section, zeros at +1 and -1, radius increasing
    assert np.allclose(bp[:, 1], 0.0) and np.allclose(bp[:, 0], -bp[:, 2])
    assert np.all(np.diff(bp[:, 5]) > 0)


def test_random_sections_properties():
    sos = filters.random_sections(3, 64, 0.5, 0.995)
    r = np.sqrt(sos[:, 5])
    assert np.all((r >= 0.5) & (r <= 0.995))
    w = np.linspace(0, math.pi, 1 << 18)
    for row in sos[:16]:
        peak = np.max(np.abs(filters.freqz_sos(row[None], w)))
        assert abs(peak - 1.0) < 1e-6
        # zeros on the unit circle: b0 == b2
        assert row[0] == pytest.approx(row[2])


def test_batched_workload_shape():
    wl = workloads.batched(n_channels=16, min_len=8, max_len=100, seed=3)
    assert wl.x.numel() == int(wl.lengths.sum())
    assert wl.sos.shape == (16, 8, 6) and wl.zi.shape == (16, 8, 2)
    assert int(wl.K.min()) >= 1 and int(wl.K.max()) <= 8
    assert int(wl.lengths.min()) >= 8 and int(wl.lengths.max()) <= 100
