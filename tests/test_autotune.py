"""Host logic of the autotuner (no GPU): cache keys, candidate sets, and the
cache file round trip; on a GPU, the chosen tuning filters correctly."""
import json

import numpy as np
import pytest
import torch

from paper_2607_14054_gb300 import autotune as at


def test_shape_key_buckets():
    assert at.shape_key([1 << 24], 8, False) == (8, 24, 0, "horizon")
    assert at.shape_key([1000, 3000], 4, True) == (4, 11, 1, "carried")
    # the mean length is bucketed by rounded log2
    assert at.shape_key([3 << 10] * 4096, 8, False)[1] == 12


def test_candidates():
    h = at.candidates(False)
    assert {c[0] for c in h} == {16, 32, 64} and {c[2] for c in h} == {1, 2}
    # warp segments at several CTAs per SM and the section pipeline, per N
    assert len(h) == 2 * sum(len(v) for v in at.KERNELS.values())
    assert all(4 in {c[3] for c in h if c[0] == n} and 0 in {c[3] for c in h if c[0] == n}
               for n in (16, 32, 64))
    assert all(c[3] & ~0xF04 == 0 for c in h)
    c = at.candidates(True)
    assert set(c) >= set(h)
    assert all((n, w) in at.SUPPORTED_NW for (n, w, _, _) in c)
    assert len(c) == 2 * sum(len(at.KERNELS[n]) for (n, _) in at.SUPPORTED_NW)
    # ill-conditioned sections: PH on the warp-segment kernel only
    e = at.candidates(False, True)
    assert e and all(n <= 32 and a == 1 and not (f & at.SECTION_PIPELINE) for (n, _, a, f) in e)
    assert set(e) <= set(h)
    assert at.shape_key([1 << 20], 8, False, True) != at.shape_key([1 << 20], 8, False)


def test_cache_file_round_trip(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("SOSFILT_TUNE_CACHE", path)
    at.clear_cache()
    key = at.shape_key([1 << 20], 8, False)
    at.seed_cache([(key, (16, 8, 2, 0))])
    at._save_file(path)
    at.clear_cache()
    assert at.cached(key) is None
    at._load_file(path)
    assert at.cached(key) == (16, 8, 2, 0)
    with open(path) as f:
        assert len(json.load(f)) == 1
    at.clear_cache()


@pytest.mark.gpu
def test_autotuned_call_matches_oracle():
    import paper_2607_14054_gb300 as P
    import oracle
    from synth import workloads
    P.build()
    at.clear_cache()
    wl = workloads.batched(n_channels=24, max_len=1 << 16, device="cuda")
    rep = []
    tu = at.autotune(wl.x, wl.sos, wl.K, wl.lengths, wl.zi, report=rep)
    # (the smallest candidate set: a plan with ill-conditioned sections)
    assert tu in [c for c, _ in rep] and len(rep) >= len(at.candidates(False, True))
    y, zf = P.sosfilt(wl.x, wl.sos, wl.K, wl.lengths, wl.zi, tuning="auto", check=True)
    y_ref, _ = oracle.sosfilt(wl.x.double().cpu().numpy(), wl.sos.cpu().numpy(),
                              K=wl.K.cpu().numpy(), lengths=wl.lengths.numpy(),
                              zi=wl.zi.double().cpu().numpy())
    err = oracle.rel_l2_per_channel(y.cpu().numpy(), y_ref, wl.lengths.numpy())
    assert err.max() <= 1e-5
