"""Precision classes of the plan, and the precision-stress workload.

Per section (Coef32::misc.w): level 2 when the largest entry of its
transition powers A^(N 2^j), A^(N l) exceeds 8 (pole pairs close to z = 1 or
z = -1 near the unit circle) or when rounding a1, a2 to FP32 displaces its
poles by more than 1e-4 of their distance to the unit circle (lane scan and
fold in double-float, coefficient low parts in the in-lane runs); level 1
when that displacement exceeds 2^-18 (the low parts alone).  Per channel
(sos_plan_extended): the largest section level, or 3 when the whole cascade
runs with double-float samples because the plan's estimate of the error that
FP32 hand-offs between sections cause exceeds 2^-17.

Checks: the levels against an FP64 recomputation of their criteria, and the
precision-stress filters (K = 8, radius 0.999..0.9999, angles U[0, pi])
against the FP64 oracle at the stated tolerance, relative L2 <= 1e-3 per
channel, on channels long enough for several segments, window by window."""
import numpy as np
import pytest
import torch

import oracle
from synth import workloads
from test_gpu_forward import _lib

pytestmark = pytest.mark.gpu

ENTRY = 8.0       # the plan's threshold on the powers' largest entry
SENS = 1e-4       # and on the poles' displacement by FP32 rounding of a1, a2


def coef_sensitivity(a1: float, a2: float) -> float:
    """First-order displacement of the poles of z^2 + a1 z + a2 when a1, a2
    are rounded to FP32, (r |da1| + |da2|) / |p1 - p2|, over their distance
    1 - r to the unit circle (FP64, from the roots)."""
    p = np.roots([1.0, a1, a2])
    r = np.abs(p).max()
    sep = abs(p[0] - p[1])
    if r >= 1.0 or sep == 0.0:
        return np.inf
    da1 = abs(a1 - float(np.float32(a1)))
    da2 = abs(a2 - float(np.float32(a2)))
    return (r * da1 + da2) / (sep * (1.0 - r))


def max_power_entry(a1: float, a2: float, N: int) -> float:
    A = np.array([[-a1, 1.0], [-a2, 0.0]])
    phi = np.linalg.matrix_power(A, N)
    m = 0.0
    P = np.eye(2)
    for _ in range(32):
        m = max(m, np.abs(P).max())
        P = P @ phi
    for j in range(5):
        m = max(m, np.abs(np.linalg.matrix_power(phi, 1 << j)).max())
    return m


ALO = 2.0 ** -18  # level 1 threshold on the displacement


def section_level(a1: float, a2: float, N: int) -> int:
    m = max_power_entry(a1, a2, N)
    v = coef_sensitivity(a1, a2)
    return 2 if (m > ENTRY or v > SENS) else (1 if v > ALO else 0)


def _near_threshold(a1, a2, N):
    m = max_power_entry(a1, a2, N)
    v = coef_sensitivity(a1, a2)
    return abs(m - ENTRY) < 1e-3 or abs(v / SENS - 1) < 0.01 or abs(v / ALO - 1) < 0.01


@pytest.mark.parametrize("N", [16, 32])
def test_extended_levels_match_criterion(N):
    P = _lib()
    wl = workloads.batched(n_channels=256, min_len=1 << 12, max_len=1 << 14, seed=71,
                           device="cuda")
    plan = P.SosFilter(wl.lengths, 8, tuning=(N, 8, 1, 0))
    plan.prepare(wl.sos, wl.K)
    ext = plan.plan_extended().numpy()
    sos = wl.sos.cpu().numpy()
    K = wl.K.cpu().numpy()
    checked = 0
    for c in range(wl.n_channels):
        rows = [r for r in sos[c, :K[c]]]
        if any(_near_threshold(r[4] / r[3], r[5] / r[3], N) for r in rows):
            continue  # too close to a threshold to call
        lv = max(section_level(r[4] / r[3], r[5] / r[3], N) for r in rows)
        if ext[c] == 3:
            continue  # whole channel in double-float (the hand-off estimate)
        assert ext[c] == lv, (c, ext[c], lv)
        checked += 1
    assert checked >= 150 and (ext == 0).any() and (ext == 1).any() and (ext == 2).any()
    # well-conditioned filters: none
    bp = workloads.plain_bandpass16(n=1 << 16, device="cuda")
    plan = P.SosFilter(bp.lengths, 8)
    plan.prepare(bp.sos, bp.K)
    assert plan.plan_extended().sum() == 0


def _stress_windows(P, L, tuning, nwin=16):
    """Per channel, the worst relative L2 error over nwin equal windows of
    the output (each against the oracle run from the channel's start), and
    the plan's segments per channel."""
    wl = workloads.precision_stress(length=L, device="cuda")
    plan = P.SosFilter(wl.lengths, 8, tuning=tuning)
    y, zf = plan(wl.x, wl.sos, wl.K, None)
    assert plan.device_status() == 0
    _, segs = plan.plan_info()
    ext = plan.plan_extended().numpy()
    y = y.cpu()
    sos = wl.sos.cpu().numpy()
    C = wl.n_channels
    worst = np.zeros(C)
    whole = np.zeros(C)
    zfe = np.zeros(C)
    for c0 in range(0, C, 16):
        c1 = min(C, c0 + 16)
        xs = wl.x[c0 * L:c1 * L].cpu().double().numpy()
        ref, zf_ref = oracle.sosfilt(xs, sos[c0:c1], K=np.full(c1 - c0, 8),
                                     lengths=np.full(c1 - c0, L))
        got = y[c0 * L:c1 * L].double().numpy()
        for c in range(c0, c1):
            r = ref[(c - c0) * L:(c - c0 + 1) * L]
            g = got[(c - c0) * L:(c - c0 + 1) * L]
            whole[c] = np.linalg.norm(g - r) / np.linalg.norm(r)
            w = L // nwin
            worst[c] = max(np.linalg.norm(g[i * w:(i + 1) * w] - r[i * w:(i + 1) * w]) /
                           np.linalg.norm(r[i * w:(i + 1) * w]) for i in range(nwin))
            dz = zf[c].cpu().double().numpy() - zf_ref[c - c0]
            zfe[c] = np.linalg.norm(dz) / max(np.linalg.norm(zf_ref[c - c0]),
                                              np.sqrt(np.mean(r[-w:] ** 2)))
    return worst, whole, zfe, segs.numpy(), ext


@pytest.mark.parametrize("tuning", [None, "auto"])
def test_precision_stress_several_segments_within_1e3(tuning):
    """64 channels of 2^22 samples (each cut into at least 4 segments, with
    horizons of 60K-300K samples), every window of 2^18 samples within the
    stated 1e-3 of the oracle, and the final states too."""
    P = _lib()
    L = 1 << 22
    if tuning == "auto":
        from paper_2607_14054_gb300.autotune import autotune
        wl = workloads.precision_stress(length=L, device="cuda")
        tuning = autotune(wl.x, wl.sos, wl.K, wl.lengths, None)
        del wl
    worst, whole, zfe, segs, ext = _stress_windows(P, L, tuning)
    print("stress 64x2^22: worst window %.3g, whole %.3g, zf %.3g, class-3 channels %d"
          % (worst.max(), whole.max(), zfe.max(), int((ext == 3).sum())))
    assert segs.min() >= 4, segs.min()
    assert worst.max() <= 1e-3, (int(worst.argmax()), float(worst.max()))
    assert zfe.max() <= 1e-3, (int(zfe.argmax()), float(zfe.max()))


def test_precision_stress_short_channels_all_tunings():
    """The same filters on 2^16 samples (one segment per channel) for the
    other tunings the library offers such plans."""
    P = _lib()
    L = 1 << 16
    for tuning in [(16, 8, 1, 0), (32, 8, 1, 0), (32, 8, 1, 2 << 8)]:
        worst, whole, zfe, segs, ext = _stress_windows(P, L, tuning, nwin=4)
        assert whole.max() <= 1e-3 and worst.max() <= 1e-3, (tuning, float(worst.max()))


@pytest.mark.parametrize("wn", [0.002, 0.005])
def test_low_cutoff_linkwitz_riley_on_the_look_back(wn):
    """Two identical 2nd-order Butterworth low-pass sections (a 4th-order
    Linkwitz-Riley crossover) at a low cutoff: coincident poles, so no
    partial-fraction memory horizon; with the look-back forced
    (SOS_FLAG_CARRY_ONLY) the state is carried in FP32 scans, and poles close
    to z = 1 (ill-conditioned: flagged).  The look-back's composition keeps
    the error well inside 1e-3 here; the default plan (the partial-fraction-
    free horizon where the channel is long enough) as well."""
    from synth import filters, rng
    P = _lib()
    s1 = filters.butter_lowpass2_closed_form(wn)
    sos = np.concatenate([s1, s1])
    n = 1 << 20
    x = rng.normal(7, rng.STREAM_SIGNAL, n, device="cuda").float()
    ref, _ = oracle.sosfilt(x.double().cpu().numpy(), sos)
    for tuning in [(0, 0, 0, 2), None]:
        plan = P.SosFilter([n], 2, tuning=tuning)
        y, _ = plan(x, torch.from_numpy(sos)[None].cuda(),
                    torch.tensor([2], dtype=torch.int32).cuda(), None)
        assert plan.device_status() == 0
        hz, _ = plan.plan_info()
        if tuning is not None:
            assert int(hz[0]) == -1 and int(plan.plan_extended()[0]) >= 1
        err = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (tuning, int(hz[0]), err)
