"""Sections ill-conditioned for FP32: pole pairs close to z = 1 or z = -1
near the unit circle, whose transition powers A^(N l) have entries up to about
min(l N, 1 / sin(theta)).  The plan flags them (Coef32::misc.w, reported per
channel by sos_plan_extended) and the warp-segment kernel runs their lane scan
and fold in double-float with the low parts of a1, a2 in the in-lane runs.

Checks: the flag against an FP64 recomputation of its criterion (largest
entry of Phi^(2^j), j < 5, and Phi^l, l < 32, above 8, Phi = A^N), and the
precision-stress filters (K = 8, radius 0.999..0.9999, angles U[0, pi])
against the FP64 oracle, per channel within max(1e-3, 8 x the error of the
same cascade run sample by sample in FP32): some of these channels are beyond
1e-3 for FP32 arithmetic of any order."""
import numpy as np
import pytest
import scipy.signal
import torch

import oracle
from synth import workloads
from test_gpu_forward import _lib

pytestmark = pytest.mark.gpu

ENTRY = 8.0       # the plan's threshold on the powers' largest entry
SENS = 1e-4       # and on the poles' displacement by FP32 rounding of a1, a2
FP32_FACTOR = 8.0


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


@pytest.mark.parametrize("N", [16, 32])
def test_extended_flag_matches_criterion(N):
    P = _lib()
    wl = workloads.precision_stress(length=1 << 14, device="cuda")
    plan = P.SosFilter(wl.lengths, 8, tuning=(N, 8, 1, 0))
    plan.prepare(wl.sos, wl.K)
    ext = plan.plan_extended().numpy()
    sos = wl.sos.cpu().numpy()
    checked = 0
    for c in range(wl.n_channels):
        ms = [max_power_entry(r[4] / r[3], r[5] / r[3], N) for r in sos[c]]
        ss = [coef_sensitivity(r[4] / r[3], r[5] / r[3]) for r in sos[c]]
        if any(abs(m - ENTRY) < 1e-3 for m in ms) or any(abs(v / SENS - 1) < 0.01 for v in ss):
            continue  # too close to a threshold to call
        assert ext[c] == int(any(m > ENTRY or v > SENS for m, v in zip(ms, ss))), (c, ms, ss)
        checked += 1
    assert checked >= 40 and 0 < ext.sum() < wl.n_channels
    # well-conditioned filters: none
    bp = workloads.plain_bandpass16(n=1 << 16, device="cuda")
    plan = P.SosFilter(bp.lengths, 8)
    plan.prepare(bp.sos, bp.K)
    assert plan.plan_extended().sum() == 0


@pytest.mark.parametrize("tuning", [None, (16, 8, 1, 0), (32, 8, 1, 0), (32, 8, 1, 2 << 8), "auto"])
def test_precision_stress_within_fp32_bound(tuning):
    P = _lib()
    L = 1 << 16
    wl = workloads.precision_stress(length=L, device="cuda")
    y, _ = P.sosfilt(wl.x, wl.sos, wl.K, lengths=wl.lengths, tuning=tuning, check=True)
    y = y.cpu().double().numpy()
    x = wl.x.cpu().numpy()
    sos = wl.sos.cpu().numpy()
    worst, bad = 0.0, []
    for c in range(wl.n_channels):
        xc = x[c * L:(c + 1) * L]
        ref, _ = oracle.sosfilt(xc.astype(np.float64), sos[c])
        nref = np.linalg.norm(ref)
        err = np.linalg.norm(y[c * L:(c + 1) * L] - ref) / nref
        y32 = scipy.signal.sosfilt(sos[c].astype(np.float32), xc.astype(np.float32))
        e32 = np.linalg.norm(y32.astype(np.float64) - ref) / nref
        bound = max(1e-3, FP32_FACTOR * e32)
        if not (np.isfinite(err) and err <= bound):
            bad.append((c, float(err), float(e32)))
        worst = max(worst, err / bound)
    assert not bad, bad
    assert worst > 0.0


@pytest.mark.parametrize("wn", [0.002, 0.005])
def test_low_cutoff_linkwitz_riley_on_the_look_back(wn):
    """Two identical 2nd-order Butterworth low-pass sections (a 4th-order
    Linkwitz-Riley crossover) at a low cutoff: coincident poles, so no memory
    horizon (the look-back carries the state, in FP32 scans), and poles close
    to z = 1 (ill-conditioned: flagged).  The look-back's composition keeps
    the error well inside 1e-3 here."""
    from synth import filters, rng
    P = _lib()
    s1 = filters.butter_lowpass2_closed_form(wn)
    sos = np.concatenate([s1, s1])
    n = 1 << 20
    x = rng.normal(7, rng.STREAM_SIGNAL, n, device="cuda").float()
    plan = P.SosFilter([n], 2)
    y, _ = plan(x, torch.from_numpy(sos)[None].cuda(), torch.tensor([2], dtype=torch.int32).cuda(),
                None)
    assert plan.device_status() == 0
    hz, _ = plan.plan_info()
    assert int(hz[0]) == -1 and int(plan.plan_extended()[0]) == 1
    ref, _ = oracle.sosfilt(x.double().cpu().numpy(), sos)
    err = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-3, err
