"""Filter designs used as synthetic inputs (FP64, numpy).

These produce second-order-section coefficient rows (b0, b1, b2, a0, a1, a2);
they do not filter anything.

* Butterworth low-pass / band-pass by the bilinear transform with
  pre-warping (Nyquist = 1 convention: a normalised cutoff w maps to the
  analog frequency tan(pi * w / 2)).  The band-pass keeps one conjugate pole
  pair per section with one zero at z = +1 and one at z = -1, sections in
  order of increasing pole radius, and the overall gain (unit magnitude at
  the geometric band centre) spread evenly over the sections.
* Random stable sections: a conjugate pole pair at radius r and angle theta,
  a conjugate zero pair on the unit circle at angle phi
  (b proportional to [1, -2 cos(phi), 1]), scaled so that the section's
  peak magnitude response is 1.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng


def butter_lowpass2_closed_form(wn: float) -> np.ndarray:
    """Second-order Butterworth low-pass, textbook closed form.
    With W = tan(pi*wn/2), D = 1 + sqrt(2) W + W^2:
    b = W^2/D [1, 2, 1], a = [1, 2(W^2 - 1)/D, (1 - sqrt(2) W + W^2)/D]."""
    W = math.tan(math.pi * wn / 2.0)
    D = 1.0 + math.sqrt(2.0) * W + W * W
    g = W * W / D
    return np.array([[g, 2 * g, g, 1.0, 2.0 * (W * W - 1.0) / D,
                      (1.0 - math.sqrt(2.0) * W + W * W) / D]])


def _prototype_poles(order: int) -> np.ndarray:
    k = np.arange(order)
    return np.exp(1j * math.pi * (2 * k + order + 1) / (2 * order))


def _bilinear(s: np.ndarray) -> np.ndarray:
    return (1.0 + s) / (1.0 - s)


def _pairs_to_sos(zpoles: np.ndarray, zero_pair, gain: float) -> np.ndarray:
    """zpoles: one representative (Im >= 0) of each conjugate pair."""
    rows = []
    for p in sorted(zpoles, key=lambda p: abs(p)):
        rows.append([1.0, 0.0, 0.0, 1.0, -2.0 * p.real, abs(p) ** 2])
    sos = np.array(rows)
    sos[:, 0:3] = np.array(zero_pair, dtype=np.float64)
    K = len(rows)
    sos[:, 0:3] *= gain ** (1.0 / K)
    return sos


def freqz_sos(sos: np.ndarray, w: np.ndarray) -> np.ndarray:
    """H(e^{jw}) of a cascade, FP64 complex."""
    zinv = np.exp(-1j * np.asarray(w, dtype=np.float64))
    h = np.ones_like(zinv)
    for b0, b1, b2, a0, a1, a2 in np.asarray(sos, dtype=np.float64).reshape(-1, 6):
        h = h * (b0 + b1 * zinv + b2 * zinv ** 2) / (a0 + a1 * zinv + a2 * zinv ** 2)
    return h


def butter_bandpass(order: int, w1: float, w2: float) -> np.ndarray:
    """Band-pass Butterworth from an order-``order`` prototype: 2*order poles,
    ``order`` second-order sections."""
    O1 = math.tan(math.pi * w1 / 2.0)
    O2 = math.tan(math.pi * w2 / 2.0)
    O0 = math.sqrt(O1 * O2)
    B = O2 - O1
    spoles = []
    for p in _prototype_poles(order):
        pb = p * B
        disc = np.sqrt(pb * pb - 4.0 * O0 * O0 + 0j)
        spoles += [(pb + disc) / 2.0, (pb - disc) / 2.0]
    zp = _bilinear(np.array(spoles))
    reps = [p for p in zp if p.imag > 0]
    assert len(reps) == order, "band-pass poles must come in conjugate pairs"
    sos = _pairs_to_sos(reps, [1.0, 0.0, -1.0], 1.0)
    wc = 2.0 * math.atan(O0)
    h = freqz_sos(sos, np.array([wc]))[0]
    sos[:, 0:3] *= (1.0 / abs(h)) ** (1.0 / order)
    return sos


def peak_gain(b: np.ndarray, a: np.ndarray, grid: int = 65536) -> np.ndarray:
    """max over w in [0, pi] of |B(e^jw)/A(e^jw)| for each row of b, a
    ([S, 3] each): dense grid, then a golden-section refinement between the
    neighbours of the best grid point."""
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    w = np.linspace(0.0, math.pi, grid + 1)
    c1 = np.cos(w)[None, :]
    c2 = np.cos(2.0 * w)[None, :]

    def sq_coeffs(p):
        # |p0 + p1 z^-1 + p2 z^-2|^2 on the unit circle
        #   = (p0^2 + p1^2 + p2^2) + 2(p0 p1 + p1 p2) cos w + 2 p0 p2 cos 2w
        return (p[:, 0] ** 2 + p[:, 1] ** 2 + p[:, 2] ** 2,
                2.0 * (p[:, 0] * p[:, 1] + p[:, 1] * p[:, 2]),
                2.0 * p[:, 0] * p[:, 2])

    out = np.empty(b.shape[0])
    g = (math.sqrt(5.0) - 1.0) / 2.0
    for s0 in range(0, b.shape[0], 256):
        B0, B1, B2 = sq_coeffs(b[s0:s0 + 256])
        A0, A1, A2 = sq_coeffs(a[s0:s0 + 256])

        def mag2(x):
            cx, c2x = np.cos(x), np.cos(2.0 * x)
            return (B0 + B1 * cx + B2 * c2x) / (A0 + A1 * cx + A2 * c2x)

        m2 = ((B0[:, None] + B1[:, None] * c1 + B2[:, None] * c2)
              / (A0[:, None] + A1[:, None] * c1 + A2[:, None] * c2))
        i = np.argmax(m2, axis=1)
        best = m2[np.arange(len(i)), i]
        lo = w[np.maximum(i - 1, 0)]
        hi = w[np.minimum(i + 1, grid)]
        for _ in range(60):
            c = hi - g * (hi - lo)
            d = lo + g * (hi - lo)
            left = mag2(c) > mag2(d)
            hi = np.where(left, d, hi)
            lo = np.where(left, lo, c)
        out[s0:s0 + 256] = np.sqrt(np.maximum(best, mag2(0.5 * (lo + hi))))
    return out


def random_sections(seed: int, n: int, rmin: float, rmax: float, start: int = 0) -> np.ndarray:
    """n random stable sections, [n, 6].  Draws (per section, 3 uniforms):
    radius r ~ U[rmin, rmax], pole angle theta ~ U[0, pi], zero angle phi ~ U[0, pi]."""
    u = rng.uniform(seed, rng.STREAM_FILTER, 3 * n, start=3 * start).numpy().reshape(n, 3)
    r = rmin + (rmax - rmin) * u[:, 0]
    th = math.pi * u[:, 1]
    ph = math.pi * u[:, 2]
    b = np.stack([np.ones(n), -2.0 * np.cos(ph), np.ones(n)], axis=1)
    a = np.stack([np.ones(n), -2.0 * r * np.cos(th), r * r], axis=1)
    b = b / peak_gain(b, a)[:, None]
    return np.concatenate([b, a], axis=1)
