"""The plan's partial-fraction-free memory bound, checked as mathematics on
the CPU: for cascades of K sections (repeated poles included) with largest
pole radius r, every sample of the FP64 impulse response (the oracle's)
satisfies |h[n]| <= A C(n + 2K - 1, 2K - 1) r^n, A = prod_k B_k r^-2,
B_k = |b0| + |b1| + |b2|; and past the terms' peak the tail sum from P on
is at most the term at P over one minus its ratio to the next.  A missing
r^-2 fails on the delayed responses over small poles, 2K - 2 instead of
2K - 1 on the slow-building responses of repeated poles."""
import math

import numpy as np
import pytest

import oracle
from synth import filters


def _bound_terms(rows, n):
    K = len(rows)
    r = 0.0
    logA = 0.0
    for b0, b1, b2, a1, a2 in rows:
        disc = a1 * a1 - 4.0 * a2
        rk = math.sqrt(a2) if disc < 0 else max(abs(0.5 * (-a1 + math.sqrt(disc))),
                                                abs(0.5 * (-a1 - math.sqrt(disc))))
        r = max(r, rk)
        logA += math.log(abs(b0) + abs(b1) + abs(b2))
    logA -= 2 * K * math.log(r)
    m = 2 * K
    logt = np.array([logA + math.lgamma(i + m) - math.lgamma(m) - math.lgamma(i + 1)
                     + i * math.log(r) for i in range(n)])
    return r, m, logt


def _cascades():
    out = []
    for seed, (rmin, rmax) in enumerate([(0.5, 0.9), (0.9, 0.97), (0.97, 0.99)]):
        half = filters.random_sections(1200 + seed, 2, rmin, rmax)
        out.append(np.concatenate([half, half]))                     # repeated poles
        out.append(filters.random_sections(1300 + seed, 3, rmin, rmax))  # distinct poles
    s1 = filters.butter_lowpass2_closed_form(0.05)
    out.append(np.concatenate([s1, s1, s1]))                          # triple poles
    # pure two-sample delays over small repeated poles: the response starts
    # at n = 2K, where the r^-2 per section is what keeps the bound above it
    d = np.array([[0.0, 0.0, 1.0, 1.0, -0.6, 0.09]])                # double pole 0.3
    out.append(np.concatenate([d, d]))
    out.append(np.concatenate([d, d, d]))
    return out


@pytest.mark.parametrize("idx", range(9))
def test_fallback_bound_dominates_the_impulse_response(idx):
    sos = _cascades()[idx]
    K = len(sos)
    rows = [(s[0] / s[3], s[1] / s[3], s[2] / s[3], s[4] / s[3], s[5] / s[3]) for s in sos]
    n = 4096
    x = np.zeros(n)
    x[0] = 1.0
    kmax = np.array([K], dtype=np.int32)
    h, _ = oracle.sosfilt(x, sos[None], K=kmax, lengths=np.array([n]))
    r, m, logt = _bound_terms(rows, n)
    with np.errstate(divide="ignore"):
        logh = np.log(np.abs(h))
    # above FP64's subnormal floor (where the recursion's rounding stalls)
    ok = logt > -690.0
    assert np.all(logh[ok] <= logt[ok] + 1e-9), int(np.argmax(logh[ok] - logt[ok]))
    # the geometric tail estimate from any P past the peak covers the true tail
    nstar = int(math.ceil((m * r - 1.0) / (1.0 - r))) + 1
    for P in (nstar, nstar + 50, nstar + 400):
        if P >= n - 1:
            continue
        ratio = r * (P + m) / (P + 1.0)
        assert ratio < 1.0
        tail_bound = math.exp(logt[P]) / (1.0 - ratio)
        assert np.abs(h[P:]).sum() <= tail_bound, (P, np.abs(h[P:]).sum(), tail_bound)
