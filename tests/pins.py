"""Pins that tie the FP64 oracle to facts other than itself.

Each pin takes an :class:`oracle.Oracle` and raises AssertionError if the
oracle disagrees with what the paper or the mathematics fixes.  They run on
the real oracle (tests/test_oracle_pins.py) and on deliberately broken
copies of it (tests/test_oracle_mutations.py), which must each fail at
least one pin.

Nothing here shares code with the oracle: impulse responses come from the
pole closed form, frequency responses from polynomial evaluation, the matrix
pins from numpy dense solves of the paper's systems, and the state pins from
zero-input / step-input closed forms.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# small independent helpers (no recurrence anywhere)
# ----------------------------------------------------------------------------


def allpole_impulse(a1: float, a2: float, n: int) -> np.ndarray:
    """g[k] for 1/(1 + a1 z^-1 + a2 z^-2) from its poles p, q (roots of
    z^2 + a1 z + a2): g[k] = (p^{k+1} - q^{k+1}) / (p - q), or (k+1) p^k for a
    double pole."""
    disc = a1 * a1 - 4.0 * a2
    k = np.arange(n, dtype=np.float64)
    if abs(disc) < 1e-14:
        p = -a1 / 2.0
        return (k + 1.0) * p ** k
    sq = np.sqrt(complex(disc))
    p = (-a1 + sq) / 2.0
    q = (-a1 - sq) / 2.0
    if disc < 0:
        r = abs(p)
        th = math.atan2(p.imag, p.real)
        return r ** k * np.sin((k + 1.0) * th) / math.sin(th)
    return ((p.real ** (k + 1.0)) - (q.real ** (k + 1.0))) / (p.real - q.real)


def section_impulse(row, n: int) -> np.ndarray:
    b0, b1, b2, a0, a1, a2 = (float(v) for v in row)
    b0, b1, b2, a1, a2 = b0 / a0, b1 / a0, b2 / a0, a1 / a0, a2 / a0
    g = allpole_impulse(a1, a2, n)
    h = b0 * g
    h[1:] += b1 * g[:-1]
    h[2:] += b2 * g[:-2]
    return h


def rational_response(sos, w) -> np.ndarray:
    """prod_k B_k(e^jw)/A_k(e^jw) by np.polyval on z^-1."""
    zi = np.exp(-1j * np.asarray(w))
    h = np.ones_like(zi)
    for row in np.asarray(sos).reshape(-1, 6):
        h *= np.polyval(row[2::-1], zi) / np.polyval(row[5:2:-1], zi)
    return h


def random_stable_sos(rs: np.random.RandomState, K: int, rmax=0.95, b0_one=False) -> np.ndarray:
    sos = np.zeros((K, 6))
    for k in range(K):
        r = rs.uniform(0.3, rmax)
        th = rs.uniform(0.05, math.pi - 0.05)
        a0 = rs.uniform(0.5, 2.0)
        sos[k, 3:] = a0 * np.array([1.0, -2.0 * r * math.cos(th), r * r])
        sos[k, :3] = rs.normal(size=3)
        if b0_one:
            sos[k, :3] /= sos[k, 0] / a0
    return sos


def df2t_state_from_history(row, xm2, xm1, ym2, ym1):
    """z1 = b1 x[-1] + b2 x[-2] - a1 y[-1] - a2 y[-2], z2 = b2 x[-1] - a2 y[-1]
    (normalised coefficients)."""
    b0, b1, b2, a0, a1, a2 = (float(v) for v in row)
    b1, b2, a1, a2 = b1 / a0, b2 / a0, a1 / a0, a2 / a0
    return np.array([b1 * xm1 + b2 * xm2 - a1 * ym1 - a2 * ym2, b2 * xm1 - a2 * ym1])


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------


def pin_single_biquad_impulse(orc):
    """One section: impulse response equals b0 g[n] + b1 g[n-1] + b2 g[n-2]
    with g the closed-form all-pole response (complex, real-distinct and
    repeated poles)."""
    rows = [
        [0.3, -0.2, 0.7, 1.0, -1.2, 0.81],            # complex pair r = 0.9
        [1.0, 0.5, 0.25, 2.0, -1.0, 0.42],            # after a0: real distinct poles
        [0.5, 1.0, -0.3, 1.0, -1.4, 0.49],            # repeated pole 0.7
        [0.02008337, 0.04016673, 0.02008337, 1.0, -1.561018, 0.6413515],
    ]
    n = 400
    for row in rows:
        x = np.zeros(n)
        x[0] = 1.0
        y, _ = orc.sosfilt(x, np.array([row]))
        ref = section_impulse(row, n)
        assert np.max(np.abs(y - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), row


def pin_cascade_is_convolution(orc):
    """Cascade impulse response equals the convolution of the section
    responses (first 600 taps; every pole has |p| <= 0.95 so the truncated
    tails cannot reach the compared window)."""
    rs = np.random.RandomState(11)
    sos = random_stable_sos(rs, 4)
    n = 600
    x = np.zeros(n)
    x[0] = 1.0
    y, _ = orc.sosfilt(x, sos)
    ref = np.zeros(1)
    ref[0] = 1.0
    for row in sos:
        ref = np.convolve(ref, section_impulse(row, n))[:n]
    assert np.max(np.abs(y - ref)) <= 1e-11 * np.max(np.abs(ref))


def pin_frequency_response(orc):
    """DFT of a length-M impulse response equals prod B_k/A_k at w = 2 pi k/M
    (the truncation error is below r^M, here < 1e-30)."""
    rs = np.random.RandomState(12)
    sos = random_stable_sos(rs, 3, rmax=0.9)
    M = 4096
    x = np.zeros(M)
    x[0] = 1.0
    y, _ = orc.sosfilt(x, sos)
    H = np.fft.fft(y)
    w = 2.0 * math.pi * np.arange(M) / M
    ref = rational_response(sos, w)
    assert np.max(np.abs(H - ref)) <= 1e-10 * np.max(np.abs(ref))


def _toeplitz_system(row, T):
    """A, B (T x T) and A_-, B_- (T x 2) of the paper's Eq. filtering_AB and
    Eq. filtering_ABm, normalised coefficients, B with b0 on the diagonal."""
    b0, b1, b2, a0, a1, a2 = (float(v) for v in row)
    b0, b1, b2, a1, a2 = b0 / a0, b1 / a0, b2 / a0, a1 / a0, a2 / a0
    A = np.eye(T) + a1 * np.eye(T, k=-1) + a2 * np.eye(T, k=-2)
    B = b0 * np.eye(T) + b1 * np.eye(T, k=-1) + b2 * np.eye(T, k=-2)
    Am = np.zeros((T, 2))
    Bm = np.zeros((T, 2))
    Am[0] = [a2, a1]
    Bm[0] = [b2, b1]
    if T > 1:
        Am[1] = [0.0, a2]
        Bm[1] = [0.0, b2]
    return A, B, Am, Bm


def pin_dense_toeplitz_solve(orc):
    """Per section, y solves A y = B x + B_- x_{-1} - A_- y_{-1} (paper Sec. III,
    Eq. recursive_equation_block_form) for T <= 64 with a random pre-history;
    the oracle receives that history as the DF2T state.  Chained over a
    3-section cascade with a fresh history per section."""
    rs = np.random.RandomState(13)
    sos = random_stable_sos(rs, 3)
    for T in (1, 2, 3, 17, 64):
        x = rs.normal(size=T)
        hist = rs.normal(size=(3, 4))  # x[-2], x[-1], y[-2], y[-1] per section
        zi = np.stack([df2t_state_from_history(sos[k], *hist[k]) for k in range(3)])
        y, zf = orc.sosfilt(x, sos, zi=zi[None])
        cur = x
        for k in range(3):
            A, B, Am, Bm = _toeplitz_system(sos[k], T)
            rhs = B @ cur + Bm @ hist[k, 0:2] - Am @ hist[k, 2:4]
            out = np.linalg.solve(A, rhs)
            # final state from the extended history
            xe = np.concatenate([hist[k, 0:2], cur])
            ye = np.concatenate([hist[k, 2:4], out])
            zref = df2t_state_from_history(sos[k], xe[-2], xe[-1], ye[-2], ye[-1])
            assert np.max(np.abs(zf[0, k] - zref)) <= 1e-10 * (1 + np.max(np.abs(zref))), (T, k)
            cur = out
        assert np.max(np.abs(y - cur)) <= 1e-10 * (1 + np.max(np.abs(cur))), T


def pin_multiblock_permuted_system(orc):
    """The stride-N permuted block system of paper Sec. V
    (Eq. multi_block_A, Eq. multi_block_Am, Eq. recursive_equation_multi_block_form)
    with blocks x_m = [x[m], x[m+N], ..., x[m+(L-1)N]], solved densely for
    N*L <= 64, equals the oracle for the simplified biquad (b0 = 1,
    Eq. simple_second_order) with a random initial history."""
    rs = np.random.RandomState(14)
    for (N, L) in ((8, 4), (4, 8), (2, 2), (16, 4)):
        T = N * L
        row = random_stable_sos(rs, 1, b0_one=True)[0]
        _, b1, b2, a0, a1, a2 = row
        b1, b2, a1, a2 = b1 / a0, b2 / a0, a1 / a0, a2 / a0
        I = np.eye(L)
        R = np.eye(L, k=-1)
        e0 = np.zeros(L)
        e0[0] = 1.0

        def blockmat(c1, c2):
            M = np.zeros((T, T))
            for m in range(N):
                M[m * L:(m + 1) * L, m * L:(m + 1) * L] = I
                if m >= 1:
                    M[m * L:(m + 1) * L, (m - 1) * L:m * L] = c1 * I
                if m >= 2:
                    M[m * L:(m + 1) * L, (m - 2) * L:(m - 1) * L] = c2 * I
            # upper corner: shift coupling to the last two blocks
            M[0:L, (N - 1) * L:N * L] += c1 * R
            M[0:L, (N - 2) * L:(N - 1) * L] += c2 * R
            M[L:2 * L, (N - 1) * L:N * L] += c2 * R
            return M

        A = blockmat(a1, a2)
        B = blockmat(b1, b2)
        Am = np.zeros((T, 2))
        Bm = np.zeros((T, 2))
        Am[0:L, 0] = a2 * e0
        Am[0:L, 1] = a1 * e0
        Am[L:2 * L, 1] = a2 * e0
        Bm[0:L, 0] = b2 * e0
        Bm[0:L, 1] = b1 * e0
        Bm[L:2 * L, 1] = b2 * e0
        x = rs.normal(size=T)
        hist = rs.normal(size=4)
        perm = np.array([l * N + m for m in range(N) for l in range(L)])  # block m, element l
        xg = x[perm]
        rhs = B @ xg + Bm @ hist[0:2] - Am @ hist[2:4]
        yg = np.linalg.solve(A, rhs)
        y_ref = np.empty(T)
        y_ref[perm] = yg
        zi = df2t_state_from_history(row, *hist)
        y, _ = orc.sosfilt(x, row[None], zi=zi[None, None])
        assert np.max(np.abs(y - y_ref)) <= 1e-10 * (1 + np.max(np.abs(y_ref))), (N, L)


def pin_zero_input_response(orc):
    """x = 0, state (z1, z2): y[n] = z1 g[n] + z2 g[n-1] (closed form), and
    the final state follows the same closed form one step on."""
    row = np.array([0.4, 0.1, -0.3, 1.0, -1.5, 0.8])
    n = 300
    z = np.array([0.7, -1.3])
    y, zf = orc.sosfilt(np.zeros(n), row[None], zi=z[None, None])
    g = allpole_impulse(-1.5, 0.8, n + 2)
    ref = z[0] * g[:n]
    ref[1:] += z[1] * g[:n - 1]
    assert np.max(np.abs(y - ref)) <= 1e-12
    # state after n zero-input samples: z1' = y[n] (the next output), z2' = -a2 y[n-1... ]
    yn = z[0] * g[n] + z[1] * g[n - 1]
    ynm1 = ref[n - 1]
    assert abs(zf[0, 0, 0] - yn) <= 1e-12
    assert abs(zf[0, 0, 1] - (-0.8 * ynm1)) <= 1e-12


def pin_step_steady_state(orc):
    """x = 1 with the steady-state initial state of every section gives the
    constant output prod_k H_k(1), H_k(1) = (b0+b1+b2)/(a0+a1+a2)."""
    rs = np.random.RandomState(15)
    sos = random_stable_sos(rs, 4)
    zi = np.zeros((4, 2))
    u = 1.0
    for k, row in enumerate(sos):
        b0, b1, b2, a0, a1, a2 = row / row[3]
        yk = (b0 + b1 + b2) / (1.0 + a1 + a2) * u
        zi[k] = [(b1 + b2) * u - (a1 + a2) * yk, b2 * u - a2 * yk]
        u = yk
    y, zf = orc.sosfilt(np.ones(257), sos, zi=zi[None])
    assert np.max(np.abs(y - u)) <= 1e-12 * max(1, abs(u))
    assert np.max(np.abs(zf[0] - zi)) <= 1e-12 * (1 + np.max(np.abs(zi)))


def pin_scipy_sosfilt(orc):
    """Agreement with scipy.signal.sosfilt (an independent DF2T implementation),
    outputs and final states, lengths 0..5 and 1000, 5 sections, nonzero zi."""
    import scipy.signal as ss
    rs = np.random.RandomState(16)
    sos = random_stable_sos(rs, 5)
    for T in (0, 1, 2, 3, 5, 1000):
        x = rs.normal(size=T)
        zi = rs.normal(size=(5, 2))
        # scipy normalises by a0 itself only in its design routines; pass normalised rows
        nsos = sos / sos[:, 3:4]
        if T == 0:  # scipy rejects empty input; an empty signal keeps its state
            y_ref, zf_ref = x, zi
        else:
            y_ref, zf_ref = ss.sosfilt(nsos, x, zi=zi)
        y, zf = orc.sosfilt(x, sos, zi=zi[None])
        if T:
            assert np.max(np.abs(y - y_ref)) <= 1e-11 * (1 + np.max(np.abs(y_ref))), T
        assert np.max(np.abs(zf[0] - zf_ref)) <= 1e-11 * (1 + np.max(np.abs(zf_ref))), T


def pin_invariants(orc):
    """Linearity in (x, zi), time invariance, and chunked streaming
    (zf of one chunk as zi of the next) equal to one shot."""
    rs = np.random.RandomState(17)
    sos = random_stable_sos(rs, 3)
    T = 500
    x1, x2 = rs.normal(size=T), rs.normal(size=T)
    z1, z2 = rs.normal(size=(1, 3, 2)), rs.normal(size=(1, 3, 2))
    al, be = 0.7, -1.9
    y1, f1 = orc.sosfilt(x1, sos, zi=z1)
    y2, f2 = orc.sosfilt(x2, sos, zi=z2)
    y3, f3 = orc.sosfilt(al * x1 + be * x2, sos, zi=al * z1 + be * z2)
    assert np.max(np.abs(y3 - (al * y1 + be * y2))) <= 1e-11
    assert np.max(np.abs(f3 - (al * f1 + be * f2))) <= 1e-11
    # time invariance (zero state): delaying the input delays the output
    d = 37
    xd = np.concatenate([np.zeros(d), x1[:T - d]])
    y0, _ = orc.sosfilt(x1, sos)
    yd, _ = orc.sosfilt(xd, sos)
    assert np.max(np.abs(yd[d:] - y0[:T - d])) <= 1e-11 and np.max(np.abs(yd[:d])) == 0.0
    # streaming
    cuts = [0, 1, 3, 64, 65, 300, T]
    zs = z1
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        yp, zs = orc.sosfilt(x1[a:b], sos, zi=zs)
        parts.append(yp)
    assert np.max(np.abs(np.concatenate(parts) - y1)) <= 1e-11
    assert np.max(np.abs(zs - f1)) <= 1e-11


def pin_multichannel(orc):
    """Packed varlen channels with per-channel K equal separate one-channel
    runs; sections beyond K[c] are ignored; a zero-length channel returns
    zf = zi."""
    rs = np.random.RandomState(18)
    lengths = np.array([5, 0, 1, 130, 2])
    K = np.array([2, 3, 1, 3, 0], dtype=np.int32)
    sos = np.stack([random_stable_sos(rs, 3) for _ in lengths])
    zi = rs.normal(size=(len(lengths), 3, 2))
    x = rs.normal(size=int(lengths.sum()))
    y, zf = orc.sosfilt(x, sos, K=K, lengths=lengths, zi=zi)
    o = 0
    for c, n in enumerate(lengths):
        if K[c] > 0:
            yc, zc = orc.sosfilt(x[o:o + n], sos[c, :K[c]], zi=zi[c:c + 1, :K[c]])
            assert np.max(np.abs(y[o:o + n] - yc), initial=0) <= 1e-14
            assert np.max(np.abs(zf[c, :K[c]] - zc[0])) <= 1e-14
        else:
            assert np.array_equal(y[o:o + n], x[o:o + n])
        if n == 0:
            assert np.array_equal(zf[c, :K[c]], zi[c, :K[c]])
        o += n


def _loss(orc, x, sos, zi, wy, wz):
    y, zf = orc.sosfilt(x, sos, zi=zi)
    return float(np.dot(y, wy) + np.sum(zf * wz))


def pin_adjoint(orc):
    """Adjoint: the dot-product test <f(v), w> = <v, f^T(w)> for the part
    linear in (x, zi) (exact up to rounding), and FP64 central finite
    differences for every raw sos entry including a0."""
    rs = np.random.RandomState(19)
    K = 3
    sos = random_stable_sos(rs, K, rmax=0.9)
    for T in (1, 2, 7, 200):
        vx = rs.normal(size=T)
        vz = rs.normal(size=(1, K, 2))
        wy = rs.normal(size=T)
        wz = rs.normal(size=(1, K, 2))
        y, zf = orc.sosfilt(vx, sos, zi=vz)
        lhs = np.dot(y, wy) + np.sum(zf * wz)
        gx, gs, gz = orc.sosfilt_adjoint(vx, sos, wy, zi=vz, g_zf=wz)
        rhs = np.dot(vx, gx) + np.sum(vz * gz)
        assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs)), (T, lhs, rhs)
        # finite differences in every coefficient
        for k in range(K):
            for j in range(6):
                h = 1e-6 * max(1.0, abs(sos[k, j]))
                sp = sos.copy()
                sm = sos.copy()
                sp[k, j] += h
                sm[k, j] -= h
                fd = (_loss(orc, vx, sp, vz, wy, wz) - _loss(orc, vx, sm, vz, wy, wz)) / (2 * h)
                assert abs(fd - gs[0, k, j]) <= 1e-6 * (1 + abs(fd)), (T, k, j, fd, gs[0, k, j])


def pin_filtfilt_autocorrelation_and_zero_phase(orc=None):
    """Zero-phase filtering (oracle.sosfiltfilt, y = R H R H x): of a unit
    impulse at sample c of a zero signal it gives the autocorrelation of the
    cascade's impulse response, y[c + n] = sum_k h[k] h[k + |n|] (symmetric
    about c), with h the convolution of the closed-form section responses;
    and a cosine far from the ends comes out scaled by |H(e^jw)|^2 with no
    phase shift (H evaluated from the coefficients)."""
    import oracle
    rs = np.random.RandomState(17)
    sos = random_stable_sos(rs, 3, rmax=0.8)
    n = 4096
    h = section_impulse(sos[0], n)
    for row in sos[1:]:
        h = np.convolve(h, section_impulse(row, n))[:n]
    c = 2000
    x = np.zeros(n)
    x[c] = 1.0
    y = oracle.sosfiltfilt(x, sos)
    acf = np.array([np.dot(h[:n - m], h[m:]) for m in range(600)])
    for m in range(600):
        assert abs(y[c + m] - acf[m]) <= 1e-12 * acf[0]
        assert abs(y[c - m] - acf[m]) <= 1e-12 * acf[0]
    w = 0.3
    t = np.arange(20000, dtype=np.float64)
    yc = oracle.sosfiltfilt(np.cos(w * t), sos)
    g = abs(rational_response(sos, np.array([w]))[0]) ** 2
    mid = slice(8000, 12000)
    assert np.max(np.abs(yc[mid] - g * np.cos(w * t[mid]))) <= 1e-9 * max(g, 1.0)


ALL_PINS = [
    pin_filtfilt_autocorrelation_and_zero_phase,
    pin_single_biquad_impulse,
    pin_cascade_is_convolution,
    pin_frequency_response,
    pin_dense_toeplitz_solve,
    pin_multiblock_permuted_system,
    pin_zero_input_response,
    pin_step_steady_state,
    pin_scipy_sosfilt,
    pin_invariants,
    pin_multichannel,
    pin_adjoint,
]
