// Plan kernel: per-call set-up of the workspace, entirely on the device so
// that a call never synchronises and can be captured into a CUDA graph.
//
//  * block C (the last one): channel offsets and look-back slots (exclusive
//    scans of the lengths and of ceil(len / T)) and the status word;
//  * block c < C: the coefficient tables of channel c, one warp per section,
//    and two more warps for the b0 factoring and the channel's memory
//    horizon and tile count;
//  * the last block to finish (order_pass): the dispatch prefix over the
//    tile counts and, when some channel carries its state by look-back, the
//    interleaved order.
//
// Coefficient tables (paper Sec. VI-B, "pre-computed before filtering"):
// the rows are normalised by a0; when every b0 of the channel is nonzero the
// common factor prod_k b0_k is split off (Sec. II, Eq. simple_second_order)
// and section k's state is carried scaled by 1/G_k, G_k = b0_1 ... b0_k.
// The DF2T transition A = [[-a1, 1], [-a2, 0]] is raised to the lane step
// Phi = A^N, the warp step Psi = A^(NL) and the tile step Theta = A^T by
// repeated squaring, then the per-lane tables Phi^l, Psi^w and Theta^d by
// binary powering, each lane forming its own entry (Psi and Theta only for
// channels whose state is carried by the look-back).  All of it runs in
// double-float arithmetic (about 48 significand bits) on the FP32 pipe:
// GB300's FP64 FMA is 1/64 of its FP32 rate with a 64-cycle latency.  The
// per-sample tables are rounded once to FP32; the Theta^d used by the
// cross-tile look-back stay double-float.
#include <cfloat>
#include <cmath>

#include "sos_common.cuh"

namespace sosf {

__device__ __forceinline__ df df_of_double(double v) {
    const float hi = (float)v;
    return df{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ float4 to_f4(const dfm2& m) {
    return make_float4(df_to_float(m.a), df_to_float(m.b), df_to_float(m.c), df_to_float(m.d));
}

// what to_f4 dropped: x - to_f4(x) per entry, the low word of the stored
// double-float power
__device__ __forceinline__ float df_rest(df x) {
    const float h = df_to_float(x);
    return (x.hi - h) + x.lo;
}

__device__ __forceinline__ float4 to_f4_lo(const dfm2& m) {
    return make_float4(df_rest(m.a), df_rest(m.b), df_rest(m.c), df_rest(m.d));
}

__device__ __forceinline__ float max_entry(const dfm2& m) {
    return fmaxf(fmaxf(fabsf(m.a.hi), fabsf(m.b.hi)), fmaxf(fabsf(m.c.hi), fabsf(m.d.hi)));
}

// How far rounding a1, a2 to FP32 moves the poles of z^2 + a1 z + a2,
// relative to their distance from the unit circle: |dp| <= (r |da1| + |da2|)
// / |p1 - p2| (first order, from p^2 + a1 p + a2 = 0), over 1 - r.
// Infinite for a double pole or one on or outside the circle.  The rounding
// errors, the discriminant and 1 - a2 are formed in FP64 (they cancel), the
// rest in FP32 (a threshold test; FP64 division and square roots are slow on
// this part).
__device__ __forceinline__ float coef_sensitivity(double a1, double a2) {
    const float da1 = fabsf((float)(a1 - (double)(float)a1));
    const float da2 = fabsf((float)(a2 - (double)(float)a2));
    const float disc = (float)fma(a1, a1, -4.0 * a2);
    float r, sep, gap;
    if (disc < 0.f) {
        sep = sqrtf(-disc);
        r = sqrtf((float)a2);
        gap = (float)(1.0 - a2) / (1.f + r);  // 1 - r
    } else {
        sep = sqrtf(disc);
        r = 0.5f * (fabsf((float)a1) + sep);
        gap = 1.f - r;
    }
    if (!(sep > 0.f) || !(gap > 0.f)) return INFINITY;
    return (r * da1 + da2) / (sep * gap);
}

// Condition number of one normalised section, kappa = ||g|| ||b|| / ||h||:
// g the impulse response of 1 / (1 + a1 z^-1 + a2 z^-2), h that of the whole
// section, b = (b0, b1, b2).  Closed forms from the autocorrelation of the
// all-pole part: c0 = ||g||^2 = (1 + a2) / ((1 - a2) ((1 + a2)^2 - a1^2)),
// c1 = -a1 c0 / (1 + a2), c2 = -a1 c1 - a2 c0, and ||h||^2 = (b0^2 + b1^2 +
// b2^2) c0 + 2 (b0 b1 + b1 b2) c1 + 2 b0 b2 c2.  Infinite for a pole on or
// outside the unit circle or a vanishing response.  FP64, one lane.
__device__ __forceinline__ double section_kappa(double b0, double b1, double b2, double a1,
                                                double a2) {
    const double d = (1.0 - a2) * ((1.0 + a2) * (1.0 + a2) - a1 * a1);
    if (!(d > 0.0) || !(1.0 + a2 > 0.0)) return INFINITY;
    const double c0 = (1.0 + a2) / d;
    const double c1 = -a1 * c0 / (1.0 + a2);
    const double c2 = -a1 * c1 - a2 * c0;
    const double bb = b0 * b0 + b1 * b1 + b2 * b2;
    const double hh = bb * c0 + 2.0 * (b0 * b1 + b1 * b2) * c1 + 2.0 * b0 * b2 * c2;
    if (!(bb > 0.0)) return 0.0;  // no numerator: nothing to amplify
    if (!(hh > 0.0)) return INFINITY;
    return sqrt(c0 * bb / hh);
}

__device__ __forceinline__ bool finite_row(const double* r) {
    for (int i = 0; i < 6; ++i)
        if (!isfinite(r[i])) return false;
    return true;
}

constexpr int kPlanWarps = kMaxSections + 3;  // one per section, two horizon warps, one
                                              // for the precision estimate
constexpr int kPlanThreads = kPlanWarps * 32;

// complex FP32 helpers for the horizon bound
struct cpx {
    float re, im;
};
__device__ __forceinline__ cpx cmul(cpx a, cpx b) {
    return cpx{fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cpx cdiv(cpx a, cpx b) {
    const float d = fmaf(b.re, b.re, b.im * b.im);
    return cpx{fmaf(a.re, b.re, a.im * b.im) / d, fmaf(a.im, b.re, -a.re * b.im) / d};
}
__device__ __forceinline__ float cabs_(cpx a) { return hypotf(a.re, a.im); }

// Memory horizon of one channel, in two parts run by two warps at once
// (rows[k] = normalised b0, b1, b2, a1, a2 of section k).  The cascade's
// impulse response is, past its first 2K samples, h[n] = sum_i R_i p_i^n over
// the nonzero poles p_i (partial fractions of prod_k B_k(z) / A_k(z), distinct
// poles), so its absolute tail from n on is at most sum_i |R_i| |p_i|^n /
// (1 - |p_i|).  A segment that starts P samples early from zero state drops
// exactly such a tail of the input's convolution; P is the smallest multiple
// of 16 (and >= 2K) for which each pole's share is below kHorizonEps *
// ||h||_2 / (2K), with ||h||_2 bounded from below by half the norm of the
// first 32 samples (horizon_norm, filtered in FP32) or, where it is larger
// and its sum does not cancel, by half the closed-form norm of the response
// past sample 0 from the residues (horizon_poles).  The initial state's
// response (DF2T state (k, j) responds with z^-j / A_k(z) * prod_{m > k}
// B_m / A_m) must likewise have decayed below the bound at the end of the
// first segment.  The horizon is -1 when no such P <= T / 2 exists, when a
// pole lies on or outside |z| = 1 - 1e-7, or when two poles are closer than
// 1e-4 (relative), where the partial fractions are not reliable.

// The horizon is scale-free in the numerators: every section's (b0, b1, b2)
// enters divided by m_k = max |b_j| (cascades of unit-peak sections near the
// unit circle have gains far below FP32's range), the input response then
// scaling by 1 / prod m_k.  The initial state's response, which does not
// pass through the sections before its own, is compared in the log domain
// with those factors put back.
__device__ __forceinline__ float num_scale(const float* row) {
    const float m = fmaxf(fabsf(row[0]), fmaxf(fabsf(row[1]), fabsf(row[2])));
    return m > 0.f ? m : 1.f;
}

// ||h||_2 lower bound: half the norm of the first 32 samples of the impulse
// response, by a systolic pipeline over the lanes (lane k < K runs section k
// on sample t - k at step t, taking its input from lane k - 1's previous
// output).  One warp.
__device__ float horizon_norm(const float (*rowsf)[5], int K, int lane) {
    float e2 = 0.f;
    const bool on = lane < K;
    const float im = on ? 1.f / num_scale(rowsf[lane]) : 1.f;
    const float cb0 = on ? rowsf[lane][0] * im : 1.f, cb1 = on ? rowsf[lane][1] * im : 0.f,
                cb2 = on ? rowsf[lane][2] * im : 0.f, ca1 = on ? rowsf[lane][3] : 0.f,
                ca2 = on ? rowsf[lane][4] : 0.f;
    float z1 = 0.f, z2 = 0.f, y = 0.f;
    for (int t = 0; t < 32 + K - 1; ++t) {
        float u = __shfl_up_sync(0xffffffffu, y, 1);
        if (lane == 0) u = t == 0 ? 1.f : 0.f;
        const int n = t - lane;
        if (on && n >= 0 && n < 32) {
            y = fmaf(cb0, u, z1);
            z1 = fmaf(cb1, u, fmaf(-ca1, y, z2));
            z2 = fmaf(cb2, u, -ca2 * y);
            if (lane == K - 1) e2 = fmaf(y, y, e2);
        }
    }
    e2 = K > 0 ? __shfl_sync(0xffffffffu, e2, K - 1) : 1.f;  // K = 0: identity
    return 0.5f * sqrtf(e2);
}

// Per-pole terms of the bound that do not depend on ||h||_2 or on the
// segment length (one warp, lane i < 2K takes pole i): la = log(kHorizonEps
// (1 - r) / (2K |R_i|)) and ilr = 1 / log r, so that pole i needs P >= (la +
// log ||h||_2) ilr; zs = the log of the initial-state response's bound
// (relative to the normalised input response), which decays as r^T over a
// first segment of T samples (lr = log r).  Returns false (for every lane)
// where the partial fractions are unusable.
__device__ bool horizon_poles(const double (*rows)[5], const float (*rowsf)[5], int K, int lane,
                              cpx* s_pole, cpx* s_res, float& la, float& ilr, float& zs, float& lr,
                              float& etail) {
    const int np = 2 * K;
    // poles: lane i < 2K takes root (i & 1) of z^2 + a1 z + a2 of section i / 2
    if (lane < np) {
        const double a1 = rows[lane >> 1][3], a2 = rows[lane >> 1][4];
        const double disc = a1 * a1 - 4.0 * a2;
        cpx z;
        if (disc < 0.0) {
            const float im = 0.5f * sqrtf((float)(-disc));
            z = cpx{(float)(-0.5 * a1), (lane & 1) ? -im : im};
        } else {
            const double sq = sqrt(disc);
            z = cpx{(float)(0.5 * ((lane & 1) ? -a1 - sq : -a1 + sq)), 0.f};
        }
        s_pole[lane] = z;
    }
    __syncwarp();
    bool bad = false;
    la = 0.f;
    ilr = 0.f;
    zs = 0.f;
    lr = 0.f;
    cpx res{0.f, 0.f};
    if (lane < np) {
        const cpx pi = s_pole[lane];
        const float r2 = fmaf(pi.re, pi.re, pi.im * pi.im);
        const float r = sqrtf(r2);
        if (r > 1e-20f) {
            if (!(r < 1.f - 1e-7f)) bad = true;
            const float ir2 = 1.f / r2;
            const cpx inv{pi.re * ir2, -pi.im * ir2};
            const cpx inv2 = cmul(inv, inv);
            // walk the sections from the last to the first: den = prod over
            // the poles of sections >= k (except p_i) of (1 - p_l / p_i),
            // num = prod_{m > k} B_m(p_i), B_m(z) = b0 + b1 z^-1 + b2 z^-2
            cpx num{1.f, 0.f}, den{1.f, 0.f};
            // log of the largest state response (unit state, true scale)
            // relative to the normalised input response
            float lz2 = -INFINITY;
            float lcum[kMaxSections];  // sum_{m <= k} log m_m
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < kMaxSections; ++k) {
                if (k < K) acc += __logf(num_scale(rowsf[k]));
                lcum[k] = acc;
            }
            const int own = lane >> 1;
            for (int k = K - 1; k >= 0; --k) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int l = 2 * k + q;
                    if (l != lane) {
                        const cpx f = cmul(s_pole[l], inv);
                        const cpx g = cpx{1.f - f.re, -f.im};
                        if (fmaf(g.re, g.re, g.im * g.im) < 1e-8f) bad = true;
                        den = cmul(den, g);
                    }
                }
                if (k <= own) {
                    // states (k, 0) and (k, 1): |residue|^2 = |num|^2 / |den|^2
                    // (times |1 / p_i|^2 for j = 1), back to true scale
                    float lk = 0.f;
#pragma unroll
                    for (int q = 0; q < kMaxSections; ++q)
                        if (q == k) lk = lcum[q];
                    const float a = __logf(fmaf(num.re, num.re, num.im * num.im)) -
                                    __logf(fmaf(den.re, den.re, den.im * den.im)) +
                                    __logf(fmaxf(1.f, ir2)) - 2.f * lk;
                    lz2 = fmaxf(lz2, a);
                }
                const float ims = 1.f / num_scale(rowsf[k]);
                const float b0 = rowsf[k][0] * ims, b1 = rowsf[k][1] * ims, b2 = rowsf[k][2] * ims;
                const cpx Bk{fmaf(b2, inv2.re, fmaf(b1, inv.re, b0)), fmaf(b2, inv2.im, b1 * inv.im)};
                num = cmul(num, Bk);
            }
            // full cascade: num = prod_m B_m(p_i), den over all other poles;
            // the residue R_i = num / den of h[n] = sum_i R_i p_i^n (n >= 1)
            res = cdiv(num, den);
            const float R = sqrtf(fmaf(num.re, num.re, num.im * num.im) /
                                  fmaf(den.re, den.re, den.im * den.im));
            lr = __logf(r);
            if (R > 0.f) {
                la = __logf(kHorizonEps * (1.f - r) / ((float)np * R));
                ilr = 1.f / lr;
            }
            // log of the initial-state response bound, before its r^T decay
            zs = 0.5f * lz2 - __logf(1.f - r);
            if (!(fabsf(la) < 1e30f) || !(zs < 1e30f)) bad = true;
        }
    }
    // the energy of the response past sample 0, sum_{n>=1} |h[n]|^2 =
    // Re sum_{i,j} R_i conj(R_j) q / (1 - q), q = p_i conj(p_j), with the sum
    // of the terms' magnitudes beside it (how much the sum cancels)
    if (lane < np) s_res[lane] = res;
    __syncwarp();
    // (the (j, i) term is the conjugate of the (i, j) one: lane i sums j >= i,
    // the off-diagonal terms twice)
    float e = 0.f, eabs = 0.f;
    if (lane < np) {
        const cpx pi = s_pole[lane];
        for (int j = lane; j < np; ++j) {
            const cpx pj = s_pole[j], rj = s_res[j];
            const cpx q = cmul(pi, cpx{pj.re, -pj.im});
            const cpx t = cdiv(cmul(cmul(res, cpx{rj.re, -rj.im}), q), cpx{1.f - q.re, -q.im});
            const float w = j == lane ? 1.f : 2.f;
            e = fmaf(w, t.re, e);
            eabs = fmaf(w, cabs_(t), eabs);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        eabs += __shfl_xor_sync(0xffffffffu, eabs, o);
    }
    etail = (e > 0.f && e >= 1e-4f * eabs && e < 1e30f) ? e : 0.f;
    return !__any_sync(0xffffffffu, bad);
}

// Relative output error that FP32 rounding of the signal handed from section
// k to section k + 1 causes, for a white input, at most over k (one warp):
// the rounding adds white noise of relative size 2^-24 to y_k, whose power is
// ||h_1..k||^2 per unit input power, and the sections after k pass it with
// gain ||h_k+1..K||^2, against an output of power ||h_1..K||^2, so
//   e = 2^-24 max_k ||h_1..k|| ||h_k+1..K|| / ||h_1..K||.
// The norms come in closed form from the partial fractions of each partial
// cascade (no truncated response, whatever the poles' distance from the unit
// circle): with residues R_i at the poles p_i, sum_n |h[n]|^2 = h[0]^2 +
// Re sum_{i,j} R_i conj(R_j) q_ij / (1 - q_ij), q_ij = p_i conj(p_j).  Lane i
// < 2K takes pole i; its residue in the cascade of sections a..b is the
// product over m in a..b of F_i(m) = B_m(p_i) / prod of (1 - p_l / p_i) over
// the poles l != i of section m, so prefixes and suffixes are running
// products.  Numerators enter scaled by 1 / max |b_j| (the scales cancel in
// the ratio).  Returns the estimate, or -1 where it cannot be formed (a pole
// at zero or coincident poles, a sum that cancels, overflow).
// Shared-memory scratch of the precision warp (its loops stay rolled: the
// code runs once per plan, and straight-line code of that size would be
// fetched from instruction memory one miss at a time).
struct HandoffScratch {
    cpx W[2 * kMaxSections][2 * kMaxSections];  // q_ij / (1 - q_ij)
    cpx F[2 * kMaxSections][kMaxSections];      // F_i(m)
    cpx R[2 * kMaxSections][2 * kMaxSections];  // residues: [cascade t][pole i]
    float h0[2 * kMaxSections];                 // direct term of cascade t
    float E[2 * kMaxSections];                  // prefix (0..K-1) and suffix energies
};

__device__ float handoff_error(const double (*rows)[5], const float (*rowsf)[5], int K, int lane,
                               cpx* s_pole, HandoffScratch& hs, int& blo, int& bhi) {
    const int np = 2 * K;
    blo = K;
    bhi = -1;
    if (K < 2) return 0x1p-24f;  // one section: nothing handed on
    if (lane < np) {
        const double a1 = rows[lane >> 1][3], a2 = rows[lane >> 1][4];
        const double disc = a1 * a1 - 4.0 * a2;
        cpx z;
        if (disc < 0.0) {
            const float im = 0.5f * sqrtf((float)(-disc));
            z = cpx{(float)(-0.5 * a1), (lane & 1) ? -im : im};
        } else {
            const double sq = sqrt(disc);
            z = cpx{(float)(0.5 * ((lane & 1) ? -a1 - sq : -a1 + sq)), 0.f};
        }
        s_pole[lane] = z;
    }
    __syncwarp();
    bool bad = false;
    // W[i][j] and F[i][m] for pole i = lane & 15, the j and m split between
    // the two half-warps (every entry on its own: the same values as one lane
    // per pole, in half the steps)
    const int ip = lane & 15, half = lane >> 4;
    if (ip < np) {
        const cpx pi = s_pole[ip];
        const float r2 = fmaf(pi.re, pi.re, pi.im * pi.im);
        if (!(r2 > 1e-24f)) bad = true;
        const float ir2 = r2 > 1e-24f ? 1.f / r2 : 0.f;
        const cpx inv{pi.re * ir2, -pi.im * ir2};
        const cpx inv2 = cmul(inv, inv);
#pragma unroll 1
        for (int j = half; j < np; j += 2) {
            const cpx pj = s_pole[j];
            const cpx q = cmul(pi, cpx{pj.re, -pj.im});
            const cpx d{1.f - q.re, -q.im};
            if (!(fmaf(d.re, d.re, d.im * d.im) > 1e-30f)) bad = true;
            hs.W[ip][j] = cdiv(q, d);
        }
#pragma unroll 1
        for (int m = half; m < K; m += 2) {
            const float ims = 1.f / num_scale(rowsf[m]);
            const float b0 = rowsf[m][0] * ims, b1 = rowsf[m][1] * ims, b2 = rowsf[m][2] * ims;
            cpx f{fmaf(b2, inv2.re, fmaf(b1, inv.re, b0)), fmaf(b2, inv2.im, b1 * inv.im)};
#pragma unroll 1
            for (int u = 0; u < 2; ++u) {
                const int l = 2 * m + u;
                if (l != ip) {
                    const cpx g = cmul(s_pole[l], inv);
                    const cpx h{1.f - g.re, -g.im};
                    if (fmaf(h.re, h.re, h.im * h.im) < 1e-8f) bad = true;
                    f = cdiv(f, h);
                }
            }
            hs.F[ip][m] = f;
        }
    }
    __syncwarp();
    // the energies: cascade t < K is the prefix 0..t, t >= K the suffix
    // (t - K + 1)..K-1.  First, for every cascade at once (lane t), its
    // direct term h0 (the product of its sections' b0 over their scales,
    // left to right); and (lane i) pole i's residue in every cascade that
    // holds its section, the product of its F_i over the cascade's sections
    // (left to right: prefixes grow by one factor, suffixes are formed
    // whole), zero in the others
    if (lane < 2 * K - 1) {
        const int t = lane;
        const bool pre = t < K;
        const int a = pre ? 0 : t - K + 1, b = pre ? t : K - 1;
        float h0 = 1.f;
#pragma unroll 1
        for (int m = a; m <= b; ++m) h0 *= rowsf[m][0] / num_scale(rowsf[m]);
        hs.h0[t] = h0;
    }
    if (lane < np) {
        const int sec = lane >> 1;
        cpx f[kMaxSections];
#pragma unroll
        for (int m = 0; m < kMaxSections; ++m) f[m] = m < K ? hs.F[lane][m] : cpx{1.f, 0.f};
        cpx P{1.f, 0.f};
#pragma unroll
        for (int t = 0; t < kMaxSections; ++t) {
            if (t < K) {
                P = cmul(P, f[t]);
                hs.R[t][lane] = sec <= t ? P : cpx{0.f, 0.f};
            }
        }
#pragma unroll
        for (int a = 1; a < kMaxSections; ++a) {
            if (a < K) {
                cpx S{1.f, 0.f};
#pragma unroll
                for (int m = 0; m < kMaxSections; ++m)
                    if (m >= a && m < K) S = cmul(S, f[m]);
                hs.R[K - 1 + a][lane] = sec >= a ? S : cpx{0.f, 0.f};
            }
        }
    }
    __syncwarp();
    bool ok = true;
    // two cascades per pass (ta, tb), their sums side by side: independent
    // chains of loads, products and shuffles for the scheduler to overlap
#pragma unroll 1
    for (int ta = 0; ta < 2 * K - 1; ta += 2) {
        const int tb = ta + 1 < 2 * K - 1 ? ta + 1 : ta;
        // pair (i, j): lane handles i = lane & 15 and half of the j
        float e = 0.f, ea = 0.f, f = 0.f, fa = 0.f;
        const int i = lane & 15;
        if (i < np) {
            const cpx Ria = hs.R[ta][i], Rib = hs.R[tb][i];
#pragma unroll 2
            for (int j = lane >> 4; j < np; j += 2) {
                const cpx Rja = hs.R[ta][j], Rjb = hs.R[tb][j], Wij = hs.W[i][j];
                const cpx u = cmul(cmul(Ria, cpx{Rja.re, -Rja.im}), Wij);
                const cpx v = cmul(cmul(Rib, cpx{Rjb.re, -Rjb.im}), Wij);
                e += u.re;
                ea += sqrtf(fmaf(u.re, u.re, u.im * u.im));
                f += v.re;
                fa += sqrtf(fmaf(v.re, v.re, v.im * v.im));
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            ea += __shfl_xor_sync(0xffffffffu, ea, o);
            f += __shfl_xor_sync(0xffffffffu, f, o);
            fa += __shfl_xor_sync(0xffffffffu, fa, o);
        }
        const float ha = hs.h0[ta], hb = hs.h0[tb];
        const float Ea = fmaf(ha, ha, e), Eb = fmaf(hb, hb, f);
        ok = ok && Ea > 0.f && Ea >= 1e-5f * ea && Ea < 1e30f;
        ok = ok && Eb > 0.f && Eb >= 1e-5f * fa && Eb < 1e30f;
        if (lane == 0) {
            hs.E[ta] = Ea;
            hs.E[tb] = Eb;
        }
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, bad) || !ok) return -1.f;
    // prefix k is E[k]; the suffix starting at section k + 1 is E[K + k];
    // the hand-offs whose own estimate is above the bound: [blo, bhi]
    float amp = 0.f;
#pragma unroll 1
    for (int k = 0; k + 1 < K; ++k) {
        const float a = hs.E[k] * hs.E[K + k];
        amp = fmaxf(amp, a);
        if (0x1p-24f * sqrtf(a / hs.E[K - 1]) > kHandOffErrMax) {
            blo = min(blo, k);
            bhi = k;
        }
    }
    amp = sqrtf(amp / hs.E[K - 1]);
    if (!(amp < 1e30f)) return -1.f;
    return 0x1p-24f * fmaxf(amp, 1.f);
}

// A memory horizon without partial fractions, for cascades whose poles
// coincide (or nearly so) and so have none to use: with r the largest pole
// modulus, each section's all-pole response is bounded by (n + 1) r^n and its
// whole response by B_k r^-2 (n + 1) r^n (B_k = |b0| + |b1| + |b2|), so the
// cascade's by A C(n + 2K - 1, 2K - 1) r^n with A = prod_k B_k r^-2 (the
// coefficients of 1 / (1 - r z)^(2K)).  Past the terms' peak the tail sum
// from P on is at most the term at P over (1 - its ratio to the next); P is
// the first point where that is below kHorizonEps h2 (found by bisection on
// the log of the bound).  Far more conservative than the partial-fraction
// horizon, but it holds for repeated poles.  tz: the same for the response
// of a unit initial state (it enters a section's recursion like an impulse
// of at most unit size, so B_k is taken as at least 1).  -1 where r >= 1 or
// no such P below 2^30.  One thread.
__device__ int horizon_fallback(const double (*rows)[5], int K, float h2, int& tz) {
    tz = -1;
    if (K < 1 || !(h2 > 0.f)) return -1;
    double r = 0.0, logA = 0.0, logAs = 0.0;
    for (int k = 0; k < K; ++k) {
        const double a1 = rows[k][3], a2 = rows[k][4];
        const double disc = a1 * a1 - 4.0 * a2;
        double rk;
        if (disc < 0.0) {
            rk = sqrt(a2);
        } else {
            const double sq = sqrt(disc);
            rk = fmax(fabs(0.5 * (-a1 + sq)), fabs(0.5 * (-a1 - sq)));
        }
        r = fmax(r, rk);
        const double B = fabs(rows[k][0]) + fabs(rows[k][1]) + fabs(rows[k][2]);
        if (!(B > 0.0) || !isfinite(B)) return -1;
        logA += log(B);
        logAs += log(fmax(B, 1.0));
    }
    if (!(r < 1.0 - 1e-12)) return -1;
    if (r < 1e-300) {  // a finite response
        tz = ((2 * K + 1) + 15) / 16 * 16;
        return tz;
    }
    const double m = 2.0 * K, lr = log(r);
    const double target = log((double)kHorizonEps * (double)h2);
    // the first n past the peak (ratio < 1) where the log tail bound with
    // prefactor log a is below the target, in multiples of 16; -1 if none
    auto first = [&](double loga) -> int {
        auto tail = [&](double n) {
            const double ratio = r * (n + m) / (n + 1.0);
            return loga + lgamma(n + m) - lgamma(m) - lgamma(n + 1.0) + n * lr - log1p(-ratio);
        };
        double lo = fmax(ceil((m * r - 1.0) / (1.0 - r)) + 1.0, m);
        double hi = 1073741824.0;
        if (!(tail(hi) <= target)) return -1;
        if (tail(lo) <= target) hi = lo;
        for (int it = 0; it < 40 && hi - lo > 1.0; ++it) {
            const double mid = floor(0.5 * (lo + hi));
            if (tail(mid) <= target) hi = mid;
            else lo = mid;
        }
        const int64_t n = ((int64_t)hi + 15) / 16 * 16;
        return n < (int64_t)1 << 30 ? (int)n : -1;
    };
    const int P = first(logA - 2.0 * K * lr);
    if (P < 0) return -1;
    tz = first(logAs - 2.0 * K * lr);
    return tz < 0 ? -1 : P;
}

// The horizon from the per-pole terms and ||h||_2 >= h2 (the pole warp), and
// the channel's segment length: the call's T, or longer when the horizon
// needs it (a segment is at least 2 P and long enough for the initial
// state's response to decay below the bound, rounded up to whole groups of
// G), so that long-memory channels keep a bounded warm-up instead of being
// carried; minseg, the shortest segment the horizon allows.  -1 where no
// horizon holds.
__device__ int horizon_combine(bool ok, float h2, int K, int64_t T, int64_t G, float la, float ilr,
                               float zs, float lr, int64_t& seg, int32_t& minseg,
                               int32_t& minseg_z) {
    float ptail = ilr != 0.f ? (la + __logf(h2)) * ilr : 0.f;
    // the initial state's response (each pole's share counted 2K times) has
    // decayed below the bound after tz samples
    const float lb = __logf(kHorizonEps * h2 / (float)(2 * K));
    float tz = (lr < 0.f && zs > -1e30f) ? (lb - zs) / lr : 0.f;
    for (int o = 16; o > 0; o >>= 1) {
        ptail = fmaxf(ptail, __shfl_xor_sync(0xffffffffu, ptail, o));
        tz = fmaxf(tz, __shfl_xor_sync(0xffffffffu, tz, o));
    }
    if (!ok || !(h2 > 0.f) || !(ptail < 1e9f) || !(tz < 1e9f)) return -1;
    const float need = fmaxf(ptail, (float)(2 * K));
    const int64_t P = ((int64_t)ceilf(need) + 15) / 16 * 16;
    const int64_t itz = (int64_t)ceilf(tz);
    const int64_t want = 2 * P > itz ? 2 * P : itz;
    seg = T;
    if (want > seg) seg = (want + G - 1) / G * G;
    // the shortest segments that still start their warm-up inside the
    // channel, and past an initial state's response (the streaming mode's
    // segments, where latency, not the warm-up's share, is what counts)
    const int64_t least = P > itz ? P : itz;
    minseg = (int32_t)((P + G - 1) / G * G > G ? (P + G - 1) / G * G : G);
    minseg_z = (int32_t)((least + G - 1) / G * G > G ? (least + G - 1) / G * G : G);
    return (int)P;
}

// Block C: the channel table.
__device__ __forceinline__ void plan_table(const Params& p) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = p.C, kmax = p.kmax;
    {
        // ---- channel table: exclusive scans of lengths and slot counts ----
        const int64_t T = (int64_t)p.W * kLanes * p.N;
        __shared__ int64_t s_wsum_len[kPlanWarps], s_wsum_til[kPlanWarps];
        __shared__ int64_t s_carry_len, s_carry_til;
        if (tid == 0) {
            s_carry_len = 0;
            s_carry_til = 0;
            p.hdr->status = 0;
            p.hdr->nchan = C;
        }
        __syncthreads();
        for (int base = 0; base < C; base += kPlanThreads) {
            const int c = base + tid;
            int64_t len = 0, nt = 0;
            int32_t K = 0;
            if (c < C) {
                len = p.lengths[c];
                K = p.K[c];
                if (len < 0 || K < 0 || K > kmax) {
                    set_status(p.hdr, SOS_ERR_ARG);
                    len = 0;
                    K = 0;
                }
                nt = len > 0 ? (len + T - 1) / T : 0;
            }
            // inclusive warp scans
            int64_t il = len, it = nt;
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t ol = __shfl_up_sync(0xffffffffu, il, d);
                const int64_t ot = __shfl_up_sync(0xffffffffu, it, d);
                if (lane >= d) {
                    il += ol;
                    it += ot;
                }
            }
            if (lane == 31) {
                s_wsum_len[warp] = il;
                s_wsum_til[warp] = it;
            }
            __syncthreads();
            int64_t wl = 0, wt = 0;
            for (int w = 0; w < warp; ++w) {
                wl += s_wsum_len[w];
                wt += s_wsum_til[w];
            }
            const int64_t cl = s_carry_len, ct = s_carry_til;
            if (c < C) {
                // mode, err, horizon and ntiles belong to the coefficient block
                p.chan[c].off = cl + wl + il - len;
                p.chan[c].len = len;
                p.chan[c].K = K;
                p.chan[c].slot = ct + wt + it - nt;
            }
            __syncthreads();
            if (tid == kPlanThreads - 1) {
                s_carry_len = cl + wl + il;
                s_carry_til = ct + wt + it;
            }
            __syncthreads();
        }
        if (tid == 0 && s_carry_til > p.cap_tiles) set_status(p.hdr, SOS_ERR_WORKSPACE);
    }
}

// Block c < C: the coefficient tables and the memory horizon of channel c.
// Returns false when the channel's tables were kept from the previous plan on
// this workspace (plan cache: same raw sos rows bit for bit, same K and
// length, same call-level inputs), true when they were recomputed.
__device__ __forceinline__ bool plan_channel(const Params& p) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kmax = p.kmax;

    // ---- coefficient tables of channel c ----
    // Warps 0..K-1: section k's row, then (lane 0) the squaring chain of its
    // transition powers and (all lanes) the per-lane tables.  Warp
    // kMaxSections: the b0 factoring, then the impulse response's norm bound;
    // warp kMaxSections + 1: the poles' terms of the memory horizon, then the
    // horizon.  The warp and tile tables (powers of Psi and Theta) are only
    // built for channels whose state is carried by the look-back, once the
    // horizon is decided.
    const int c = blockIdx.x;
    __shared__ double s_row[kMaxSections][5];
    __shared__ float s_rowf[kMaxSections][5];  // the same rows rounded to FP32
    __shared__ double s_G[kMaxSections];
    __shared__ float s_Ginv[kMaxSections];      // 1 / G_k
    __shared__ float s_dfscan[kMaxSections];    // the section's precision level (misc.w)
    __shared__ float s_kappa[kMaxSections];     // section_kappa()
    __shared__ float s_handoff;                 // handoff_error(), -1 if unknown
    __shared__ int s_blo, s_bhi;                // the hand-offs it blames (first, last)
    __shared__ double s_b0inv[kMaxSections];    // 1 / b0 (normalised), 0 if b0 = 0
    __shared__ float s_h2;                      // ||h||_2 lower bound
    __shared__ int s_mode, s_horizon, s_err;
    __shared__ cpx s_pole[2 * kMaxSections];
    __shared__ cpx s_res[2 * kMaxSections];
    __shared__ cpx s_pole2[2 * kMaxSections];  // the precision warp's copy
    // [0..4] Phi^(2^j); [5..9] Psi^(2^r); [10..19] Theta^(2^i)
    __shared__ dfm2 s_chain[kMaxSections][20];

    const int k = warp;
    // the section's row is read before K is known (one memory round trip, not
    // two): every section k < kmax exists in the sos array
    double row[6] = {0, 0, 0, 1, 0, 0};
    if (lane == 0 && k < kmax) {
        const double* r = p.sos + ((int64_t)c * kmax + k) * 6;
        for (int i = 0; i < 6; ++i) row[i] = r[i];
    }
    const int K = p.K[c];
    const int Kc = (K >= 0 && K <= kmax) ? K : 0;
    const bool active = k < Kc;
    if (tid == 0) s_err = 0;

    // ---- plan cache: are this channel's tables those of these inputs? ----
    unsigned char* kb = p.key + chan_key_stride(kmax) * (size_t)c;
    ChanKeyHead* kh = reinterpret_cast<ChanKeyHead*>(kb);
    unsigned long long* krow = reinterpret_cast<unsigned long long*>(kb + sizeof(ChanKeyHead));
    __shared__ int s_same[kMaxSections + 1];
    // (every value is loaded before any is compared: a short-circuit chain
    // would make the loads wait for one another)
    if (lane == 0 && k < kMaxSections) {
        unsigned long long diff = 0;
        if (k < Kc) {
            unsigned long long st[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) st[i] = krow[k * 6 + i];
#pragma unroll
            for (int i = 0; i < 6; ++i) diff |= (unsigned long long)__double_as_longlong(row[i]) ^ st[i];
        }
        s_same[k] = diff == 0;
    }
    if (tid == 0) {
        const WsHeader* h = p.hdr;
        const int32_t hv = h->key_valid, hN = h->key_N, hW = h->key_W, ha = h->key_algo,
                      hf = h->key_flags, hk = h->key_kmax, hC = h->key_C;
        const int64_t hs = h->key_seg, hc = h->key_cap;
        const int32_t kv = kh->valid, kK = kh->K;
        const int64_t kl = kh->len, len = p.lengths[c];
        const bool same = !(p.flags_opt & SOS_FLAG_REPLAN) & (hv == 1) & (hN == p.N) &
                          (hW == p.W) & (ha == p.algo) & (hf == p.flags_opt) & (hk == kmax) &
                          (hC == p.C) & (hs == p.seg) & (hc == p.cap_tiles) & (kv == 1) &
                          (kK == K) & (kl == len);
        s_same[kMaxSections] = same;
    }
    __syncthreads();
    {
        bool reuse = true;
        for (int i = 0; i <= kMaxSections; ++i) reuse = reuse && s_same[i] != 0;
        if (reuse) return false;
    }
    // recomputing: record the inputs the new tables are built from (read only
    // by the next plan launch on this workspace)
    if (lane == 0 && k < Kc)
        for (int i = 0; i < 6; ++i) krow[k * 6 + i] = (unsigned long long)__double_as_longlong(row[i]);
    if (tid == 0) {
        kh->K = K;
        kh->len = p.lengths[c];
        kh->valid = 1;
    }
    // lane 0 of each section warp normalises its row in FP64 (the FP64 unit is
    // narrow on this part: one lane per row, not the whole warp)
    if (lane == 0 && k < kMaxSections) {
        if (!active) {
            row[0] = 0; row[1] = 0; row[2] = 0; row[3] = 1; row[4] = 0; row[5] = 0;
        } else {
            if (!(finite_row(row) && row[3] != 0.0)) {
                atomicCAS(&s_err, 0, (int)SOS_ERR_COEF);
                row[0] = 0; row[1] = 0; row[2] = 0; row[3] = 1; row[4] = 0; row[5] = 0;
            }
        }
        const double ia0 = 1.0 / row[3];
        const double nb0 = row[0] * ia0, nb1 = row[1] * ia0, nb2 = row[2] * ia0;
        const double na1 = row[4] * ia0, na2 = row[5] * ia0;
        s_row[k][0] = nb0;
        s_row[k][1] = nb1;
        s_row[k][2] = nb2;
        s_row[k][3] = na1;
        s_row[k][4] = na2;
        s_rowf[k][0] = (float)nb0;
        s_rowf[k][1] = (float)nb1;
        s_rowf[k][2] = (float)nb2;
        s_rowf[k][3] = (float)na1;
        s_rowf[k][4] = (float)na2;
        s_b0inv[k] = nb0 != 0.0 ? row[3] / row[0] : 0.0;
        // both roots of z^2 + a1 z + a2 strictly inside the unit circle
        // (Jury: |a2| < 1 and |a1| < 1 + a2)
        if (active && (p.flags_opt & SOS_FLAG_CHECK_STABLE) &&
            !(fabs(na2) < 1.0 && fabs(na1) < 1.0 + na2))
            atomicCAS(&s_err, 0, (int)SOS_ERR_UNSTABLE);
    }
    __syncthreads();  // rows and errors in shared memory; nothing block-wide after this
    const int kr = k < kMaxSections ? k : 0;
    const double b0 = s_row[kr][0], b1 = s_row[kr][1], b2 = s_row[kr][2];
    const double a1 = s_row[kr][3], a2 = s_row[kr][4];

    const bool carry_only = (p.flags_opt & SOS_FLAG_CARRY_ONLY) != 0;
    if (warp == kMaxSections) {
        // the first horizon warp.  First the b0 factoring: every b0 nonzero
        // and 2^-60 < |G_k| < 2^60 for the cumulative gains G_k = b0_1 ...
        // b0_k (warp prefix product); it releases the section warps (barrier
        // 1: the Kc section warps and this one), which have been building
        // their transition powers meanwhile.
        {
            const double bj = lane < Kc ? s_row[lane < kMaxSections ? lane : 0][0] : 1.0;
            double g = bj;
            for (int d = 1; d < kMaxSections; d <<= 1) {
                const double t = __shfl_up_sync(0xffffffffu, g, d);
                if (lane >= d) g *= t;
            }
            const bool ok = lane >= Kc || (bj != 0.0 && fabs(g) > 0x1p-60 && fabs(g) < 0x1p60);
            const int mode = (Kc > 0 && __all_sync(0xffffffffu, ok)) ? 1 : 0;
            if (lane < kMaxSections) {
                s_G[lane] = mode ? g : 1.0;
                s_Ginv[lane] = mode ? 1.f / (float)g : 1.f;
            }
            if (lane == 0) {
                s_mode = mode;
                p.chan[c].mode = mode;
                p.chan[c].err = s_err;
            }
            if (Kc > 0) asm volatile("bar.arrive 1, %0;" ::"r"(32 * (Kc + 1)) : "memory");
        }
        // then the norm bound of the impulse response, for the second
        // horizon warp (barrier 3: the two horizon warps)
        const float h2 = carry_only ? 0.f : horizon_norm(s_rowf, Kc, lane);
        if (lane == 0) s_h2 = h2;
        asm volatile("bar.arrive 3, 64;" ::: "memory");
        return true;
    }
    if (warp == kMaxSections + 1) {
        // the second horizon warp: the memory horizon of channel c (against
        // the segment length) and its work units: segments when it has a
        // horizon, look-back tiles otherwise
        const int64_t T = (int64_t)p.W * kLanes * p.N;
        float la = 0.f, ilr = 0.f, zs = 0.f, lr = 0.f, etail = 0.f;
        const bool ok = !carry_only && horizon_poles(s_row, s_rowf, Kc, lane, s_pole, s_res, la,
                                                     ilr, zs, lr, etail);
        asm volatile("bar.sync 3, 64;" ::: "memory");
        // ||h||_2 from below: the first 32 samples, or half the closed-form
        // norm of the response past sample 0 where that sum is well
        // conditioned (slow-building responses of poles near the unit circle)
        const float h2 = fmaxf(s_h2, 0.5f * sqrtf(etail));
        int64_t seg = p.seg;
        int32_t minseg = 0, minseg_z = 0;
        int P = carry_only ? -1
                           : horizon_combine(ok, h2, Kc, p.seg, 32LL * p.N, la, ilr, zs, lr, seg,
                                             minseg, minseg_z);
        // a channel without a partial-fraction horizon (repeated poles)
        // takes the cruder bound: always in backward plans, which have no
        // look-back (so that it is still cut into segments, warm-ups of P on
        // both sides), and in forward plans where the channel is long enough
        // for at least eight segments (the look-back is faster below that)
        if (P < 0 && !carry_only && Kc > 0) {
            int Pf = -1, tzf = -1;
            if (lane == 0) Pf = horizon_fallback(s_row, Kc, s_h2, tzf);
            Pf = __shfl_sync(0xffffffffu, Pf, 0);
            tzf = __shfl_sync(0xffffffffu, tzf, 0);
            const int64_t want = Pf >= 0 ? (2LL * Pf > tzf ? 2LL * Pf : (int64_t)tzf) : 0;
            const int64_t lenc = p.lengths[c];
            if (Pf >= 0 && ((p.flags_opt & kFlagBackwardPlan) || lenc >= 8 * want)) {
                const int64_t G = 32LL * p.N;
                P = Pf;
                seg = p.seg;
                if (want > seg) seg = (want + G - 1) / G * G;
                minseg = (int32_t)((Pf + G - 1) / G * G > G ? (Pf + G - 1) / G * G : G);
                minseg_z = (int32_t)((tzf + G - 1) / G * G > minseg ? (tzf + G - 1) / G * G
                                                                     : minseg);
            }
        }
        // and a channel with no horizon at all is one segment, run from its
        // start to its end by one pipeline
        const int single = (P < 0 && (p.flags_opt & kFlagBackwardPlan)) ? 1 : 0;
        if (single) P = 0;
        if (lane == 0) {
            int64_t len = p.lengths[c];
            if (len < 0) len = 0;
            int64_t nt;
            if (len == 0) nt = 0;
            else if (single) nt = 1;
            else if (P >= 0) nt = (len + seg - 1) / seg;
            else nt = (len + T - 1) / T;
            p.chan[c].horizon = P;
            p.chan[c].single = (int16_t)single;
            if (Kc == 0) p.chan[c].ext = 0;  // (else written by the first section warp)
            p.chan[c].seg = P >= 0 ? seg : p.seg;
            p.chan[c].minseg = P >= 0 ? minseg : 0;
            p.chan[c].minseg_z = P >= 0 ? minseg_z : 0;
            p.chan[c].ntiles = (int32_t)nt;
            s_horizon = P;
        }
        // release the section warps waiting for the decision (barrier 2:
        // the Kc section warps and this one)
        if (Kc > 0) asm volatile("bar.arrive 2, %0;" ::"r"(32 * (Kc + 2)) : "memory");
        return true;
    }
    if (warp == kMaxSections + 2) {
        // the precision warp: how much FP32 rounding between sections would
        // cost at the output (released with barrier 2)
        const bool skip = carry_only || (p.flags_opt & kFlagBackwardPlan) || Kc == 0;
        __shared__ HandoffScratch s_hs;
        int blo = Kc, bhi = -1;
        const float e =
            skip ? 0.f : handoff_error(s_row, s_rowf, Kc, lane, s_pole2, s_hs, blo, bhi);
        if (lane == 0) {
            s_handoff = e;
            s_blo = blo;
            s_bhi = bhi;
        }
        if (Kc > 0) asm volatile("bar.arrive 2, %0;" ::"r"(32 * (Kc + 2)) : "memory");
        return true;
    }
    if (!active) return true;

    // ---- Phi: double-float squaring chain (lane 0) ----
    const int N = p.N, W = p.W;
    if (lane == 0) {
        const dfm2 A{df_of_double(-a1), df{1.f, 0.f}, df_of_double(-a2), df{0.f, 0.f}};
        dfm2 P = A;
        // (exact additions: Phi^16 also seeds the look-back's tile powers)
        for (int n = 1; n < N; n <<= 1) P = dfm_mul(P, P);  // A^N (N a power of two)
        s_chain[k][0] = P;
        for (int j = 1; j < 5; ++j) {
            P = dfm_mul(P, P);
            s_chain[k][j] = P;
        }
    }
    // cyclic-reduction coefficients in double-float (lane 1, alongside lane
    // 0's chain; about 44 bits, the FP64 unit being narrow on this part)
    if (lane == 1 && p.algo == 2) {
        Coef32* o = p.c32 + ((int64_t)c * kmax + k);
        df e = df_of_double(a1), f = df_of_double(a2);
        float kappa = 0.f;
        float dd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int lv = 0;
        for (int n = 1; n < N; n <<= 1, ++lv) {
            const df g = df_div(f, e);
            const float gh = df_to_float(g);
            if (e.hi == 0.f || !(fabsf(gh) < INFINITY)) kappa = INFINITY;
            else if (fabsf(gh) > kappa) kappa = fabsf(gh);
            o->cr_lv[lv] = make_float4(df_to_float(e), df_to_float(f), gh,
                                       df_to_float(df_add(e, df_neg(g))));
            dd[lv] = -df_to_float(df_mul(f, g));
            const df e2 = df_add(df_add(f, f), df_neg(df_mul(e, e)));
            f = df_mul(f, f);
            e = e2;
        }
        o->cr_d[0] = make_float4(dd[0], dd[1], dd[2], dd[3]);
        o->cr_d[1] = make_float4(dd[4], dd[5], dd[6], dd[7]);
        // terminal scan powers C^(2^j), C = [[-e_n, -f_n], [1, 0]], double-float
        dfm2 C{df_neg(e), df_neg(f), df{1.f, 0.f}, df{0.f, 0.f}};
        for (int j = 0; j < 5; ++j) {
            o->cr_tpow[j] = to_f4(C);
            C = dfm_mul(C, C);
        }
        const bool ok = kappa <= kCrKappaMax;
        o->cr_misc = make_float4(df_to_float(e), df_to_float(f), kappa, ok ? 1.f : 0.f);
    }
    // barrier 1 (the Kc section warps and the horizon warp): the mode and
    // gains are in shared memory, and this warp's lane 0 has finished its
    // chain
    asm volatile("bar.sync 1, %0;" ::"r"(32 * (Kc + 1)) : "memory");
    const int mode = s_mode;

    Coef32* out32 = p.c32 + ((int64_t)c * kmax + k);
    CoefDF* outdf = p.cdf + ((int64_t)c * kmax + k);
    float m;  // largest entry of the section's powers (all lanes)
    {
        // Phi^lane by binary powering (exact additions: for poles near the
        // unit circle the entries come out of near-cancelling sums)
        dfm2 P = dfm_identity();
        for (int j = 0; j < 5; ++j)
            if ((lane >> j) & 1) P = dfm_mul(P, s_chain[k][j]);
        out32->lane_pow[lane] = to_f4(P);
        out32->lane_lo[lane] = to_f4_lo(P);
        m = max_entry(P);
        if (lane < 5) {
            const dfm2 Q = s_chain[k][lane];
            out32->phi_pow[lane] = to_f4(Q);
            out32->phi_lo[lane] = to_f4_lo(Q);
            m = fmaxf(m, max_entry(Q));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
        // extended precision (FP64 work on one lane: the FP64 pipe is narrow)
        const float sens = coef_sensitivity(a1, a2);
        const float ext = (m > kDfScanEntry || sens > (float)kDfCoefSens)
                              ? 2.f
                              : (sens > (float)kAloCoefSens ? 1.f : 0.f);
        s_dfscan[k] = ext;
        s_kappa[k] = (float)section_kappa(b0, b1, b2, a1, a2);
        // b1 / b0 and b2 / b0 when b0 is factored (1 / b0 from the rows phase)
        const double sb = mode ? s_b0inv[k] : 1.0;
        out32->ab = make_float4((float)a1, (float)a2, (float)(b1 * sb), (float)(b2 * sb));
        out32->alo = make_float4((float)(a1 - (double)(float)a1), (float)(a2 - (double)(float)a2),
                                 0.0f, 0.0f);
        out32->misc = make_float4((float)b0, (float)s_G[k], s_Ginv[k], ext);
        out32->braw = make_float4((float)b0, (float)b1, (float)b2, 0.0f);
        out32->blo = make_float4((float)(b0 - (double)(float)b0), (float)(b1 - (double)(float)b1),
                                 (float)(b2 - (double)(float)b2), 0.0f);
    }

    // ---- Psi = A^(NL) and Theta = A^T, only for channels carried by the
    // look-back (its warp and tile steps) ----
    asm volatile("bar.sync 2, %0;" ::"r"(32 * (Kc + 2)) : "memory");
    if (k == 0 && lane == 0) {
        // the channel's precision class: the largest section level, or 3
        // (double-float samples) for a channel within its memory horizon
        // whose hand-off error estimate is too large (or unknown while some
        // section needs the double-float scan), whose sections are
        // ill-conditioned (kappa), or when the call asks for it
        int16_t e = 0;
        float kap = 0.f;
        // the double-float range: the sections on both sides of every
        // hand-off the estimate blames (the signal there has to be handed on
        // beyond FP32, so it is computed in double-float up to it and taken in
        // double-float after it) and every ill-conditioned section; all of
        // them when the estimate is unreliable or the call asks for it
        int lo = s_bhi >= 0 ? s_blo : Kc, hi = s_bhi >= 0 ? s_bhi + 1 : -1;
        for (int j = 0; j < Kc; ++j) {
            e = (int16_t)max((int)e, (int)s_dfscan[j]);
            kap = fmaxf(kap, s_kappa[j]);
            if (!(s_kappa[j] * 0x1p-24f <= kSectionErrMax)) {
                lo = min(lo, j);
                hi = max(hi, j);
            }
        }
        const float h = s_handoff;
        const bool all = (p.flags_opt & SOS_FLAG_DOUBLE_FLOAT) || (h < 0.f && e >= 2);
        const bool whole = all || h > kHandOffErrMax || !(kap * 0x1p-24f <= kSectionErrMax);
        if (all || hi < lo) {
            lo = 0;
            hi = Kc - 1;
        }
        if (whole && s_horizon >= 0 && !(p.flags_opt & kFlagBackwardPlan)) e = 3;
        p.chan[c].ext = e;
        p.chan[c].dflo = (int16_t)(e == 3 ? lo : 0);
        p.chan[c].dfhi = (int16_t)(e == 3 ? hi : Kc - 1);
    }
    if (s_horizon >= 0) return true;
    if (lane == 0) {
        dfm2 P = dfm_mul(s_chain[k][4], s_chain[k][4]);  // Psi = Phi^32
        s_chain[k][5] = P;
        for (int r = 1; r < 5; ++r) {
            P = dfm_mul(P, P);
            s_chain[k][5 + r] = P;
        }
    }
    __syncwarp();
    if (lane < 16) {
        dfm2 P = dfm_identity();
        for (int r = 0; r < 4; ++r)
            if ((lane >> r) & 1) P = dfm_mul(P, s_chain[k][5 + r]);
        out32->psi_w[lane] = to_f4(P);
    }
    if (lane < 4) out32->psi_pow[lane] = to_f4(s_chain[k][5 + lane]);
    if (lane == 0) {
        dfm2 Th = dfm_identity();  // Theta = Psi^W, any W <= 31
        for (int r = 0; r < 5; ++r)
            if ((W >> r) & 1) Th = dfm_mul(Th, s_chain[k][5 + r]);
        s_chain[k][10] = Th;
        for (int i = 1; i < 10; ++i) s_chain[k][10 + i] = dfm_mul(s_chain[k][9 + i], s_chain[k][9 + i]);
    }
    __syncwarp();
    {
        // Theta^lane and Theta^(32 lane) by binary powering
        dfm2 Q = dfm_identity(), R = dfm_identity();
        for (int j = 0; j < 5; ++j)
            if ((lane >> j) & 1) {
                Q = dfm_mul(Q, s_chain[k][10 + j]);
                R = dfm_mul(R, s_chain[k][15 + j]);
            }
        outdf->theta_pow[lane][0] = make_float4(Q.a.hi, Q.a.lo, Q.b.hi, Q.b.lo);
        outdf->theta_pow[lane][1] = make_float4(Q.c.hi, Q.c.lo, Q.d.hi, Q.d.lo);
        if (lane < 18) {
            outdf->theta_hi[lane][0] = make_float4(R.a.hi, R.a.lo, R.b.hi, R.b.lo);
            outdf->theta_hi[lane][1] = make_float4(R.c.hi, R.c.lo, R.d.hi, R.d.lo);
        }
        if (lane == 0) {
            const dfm2 T32 = s_chain[k][15];
            outdf->theta_pow[32][0] = make_float4(T32.a.hi, T32.a.lo, T32.b.hi, T32.b.lo);
            outdf->theta_pow[32][1] = make_float4(T32.c.hi, T32.c.lo, T32.d.hi, T32.d.lo);
        }
    }
    return true;
}

// Dispatch (the whole CTA that finishes the plan last).  First the
// tile prefix tb over the channels' tile counts.  Then, when some channel
// with more than one tile carries its state by look-back, the interleaved
// order: tiles are handed out round by round, round r holding tile r of every
// channel that has more than r tiles, so that a tile's predecessor in its own
// channel was dispatched a whole round earlier and has usually finished and
// the look-back finds its outgoing state at once.  Channels are sorted by
// decreasing tile count (bitonic sort in shared memory), which makes each
// round a prefix of that order.  Otherwise (every channel within its memory
// horizon, or more than kMaxSortChannels channels) nrounds = 0 and tiles go
// channel by channel, which keeps a tile's overlap with its predecessor in L2.
__device__ __noinline__ void order_pass(const Params& p, unsigned long long* s_key) {
    const int tid = threadIdx.x, C = p.C;
    const int lane = tid & 31, warp = tid >> 5;
    __shared__ int64_t s_carry;
    __shared__ int64_t s_wsum[32];
    // ---- prefixes: look-back tiles of the carried channels (tb, by
    // channel) and segments of the channels within their horizon (tbp, by
    // dispatch position: porder lists the channels run with double-float
    // samples first, their segments costing about ten times the others',
    // so that they are handed out first and do not trail the launch) ----
    __shared__ int64_t s_carry2;
    __shared__ int64_t s_wsum2[32];
    // block-wide exclusive scan of one value per thread (every thread
    // calls it); s_c carries the running total between rounds
    auto scan = [&](int64_t v, int64_t* s_w, int64_t* s_c) -> int64_t {
        int64_t inc = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        int64_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_w[w];
        const int64_t carry = *s_c;
        __syncthreads();
        if (tid == blockDim.x - 1) *s_c = carry + wpre + inc;
        __syncthreads();
        return carry + wpre + inc - v;
    };
    if (tid == 0) {
        s_carry = 0;
        s_carry2 = 0;
    }
    __syncthreads();
    int carried = 0;
    // channels run with double-float samples: tiles of carried channels, and
    // the class-3 channels' dispatch positions
    for (int base = 0; base < C; base += blockDim.x) {
        const int c = base + tid;
        int64_t nt = 0, f3 = 0;
        if (c < C) {
            // written by other blocks of this launch: read past L1
            const int32_t hz = __ldcg(&p.chan[c].horizon), ntl = __ldcg(&p.chan[c].ntiles);
            const int16_t ext = __ldcg(&p.chan[c].ext);
            if (hz < 0) {
                nt = ntl;
                if (nt > 1) carried = 1;
            } else {
                f3 = ext >= 3 ? 1 : 0;
            }
        }
        const int64_t t0 = scan(nt, s_wsum, &s_carry);
        const int64_t q0 = scan(f3, s_wsum2, &s_carry2);
        if (c < C) {
            p.tb[c] = t0;
            if (f3) p.porder[q0] = c;
        }
    }
    const int64_t total = s_carry, n3 = s_carry2;
    __syncthreads();
    if (tid == 0) s_carry2 = 0;
    __syncthreads();
    for (int base = 0; base < C; base += blockDim.x) {
        const int c = base + tid;
        int64_t f = 0;
        if (c < C) {
            const int32_t hz = __ldcg(&p.chan[c].horizon);
            const int16_t ext = __ldcg(&p.chan[c].ext);
            f = (hz >= 0 && ext >= 3) ? 0 : 1;
        }
        const int64_t q = scan(f, s_wsum2, &s_carry2);
        if (c < C && f) p.porder[n3 + q] = c;
    }
    __syncthreads();  // porder complete (block-wide visibility of its global writes)
    if (tid == 0) s_carry2 = 0;
    __syncthreads();
    for (int base = 0; base < C; base += blockDim.x) {
        const int i = base + tid;
        int64_t ns = 0;
        if (i < C) {
            const int c = p.porder[i];
            const int32_t hz = __ldcg(&p.chan[c].horizon), ntl = __ldcg(&p.chan[c].ntiles);
            if (hz >= 0) ns = ntl;
        }
        const int64_t q = scan(ns, s_wsum2, &s_carry2);
        if (i < C) p.tbp[i] = q;
    }
    const int64_t total2 = s_carry2;
    const bool interleave = __syncthreads_or(carried) != 0 && C <= kMaxSortChannels;
    if (tid == 0) {
        const bool bad = __ldcg(&p.hdr->status) == SOS_ERR_WORKSPACE;
        p.tb[C] = total;
        p.tbp[C] = total2;
        p.hdr->total_tiles = bad ? 0 : total;
        p.hdr->total_pipe = bad ? 0 : total2;
        if (!interleave) p.hdr->nrounds = 0;
    }
    if (!interleave) return;
    __syncthreads();
    int n = 1;
    while (n < C) n <<= 1;
    for (int i = tid; i < n; i += blockDim.x) {
        // ascending sort of (MAX - ntiles, channel): decreasing tile count,
        // then increasing channel index; padding sorts last
        const unsigned long long nt = (i < C && __ldcg(&p.chan[i].horizon) < 0)
                                          ? (unsigned long long)__ldcg(&p.chan[i].ntiles)
                                          : 0ull;
        s_key[i] = i < C ? (((0xffffffffull - nt) << 32) | (unsigned)i) : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = s_key[i], b = s_key[j];
                    if ((a > b) == up) {
                        s_key[i] = b;
                        s_key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < C; i += blockDim.x) p.order[i] = (int32_t)(s_key[i] & 0xffffffffu);
    const int64_t nrounds = C > 0 ? (int64_t)(0xffffffffull - (s_key[0] >> 32)) : 0;
    // rp[r] = sum over rounds q < r of (channels with more than q tiles)
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base <= nrounds; base += blockDim.x) {
        const int64_t r = base + tid;
        int64_t cnt = 0;
        if (r < nrounds) {
            // channels with ntiles > r: a prefix of the sorted order (binary search)
            int lo = 0, hi = C;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const int64_t nt = (int64_t)(0xffffffffull - (s_key[mid] >> 32));
                if (nt > r) lo = mid + 1; else hi = mid;
            }
            cnt = lo;
        }
        int64_t inc = cnt;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        int64_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        const int64_t carry = s_carry;
        if (r <= nrounds) p.rp[r] = carry + wpre + inc - cnt;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = carry + wpre + inc;
        __syncthreads();
    }
    if (tid == 0) p.hdr->nrounds = nrounds;
}

}  // namespace sosf

namespace sosf {

// Blocks 0..C-1: coefficients and horizon of one channel each.  Block C: the
// channel table.  The last block to finish then builds the dispatch order
// (order_pass), so that a call's set-up is a single launch.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(Params p) {
    // the filtering kernel queued behind this one may be launched once every
    // CTA of the plan has started (it waits for the plan's completion before
    // it reads anything the plan writes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ unsigned long long s_key[];
    __shared__ int s_last, s_changed;
    bool changed = false;
    if ((int)blockIdx.x == p.C) plan_table(p);
    else changed = plan_channel(p);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (changed) atomicAdd(&p.hdr->plan_changed, 1u);
        __threadfence();  // this block's tables before its arrival
        const unsigned prev = atomicAdd(&p.hdr->plan_done, 1u);
        s_last = prev == (unsigned)p.C;  // C + 1 blocks
        if (s_last) p.hdr->plan_done = 0;  // for the next launch on this workspace
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // every block's tables before the order pass reads them
    if (threadIdx.x == 0) s_changed = (int)__ldcg(&p.hdr->plan_changed);
    __syncthreads();
    // every channel kept its tables (which implies the same call-level
    // inputs): the prefixes and the dispatch order are those of the previous
    // plan as well
    if (s_changed != 0) order_pass(p, s_key);
    __syncthreads();
    if (threadIdx.x == 0) {
        WsHeader* h = p.hdr;
        h->key_N = p.N;
        h->key_W = p.W;
        h->key_algo = p.algo;
        h->key_flags = p.flags_opt;
        h->key_kmax = p.kmax;
        h->key_C = p.C;
        h->key_seg = p.seg;
        h->key_cap = p.cap_tiles;
        h->key_valid = 1;
        h->last_recomputed = s_changed;
        h->plan_changed = 0;
    }
}

cudaError_t launch_plan(const Params& p, cudaStream_t stream) {
    int n = 1;
    while (n < p.C && n < kMaxSortChannels) n <<= 1;
    const size_t smem = p.C <= kMaxSortChannels ? sizeof(unsigned long long) * (size_t)n : 0;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t err =
            cudaFuncSetAttribute(plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(unsigned long long) * kMaxSortChannels));
        if (err != cudaSuccess) return err;
        attr_set = true;
    }
    plan_kernel<<<p.C + 1, kPlanThreads, smem, stream>>>(p);
    return cudaGetLastError();
}
}  // namespace sosf
