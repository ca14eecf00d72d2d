// One section of the cascade over one group of 32 N samples held as lane
// chunks in registers: S3 non-recursive stage, S4-PH (particular solution,
// lane scan, re-run from the true lane state), the group's outgoing DF2T
// state, and S8 (zf) for the lane holding the channel's last sample.  Used
// by the forward section pipeline and, on time-reversed data, by the adjoint.
#pragma once

#include "sos_pipe.cuh"

namespace sosf {

// v[mq] and v[mq - 1] (0 when mq = 0) by compile-time-indexed selects, for
// a run-time mq: no dynamic register indexing, no scratch memory.
template <int N>
__device__ __forceinline__ void pick_pair(const float (&v)[N], int mq, float& q0, float& q1) {
    q0 = v[0];
    q1 = 0.f;
#pragma unroll
    for (int m = 1; m < N; ++m) {
        q0 = m == mq ? v[m] : q0;
        q1 = m == mq ? v[m - 1] : q1;
    }
}

// Chunk v[] <-> the lane's row (N floats, 16-byte aligned).
template <int N>
__device__ __forceinline__ void chunk_to_row(const float (&v)[N], float* row) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
        *reinterpret_cast<float4*>(row + 4 * q) =
            make_float4(v[4 * q + 0], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

template <int N>
__device__ __forceinline__ void row_to_chunk(float (&v)[N], const float* row) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 t = *reinterpret_cast<const float4*>(row + 4 * q);
        v[4 * q + 0] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}


// One section over one group, lane chunk v[] in registers, from the group's
// incoming DF2T state (Z1, Z2) (scaled by 1/G_k when b0 is factored); leaves
// the group's outgoing state in (Z1, Z2).  ZF: the group holds the channel's
// last sample (at element mq of the chunk of the lane where zf_owner is set),
// whose DF2T state goes to zf_dst; a separate instantiation, so that other
// groups do not run the selects it needs.  s_own: the lane's row (N floats,
// 16-byte aligned), scratch for DFS.
// INJ: a DF2T state (zi1, zi2) enters at group-relative sample pinj instead
// of the group start (the inputs before it being zero): added to the
// all-pole input at pinj and pinj + 1 (the backward's recompute of a
// channel's first group, whose grid is anchored elsewhere).
// DFS: extended precision for ill-conditioned sections: the lane scan and the
// fold run in double-float, with the powers' low parts phi_lo and lpl beside
// phi and lp, and the in-lane recursions add the low parts alo of a1, a2
// (the samples stay FP32).
// AL: the in-lane recursions add the low parts alo of a1, a2 (a section
// whose poles FP32 coefficients would displace noticeably; implied by DFS).
template <int N, bool FACT, bool ZF = false, bool INJ = false, bool DFS = false, bool AL = DFS>
__device__ __forceinline__ void pipe_section(float (&v)[N], const float4 ab, const float b0,
                                             const float4* phi, const float4 lp, float& Z1,
                                             float& Z2, bool zf_owner, int mq, float* s_own,
                                             float* zf_dst, float G, int pinj = -1,
                                             float zi1 = 0.f, float zi2 = 0.f,
                                             const float4* phi_lo = nullptr,
                                             float4 lpl = {0.f, 0.f, 0.f, 0.f},
                                             float2 alo = {0.f, 0.f}) {
    const int lane = threadIdx.x & 31;
    const float a1 = ab.x, a2 = ab.y, b1 = ab.z, b2 = ab.w;
    // the all-pole terms, with a_i = ab + alo for AL (the low-part products
    // go first, into the smaller terms), FP32 a_i otherwise:
    // ap2 = t - a1 y1 - a2 y2, ap1 = t - a1 y1, st2 = -a1 y1 - a2 y2, st1 = -a2 y
    auto ap2 = [&](float y1, float y2, float t) {
        return fmaf(-a1, y1, fmaf(-a2, y2, AL ? fmaf(-alo.x, y1, fmaf(-alo.y, y2, t)) : t));
    };
    auto ap1 = [&](float y1, float t) { return fmaf(-a1, y1, AL ? fmaf(-alo.x, y1, t) : t); };
    auto st2 = [&](float y1, float y2) {
        return fmaf(-a1, y1, AL ? fmaf(-a2, y2, fmaf(-alo.x, y1, -alo.y * y2)) : -a2 * y2);
    };
    auto st1 = [&](float y) { return AL ? fmaf(-a2, y, -alo.y * y) : -a2 * y; };

    // S8 support: the section input at the channel's last sample (element mq
    // of the owner's chunk), picked by compile-time-indexed selects
    float xq = 0.f, xqm1 = 0.f;
    if (ZF) pick_pair<N>(v, mq, xq, xqm1);

    // S3: non-recursive stage with zero history inside the lane
    const float xl1 = v[N - 1], xl2 = v[N - 2];
#pragma unroll
    for (int m = N - 1; m >= 2; --m)
        v[m] = fmaf(b2, v[m - 2], fmaf(b1, v[m - 1], FACT ? v[m] : b0 * v[m]));
    v[1] = fmaf(b1, v[0], FACT ? v[1] : b0 * v[1]);
    if (!FACT) v[0] = b0 * v[0];
    if (INJ) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
            const int pos = lane * N + m;
            v[m] += pos == pinj ? zi1 : (pos == pinj + 1 ? zi2 : 0.f);
        }
    }

    // S4 (i): particular solution from zero state, terminal values only
    float w0 = v[0], w1 = ap1(w0, v[1]);
#pragma unroll
    for (int m = 2; m < N; ++m) {
        const float w2 = ap2(w1, w0, v[m]);
        w0 = w1;
        w1 = w2;
    }
    float S1 = fmaf(b1, xl1, fmaf(b2, xl2, st2(w1, w0)));
    float S2 = fmaf(b2, xl1, st1(w1));

    float zin1, zin2;
    if (DFS) {
        // S4 (ii) and the fold in double-float; the chunk waits in the lane's
        // row (s_own) meanwhile, so that its registers serve the scan
        chunk_to_row<N>(v, s_own);
        df s1 = df_from(S1), s2 = df_from(S2);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int d = 1 << j;
            df t1{__shfl_up_sync(0xffffffffu, s1.hi, d), __shfl_up_sync(0xffffffffu, s1.lo, d)};
            df t2{__shfl_up_sync(0xffffffffu, s2.hi, d), __shfl_up_sync(0xffffffffu, s2.lo, d)};
            if (lane < d) {
                t1 = df_from(0.f);
                t2 = df_from(0.f);
            }
            const float4 h = phi[j], l = phi_lo[j];
            s1 = df_add_fast(s1, df_add_fast(df_mul(df{h.x, l.x}, t1), df_mul(df{h.y, l.y}, t2)));
            s2 = df_add_fast(s2, df_add_fast(df_mul(df{h.z, l.z}, t1), df_mul(df{h.w, l.w}, t2)));
        }
        df e1{__shfl_up_sync(0xffffffffu, s1.hi, 1), __shfl_up_sync(0xffffffffu, s1.lo, 1)};
        df e2{__shfl_up_sync(0xffffffffu, s2.hi, 1), __shfl_up_sync(0xffffffffu, s2.lo, 1)};
        if (lane == 0) {
            e1 = df_from(0.f);
            e2 = df_from(0.f);
        }
        const df z1 = df_from(Z1), z2 = df_from(Z2);
        zin1 = df_to_float(df_add_fast(
            e1, df_add_fast(df_mul(df{lp.x, lpl.x}, z1), df_mul(df{lp.y, lpl.y}, z2))));
        zin2 = df_to_float(df_add_fast(
            e2, df_add_fast(df_mul(df{lp.z, lpl.z}, z1), df_mul(df{lp.w, lpl.w}, z2))));
        row_to_chunk<N>(v, s_own);
    } else {
        // S4 (ii): inclusive scan over lanes, z_{l+1} = Phi z_l + s_l
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int d = 1 << j;
            float t1 = __shfl_up_sync(0xffffffffu, S1, d);
            float t2 = __shfl_up_sync(0xffffffffu, S2, d);
            t1 = lane >= d ? t1 : 0.f;
            t2 = lane >= d ? t2 : 0.f;
            S1 = fmaf(phi[j].x, t1, fmaf(phi[j].y, t2, S1));
            S2 = fmaf(phi[j].z, t1, fmaf(phi[j].w, t2, S2));
        }
        float E1 = __shfl_up_sync(0xffffffffu, S1, 1);
        float E2 = __shfl_up_sync(0xffffffffu, S2, 1);
        if (lane == 0) {
            E1 = 0.f;
            E2 = 0.f;
        }
        // fold the group's incoming state into this lane's: Phi^lane Z + E
        zin1 = fmaf(lp.x, Z1, fmaf(lp.y, Z2, E1));
        zin2 = fmaf(lp.z, Z1, fmaf(lp.w, Z2, E2));
    }

    // S4 (iii): re-run the recursion from the true incoming state
    v[0] = v[0] + zin1;
    v[1] = ap1(v[0], v[1] + zin2);
#pragma unroll
    for (int m = 2; m < N; ++m) v[m] = ap2(v[m - 1], v[m - 2], v[m]);

    // the group's outgoing state, from lane 31's last two inputs and outputs
    const float o1 = fmaf(b1, xl1, fmaf(b2, xl2, st2(v[N - 1], v[N - 2])));
    const float o2 = fmaf(b2, xl1, st1(v[N - 1]));
    Z1 = __shfl_sync(0xffffffffu, o1, 31);
    Z2 = __shfl_sync(0xffffffffu, o2, 31);
    // a state injected at the group's last sample: its second component
    // belongs to the next group
    if (INJ && pinj == 32 * N - 1) Z1 += zi2;

    // S8: final state at the channel's last sample
    if (ZF) {
        float yq, yqm1;
        pick_pair<N>(v, mq, yq, yqm1);
        float f1;
        if (mq >= 1) f1 = fmaf(b1, xq, fmaf(b2, xqm1, st2(yq, yqm1)));
        else f1 = fmaf(b1, xq, ap1(yq, zin2));
        const float f2 = fmaf(b2, xq, st1(yq));
        if (zf_owner) {
            zf_dst[0] = f1 * G;
            zf_dst[1] = f2 * G;
        }
    }
}

// Coefficients of one section in double-float, for channels run in extended
// precision throughout (normalised by a0, never factored).
struct SecDF {
    df a1, a2, b0, b1, b2;
};

// One section over one group with the samples themselves in double-float:
// the high parts in the lane's chunk vh[] (registers), the low parts in the
// lane's row lo[] (shared memory, 16-byte aligned, read and written four at
// a time, which the row padding makes bank-conflict free; registers would
// double the section's footprint).  The same steps as pipe_section -- S3 with
// zero in-lane history, S4 (i) the particular solution's terminal pair, (ii)
// the lane scan and the fold of the group's incoming state, (iii) the re-run
// from the true lane state, the group's outgoing state, S8 -- every one in
// double-float (about 44 bits), so that neither the samples handed from
// section to section nor the recursions' own roundings are limited to FP32.
// For cascades in which later sections attenuate what earlier ones pass
// (poles next to the unit circle), where FP32 rounding of an intermediate
// signal reaches the output amplified many times.  Z1, Z2: the group's
// incoming DF2T state, left outgoing.  ZF: the group holds the channel's last
// sample (element mq of the chunk of the lane where zf_owner is set), whose
// state goes to zf_dst.
template <int N, bool ZF = false>
__device__ __forceinline__ void pipe_section_dfx(float (&vh)[N], float* lo, const SecDF& q,
                                                 const float4* phi, const float4* phi_lo,
                                                 const float4 lp, const float4 lpl, df& Z1,
                                                 df& Z2, bool zf_owner, int mq, float* zf_dst) {
    const int lane = threadIdx.x & 31;
    const df na1 = df_neg(q.a1);
    float4* lo4 = reinterpret_cast<float4*>(lo);
    df xq{0.f, 0.f}, xqm1{0.f, 0.f};
    if (ZF) {
        pick_pair<N>(vh, mq, xq.hi, xqm1.hi);
        xq.lo = lo[mq];
        xqm1.lo = mq >= 1 ? lo[mq - 1] : 0.f;
    }
    const float4 top = lo4[N / 4 - 1];
    const df xl1{vh[N - 1], top.w}, xl2{vh[N - 2], top.z};
    // S3, top down (block q of four samples reads the inputs of blocks q and
    // q - 1, which the steps below it have not overwritten yet)
#pragma unroll
    for (int b = N / 4 - 1; b >= 0; --b) {
        const float4 c = lo4[b];
        const float4 d = b > 0 ? lo4[b > 0 ? b - 1 : 0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float l[6] = {d.z, d.w, c.x, c.y, c.z, c.w};  // lo of x_{4b-2} .. x_{4b+3}
        float h[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int m = 4 * b - 2 + i;
            h[i] = m >= 0 ? vh[m >= 0 ? m : 0] : 0.f;
        }
        float out[4];
#pragma unroll
        for (int i = 3; i >= 0; --i) {
            const int m = 4 * b + i;
            df u;
            if (m >= 2)
                u = df_dot3(q.b0, df{h[i + 2], l[i + 2]}, q.b1, df{h[i + 1], l[i + 1]}, q.b2,
                            df{h[i], l[i]});
            else if (m == 1)
                u = df_dot3(q.b0, df{h[i + 2], l[i + 2]}, q.b1, df{h[i + 1], l[i + 1]},
                            df{0.f, 0.f}, df{0.f, 0.f});
            else
                u = df_mul(q.b0, df{h[i + 2], l[i + 2]});
            vh[m] = u.hi;
            out[i] = u.lo;
        }
        lo4[b] = make_float4(out[0], out[1], out[2], out[3]);
    }
    // S4 (i): the particular solution from zero state, its terminal pair
    df w0{0.f, 0.f}, w1{0.f, 0.f};
#pragma unroll
    for (int b = 0; b < N / 4; ++b) {
        const float4 c = lo4[b];
        const float l[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = 4 * b + i;
            const df u{vh[m], l[i]};
            df w2;
            if (m == 0) w2 = u;
            else if (m == 1) w2 = df_rec1(u, q.a1, w1);
            else w2 = df_rec(u, q.a1, w1, q.a2, w0);
            w0 = w1;
            w1 = w2;
        }
    }
    df s1 = df_rec1(df_dot3(q.b1, xl1, q.b2, xl2, na1, w1), q.a2, w0);
    df s2 = df_rec1(df_mul(q.b2, xl1), q.a2, w1);
    // S4 (ii): lane scan, z_{l+1} = Phi z_l + s_l, in double-float
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        df t1{__shfl_up_sync(0xffffffffu, s1.hi, d), __shfl_up_sync(0xffffffffu, s1.lo, d)};
        df t2{__shfl_up_sync(0xffffffffu, s2.hi, d), __shfl_up_sync(0xffffffffu, s2.lo, d)};
        if (lane < d) {
            t1 = df{0.f, 0.f};
            t2 = df{0.f, 0.f};
        }
        const float4 h = phi[j], l = phi_lo[j];
        s1 = df_add(s1, df_add(df_mul(df{h.x, l.x}, t1), df_mul(df{h.y, l.y}, t2)));
        s2 = df_add(s2, df_add(df_mul(df{h.z, l.z}, t1), df_mul(df{h.w, l.w}, t2)));
    }
    df e1{__shfl_up_sync(0xffffffffu, s1.hi, 1), __shfl_up_sync(0xffffffffu, s1.lo, 1)};
    df e2{__shfl_up_sync(0xffffffffu, s2.hi, 1), __shfl_up_sync(0xffffffffu, s2.lo, 1)};
    if (lane == 0) {
        e1 = df{0.f, 0.f};
        e2 = df{0.f, 0.f};
    }
    // fold the group's incoming state into this lane's: Phi^lane Z + E
    const df zin1 = df_add(e1, df_add(df_mul(df{lp.x, lpl.x}, Z1), df_mul(df{lp.y, lpl.y}, Z2)));
    const df zin2 = df_add(e2, df_add(df_mul(df{lp.z, lpl.z}, Z1), df_mul(df{lp.w, lpl.w}, Z2)));
    // S4 (iii): the re-run from the true lane state
    df y1{0.f, 0.f}, y2{0.f, 0.f};  // y_{m-1}, y_{m-2}
#pragma unroll
    for (int b = 0; b < N / 4; ++b) {
        const float4 c = lo4[b];
        const float l[4] = {c.x, c.y, c.z, c.w};
        float out[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = 4 * b + i;
            const df u{vh[m], l[i]};
            df y;
            if (m == 0) y = df_add(u, zin1);
            else if (m == 1) y = df_rec1(df_add(u, zin2), q.a1, y1);
            else y = df_rec(u, q.a1, y1, q.a2, y2);
            vh[m] = y.hi;
            out[i] = y.lo;
            y2 = y1;
            y1 = y;
        }
        lo4[b] = make_float4(out[0], out[1], out[2], out[3]);
    }
    // the group's outgoing state, from lane 31's last two inputs and outputs
    const df o1 = df_rec1(df_dot3(q.b1, xl1, q.b2, xl2, na1, y1), q.a2, y2);
    const df o2 = df_rec1(df_mul(q.b2, xl1), q.a2, y1);
    Z1 = df{__shfl_sync(0xffffffffu, o1.hi, 31), __shfl_sync(0xffffffffu, o1.lo, 31)};
    Z2 = df{__shfl_sync(0xffffffffu, o2.hi, 31), __shfl_sync(0xffffffffu, o2.lo, 31)};
    // S8: final state at the channel's last sample
    if (ZF) {
        df yq, yqm1;
        pick_pair<N>(vh, mq, yq.hi, yqm1.hi);
        yq.lo = lo[mq];
        yqm1.lo = mq >= 1 ? lo[mq - 1] : 0.f;
        df f1;
        if (mq >= 1) f1 = df_rec1(df_dot3(q.b1, xq, q.b2, xqm1, na1, yq), q.a2, yqm1);
        else f1 = df_add(df_dot3(q.b1, xq, na1, yq, df{0.f, 0.f}, df{0.f, 0.f}), zin2);
        const df f2 = df_rec1(df_mul(q.b2, xq), q.a2, yq);
        if (zf_owner) {
            zf_dst[0] = df_to_float(f1);
            zf_dst[1] = df_to_float(f2);
        }
    }
}

// The same section solved by cyclic reduction (Sec. VI-C) instead of PH.
// Register m across the 32 lanes is the strided block y_m of Eq.
// cr_permuted_system, and S_R (the shift onto the previous lane) is a
// one-lane shuffle, zero for lane 0: the group's incoming DF2T state enters
// as the corrections to lane 0's v_0 and v_1 (Eq. feedforward_block_uniform).
//   reduction (Eq. cr_elim_step2), level i, s = 2^i, kept blocks m = 2s-1,
//     4s-1, ..: v_m <- v_m - e_i v_{m-s} + f_i v_{m-2s}, and the eliminated
//     block keeps v~_{m-s} = v_{m-s} - g_i v_{m-2s} (g_i = f_i / e_i);
//   terminal block (Eq. cr_terminal_block): Y_l + e_n Y_{l-1} + f_n Y_{l-2}
//     = V_l across lanes, by a 5-round scan;
//   back substitution (Eqs. cr_backsub_penultimate, cr_backsub_final):
//     y_{m-s} = v~_{m-s} - c_i y_{m-2s} - d_i y_{m-4s}, indices below 0
//     taken from the previous lane (S_R) or the one before (S_R^2).
// Sequential depth log2 N per stage instead of N.
template <int N, bool FACT, bool ZF = false>
__device__ __forceinline__ void pipe_section_cr(float (&v)[N], const float4 ab, const float b0,
                                                const float4* cr, float& Z1, float& Z2,
                                                bool zf_owner, int mq, float* s_own,
                                                float* zf_dst, float G) {
    // cr: cr_lv[6], cr_d[2], cr_tpow[5], cr_misc (the Coef32 fields, staged)
    const float4* lv = cr;
    const float* dd = reinterpret_cast<const float*>(cr + 6);
    const float4* tp = cr + 8;
    const int lane = threadIdx.x & 31;
    const float a1 = ab.x, a2 = ab.y, b1 = ab.z, b2 = ab.w;
    const float zi1 = Z1, zi2 = Z2;

    float xq = 0.f, xqm1 = 0.f;
    if (ZF) pick_pair<N>(v, mq, xq, xqm1);

    // S3 with the true history: the previous lane's last two inputs (lane 0's
    // history is inside the group state)
    const float xl1 = v[N - 1], xl2 = v[N - 2];
    float px1 = __shfl_up_sync(0xffffffffu, xl1, 1);
    float px2 = __shfl_up_sync(0xffffffffu, xl2, 1);
    if (lane == 0) {
        px1 = 0.f;
        px2 = 0.f;
    }
#pragma unroll
    for (int m = N - 1; m >= 2; --m)
        v[m] = fmaf(b2, v[m - 2], fmaf(b1, v[m - 1], FACT ? v[m] : b0 * v[m]));
    v[1] = fmaf(b2, px1, fmaf(b1, v[0], FACT ? v[1] : b0 * v[1]));
    v[0] = fmaf(b2, px2, fmaf(b1, px1, FACT ? v[0] : b0 * v[0]));
    if (lane == 0) {
        v[0] += zi1;
        v[1] += zi2;
    }

    // reduction
#pragma unroll
    for (int i = 0; (1 << i) < N; ++i) {
        const int s = 1 << i;
        const float4 q = lv[i];  // e, f, g, c
        float pv = __shfl_up_sync(0xffffffffu, v[N - 1], 1);
        if (lane == 0) pv = 0.f;
#pragma unroll
        for (int m = N - 1; m >= 2 * s - 1; m -= 2 * s) {
            const float vms = v[m - s];
            const float vm2s = m - 2 * s >= 0 ? v[m - 2 * s] : pv;
            v[m] = fmaf(q.y, vm2s, fmaf(-q.x, vms, v[m]));
            v[m - s] = fmaf(-q.z, vm2s, vms);
        }
    }

    // terminal recurrence across lanes: inclusive scan of (Y_l, Y_{l-1})
    float S1 = v[N - 1], S2 = 0.f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        float t1 = __shfl_up_sync(0xffffffffu, S1, d);
        float t2 = __shfl_up_sync(0xffffffffu, S2, d);
        t1 = lane >= d ? t1 : 0.f;
        t2 = lane >= d ? t2 : 0.f;
        S1 = fmaf(tp[j].x, t1, fmaf(tp[j].y, t2, S1));
        S2 = fmaf(tp[j].z, t1, fmaf(tp[j].w, t2, S2));
    }
    v[N - 1] = S1;
    const float Y1 = S2;  // S_R y_{N-1}: the previous lane's (0 for lane 0)
    float Y2 = __shfl_up_sync(0xffffffffu, S2, 1);  // S_R^2 y_{N-1}
    if (lane == 0) Y2 = 0.f;

    // back substitution
    constexpr int kLv = N == 16 ? 4 : N == 32 ? 5 : 6;
#pragma unroll
    for (int ii = 0; ii < kLv; ++ii) {
        const int lvl = kLv - 1 - ii;
        const int s = 1 << lvl;
        const float c = lv[lvl].w, d = dd[lvl];
        float sh4 = Y2;  // S_R y_{N-2s-1}, or S_R^2 y_{N-1} when 2s = N
        if (2 * s + 1 <= N) {
            sh4 = __shfl_up_sync(0xffffffffu, v[(N - 2 * s - 1) >= 0 ? N - 2 * s - 1 : 0], 1);
            if (lane == 0) sh4 = 0.f;
        }
#pragma unroll
        for (int m = 2 * s - 1; m < N; m += 2 * s) {
            const float ym2s = m - 2 * s >= 0 ? v[m - 2 * s >= 0 ? m - 2 * s : 0] : Y1;
            const int q = m - 4 * s;
            const float ym4s = q >= 0 ? v[q >= 0 ? q : 0] : (q == -1 ? Y1 : sh4);
            v[m - s] = fmaf(-d, ym4s, fmaf(-c, ym2s, v[m - s]));
        }
    }

    // the group's outgoing state, from lane 31's last two inputs and outputs
    const float o1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, v[N - 1], -a2 * v[N - 2])));
    const float o2 = fmaf(b2, xl1, -a2 * v[N - 1]);
    Z1 = __shfl_sync(0xffffffffu, o1, 31);
    Z2 = __shfl_sync(0xffffffffu, o2, 31);

    // S8: final state at the channel's last sample
    if (ZF) {
        // DF2T z2 entering this lane: b2 x_{-1} - a2 y_{-1}
        const float zin2 = lane == 0 ? zi2 : fmaf(b2, px1, -a2 * Y1);
        float yq, yqm1;
        pick_pair<N>(v, mq, yq, yqm1);
        float f1;
        if (mq >= 1) f1 = fmaf(b1, xq, fmaf(b2, xqm1, fmaf(-a1, yq, -a2 * yqm1)));
        else f1 = fmaf(b1, xq, fmaf(-a1, yq, zin2));
        const float f2 = fmaf(b2, xq, -a2 * yq);
        if (zf_owner) {
            zf_dst[0] = f1 * G;
            zf_dst[1] = f2 * G;
        }
    }
}

// The adjoint's two runs of one section on the same reversed input g, fused
// so that their recursions interleave (two independent chains per lane): l
// gets the all-pole part (lambda, from state (L1, L2)), u the whole section
// with coefficients (b0, b1, b2) (dL/du, from state (U1, U2)).  Both share
// the poles, hence Phi^(2^j) and Phi^lane.  Same arithmetic as two
// pipe_section calls.
template <int N>
__device__ __forceinline__ void pipe_section_dual(float (&l)[N], float (&u)[N], const float a1,
                                                  const float a2, const float b0, const float b1,
                                                  const float b2, const float4* phi,
                                                  const float4 lp, float& L1, float& L2,
                                                  float& U1, float& U2) {
    const int lane = threadIdx.x & 31;
    // S3 for u (l has no FIR)
    const float xl1 = u[N - 1], xl2 = u[N - 2];
#pragma unroll
    for (int m = N - 1; m >= 2; --m) u[m] = fmaf(b2, u[m - 2], fmaf(b1, u[m - 1], b0 * u[m]));
    u[1] = fmaf(b1, u[0], b0 * u[1]);
    u[0] = b0 * u[0];

    // S4 (i): both particular solutions, interleaved
    float lw0 = l[0], lw1 = fmaf(-a1, lw0, l[1]);
    float uw0 = u[0], uw1 = fmaf(-a1, uw0, u[1]);
#pragma unroll
    for (int m = 2; m < N; ++m) {
        const float lw2 = fmaf(-a1, lw1, fmaf(-a2, lw0, l[m]));
        const float uw2 = fmaf(-a1, uw1, fmaf(-a2, uw0, u[m]));
        lw0 = lw1;
        lw1 = lw2;
        uw0 = uw1;
        uw1 = uw2;
    }
    float LS1 = fmaf(-a1, lw1, -a2 * lw0);
    float LS2 = -a2 * lw1;
    float US1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, uw1, -a2 * uw0)));
    float US2 = fmaf(b2, xl1, -a2 * uw1);

    // S4 (ii): both lane scans
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        float t1 = __shfl_up_sync(0xffffffffu, LS1, d);
        float t2 = __shfl_up_sync(0xffffffffu, LS2, d);
        float t3 = __shfl_up_sync(0xffffffffu, US1, d);
        float t4 = __shfl_up_sync(0xffffffffu, US2, d);
        t1 = lane >= d ? t1 : 0.f;
        t2 = lane >= d ? t2 : 0.f;
        t3 = lane >= d ? t3 : 0.f;
        t4 = lane >= d ? t4 : 0.f;
        const float4 ph = phi[j];
        LS1 = fmaf(ph.x, t1, fmaf(ph.y, t2, LS1));
        LS2 = fmaf(ph.z, t1, fmaf(ph.w, t2, LS2));
        US1 = fmaf(ph.x, t3, fmaf(ph.y, t4, US1));
        US2 = fmaf(ph.z, t3, fmaf(ph.w, t4, US2));
    }
    float LE1 = __shfl_up_sync(0xffffffffu, LS1, 1);
    float LE2 = __shfl_up_sync(0xffffffffu, LS2, 1);
    float UE1 = __shfl_up_sync(0xffffffffu, US1, 1);
    float UE2 = __shfl_up_sync(0xffffffffu, US2, 1);
    if (lane == 0) {
        LE1 = 0.f;
        LE2 = 0.f;
        UE1 = 0.f;
        UE2 = 0.f;
    }
    const float lz1 = fmaf(lp.x, L1, fmaf(lp.y, L2, LE1));
    const float lz2 = fmaf(lp.z, L1, fmaf(lp.w, L2, LE2));
    const float uz1 = fmaf(lp.x, U1, fmaf(lp.y, U2, UE1));
    const float uz2 = fmaf(lp.z, U1, fmaf(lp.w, U2, UE2));

    // S4 (iii): both re-runs, interleaved
    l[0] = l[0] + lz1;
    l[1] = fmaf(-a1, l[0], l[1] + lz2);
    u[0] = u[0] + uz1;
    u[1] = fmaf(-a1, u[0], u[1] + uz2);
#pragma unroll
    for (int m = 2; m < N; ++m) {
        l[m] = fmaf(-a1, l[m - 1], fmaf(-a2, l[m - 2], l[m]));
        u[m] = fmaf(-a1, u[m - 1], fmaf(-a2, u[m - 2], u[m]));
    }

    // the group's outgoing states, from lane 31
    const float lo1 = fmaf(-a1, l[N - 1], -a2 * l[N - 2]);
    const float lo2 = -a2 * l[N - 1];
    const float uo1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, u[N - 1], -a2 * u[N - 2])));
    const float uo2 = fmaf(b2, xl1, -a2 * u[N - 1]);
    L1 = __shfl_sync(0xffffffffu, lo1, 31);
    L2 = __shfl_sync(0xffffffffu, lo2, 31);
    U1 = __shfl_sync(0xffffffffu, uo1, 31);
    U2 = __shfl_sync(0xffffffffu, uo2, 31);
}


}  // namespace sosf
