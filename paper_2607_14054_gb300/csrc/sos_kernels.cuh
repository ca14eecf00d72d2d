// Device helpers shared by the forward and adjoint kernels: the swizzled
// shared-memory tile layout, the tagged look-back slots and the decoupled
// look-back itself.
#pragma once

#include "sos_common.cuh"

namespace sosf {

template <int N>
struct Swz {
    // 16-byte granule index within the tile -> physical granule.  A lane's
    // chunk is N/4 granules; XOR with the chunk index (mod 8) makes both the
    // row-wise (global <-> shared) and the chunk-wise (shared <-> registers)
    // 128-bit accesses bank-conflict free.
    static constexpr int kShift = (N == 16) ? 2 : (N == 32) ? 3 : 4;
    __device__ __forceinline__ static int g(int G) { return G ^ ((G >> kShift) & 7); }
    __device__ __forceinline__ static int e(int j) { return (g(j >> 2) << 2) | (j & 3); }
};

// Theta^d (TR: its transpose, the adjoint's transition)
template <bool TR = false>
__device__ __forceinline__ dfm2 load_theta(const CoefDF* cd, int d) {
    const float4 r0 = cd->theta_pow[d][0];
    const float4 r1 = cd->theta_pow[d][1];
    if (TR) return dfm2{df{r0.x, r0.y}, df{r1.x, r1.y}, df{r0.z, r0.w}, df{r1.z, r1.w}};
    return dfm2{df{r0.x, r0.y}, df{r0.z, r0.w}, df{r1.x, r1.y}, df{r1.z, r1.w}};
}

// Reads the inclusive half of a slot; true if all four words carry `tag`.
__device__ __forceinline__ bool read_inc(const Slot& sl, uint32_t tag, df& z1, df& z2) {
    unsigned long long w0, w1, w2, w3;
    ld_relaxed_v2u64(sl.inc, w0, w1);
    ld_relaxed_v2u64(sl.inc + 2, w2, w3);
    z1 = df{word_value(w0), word_value(w1)};
    z2 = df{word_value(w2), word_value(w3)};
    return word_has(w0, tag) && word_has(w1, tag) && word_has(w2, tag) && word_has(w3, tag);
}

__device__ __forceinline__ bool read_agg(const Slot& sl, uint32_t tag, float& c1, float& c2) {
    unsigned long long w0, w1;
    ld_relaxed_v2u64(sl.agg, w0, w1);
    c1 = word_value(w0);
    c2 = word_value(w1);
    return word_has(w0, tag) && word_has(w1, tag);
}

__device__ __forceinline__ void write_inc(Slot& sl, uint32_t tag, df z1, df z2) {
    st_relaxed_v2u64(sl.inc, tag_word(z1.hi, tag), tag_word(z1.lo, tag));
    st_relaxed_v2u64(sl.inc + 2, tag_word(z2.hi, tag), tag_word(z2.lo, tag));
}

__device__ __forceinline__ void write_agg(Slot& sl, uint32_t tag, float c1, float c2) {
    st_relaxed_v2u64(sl.agg, tag_word(c1, tag), tag_word(c2, tag));
}

__device__ __forceinline__ df shfl_xor_df(df v, int m) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// Theta^(32 j) (TR: transposed)
template <bool TR = false>
__device__ __forceinline__ dfm2 load_theta_hi(const CoefDF* cd, int j) {
    const float4 r0 = cd->theta_hi[j][0];
    const float4 r1 = cd->theta_hi[j][1];
    if (TR) return dfm2{df{r0.x, r0.y}, df{r1.x, r1.y}, df{r0.z, r0.w}, df{r1.z, r1.w}};
    return dfm2{df{r0.x, r0.y}, df{r0.z, r0.w}, df{r1.x, r1.y}, df{r1.z, r1.w}};
}

// Shared scratch of the cooperative look-back (NW warps).
template <int NW>
struct LookbackShared {
    uint32_t first[NW];  // per warp: first lane holding an inclusive value, 32 if none
    uint32_t ready[NW];  // per warp: lanes whose slot is published (either kind)
    float4 part[NW];     // per warp: its partial sum (z1.hi, z1.lo, z2.hi, z2.lo)
};

// Incoming state of tile t (global index), section k, which has `npred` >= 1
// predecessors in its channel.  Called by all NW warps of the CTA (uniform
// control flow); the result is returned in (Z1, Z2) of warp `cw` (the
// coordinator), other warps get zeros.
//
// Forward (REV = false): predecessors are t-1, t-2, ... and the state is the
// DF2T state entering the tile.  Adjoint (REV = true): predecessors are t+1,
// t+2, ... (time runs backwards), the state is the adjoint state entering the
// tile from its end, and every transition matrix is transposed.
//
// Predecessor tiles publish their aggregate c (zero-state outgoing state)
// and, once known, their inclusive value P (true outgoing state).  With f the
// nearest predecessor holding an inclusive value, the incoming state is
//     Z = sum_{i<f} Theta^i c_i + Theta^f P_f       (i = 0: the nearest).
// All NW*32 threads read one predecessor each, so a window of NW*32 tiles is
// examined per L2 round trip (the tiles resident on the GPU tend to reach a
// section together, so a narrow window would let the known prefix advance
// only a few tiles per round trip).  Lane l of warp w forms Theta^l v for
// predecessor 32 w + l; each warp sums its terms, and the coordinator applies
// Theta^(32 w) to warp w's sum.  A full window without an inclusive value is
// folded with Theta^(32 NW) and the walk continues.  All in double-float.
template <bool REV, int NW>
__device__ void lookback_cta(const Params& p, int64_t t, int64_t npred, int k, uint32_t epoch,
                             const CoefDF* cd, LookbackShared<NW>* lb, int cw, df& Z1, df& Z2) {
    constexpr int WIN = NW * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t tag_inc = (epoch << 2) | kFlagInc, tag_agg = (epoch << 2) | kFlagAgg;
    const Slot* sl = p.slots + (int64_t)k * p.cap_tiles;
    const int g = warp * 32 + lane;  // this thread's predecessor distance - 1
    df acc1 = df{0.f, 0.f}, acc2 = df{0.f, 0.f};  // meaningful in warp cw
    dfm2 M = dfm_identity();
    bool first_window = true;
    int64_t base = REV ? t + 1 : t - 1;
    int64_t remaining = npred;
    uint32_t spins = 0;
    for (;;) {
        const int cnt = (int)(remaining < WIN ? remaining : WIN);
        const bool valid = g < cnt;
        const int64_t j = REV ? base + g : base - g;
        df i1 = df{0.f, 0.f}, i2 = df{0.f, 0.f};
        float a1 = 0.f, a2 = 0.f;
        bool isinc = false, isagg = false;
        if (valid) {
            isinc = read_inc(sl[j], tag_inc, i1, i2);
            if (!isinc) isagg = read_agg(sl[j], tag_agg, a1, a2);
        }
        const uint32_t incm = __ballot_sync(0xffffffffu, isinc);
        const uint32_t readym = __ballot_sync(0xffffffffu, isinc || isagg);
        if (lane == 0) {
            lb->first[warp] = incm ? (uint32_t)(__ffs(incm) - 1) : 32u;
            lb->ready[warp] = readym;
        }
        __syncthreads();
        // the same decision in every thread
        int fstar = WIN;
        for (int w = 0; w < NW; ++w) {
            const uint32_t f = lb->first[w];
            if (f < 32) {
                fstar = w * 32 + (int)f;
                break;
            }
        }
        const int need = fstar < WIN ? fstar : cnt;  // predecessors that must hold an aggregate
        bool ok = fstar < cnt || (cnt == WIN && remaining > WIN);
        for (int w = 0; w < NW && ok; ++w) {
            const int nl = need - 32 * w;
            if (nl <= 0) break;
            const uint32_t m = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
            if ((lb->ready[w] & m) != m) ok = false;
        }
        if (!ok) {
            ++spins;
            const bool give_up = spins > kSpinLimit || ((spins & 63u) == 0u &&
                                                        ld_volatile_i32(&p.hdr->status) != 0);
            if (give_up && spins > kSpinLimit && threadIdx.x == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
            __syncthreads();  // everyone has read first/ready before they are rewritten
            if (give_up) break;
            __nanosleep(32);
            continue;
        }
        // this window's contribution: sum_{g <= fstar} Theta^g v_g
        df v1 = df{0.f, 0.f}, v2 = df{0.f, 0.f};
        if (g < fstar) {
            v1 = df_from(a1);
            v2 = df_from(a2);
        } else if (g == fstar) {
            v1 = i1;
            v2 = i2;
        }
        df u1 = df{0.f, 0.f}, u2 = df{0.f, 0.f};
        const int last = (fstar < WIN ? fstar : cnt - 1) - warp * 32;  // highest contributing lane
        if (last >= 0) {                                               // warp-uniform
            if (lane <= last)
                dfm_affine_fast(load_theta<REV>(cd, lane), v1, v2, df{0.f, 0.f}, df{0.f, 0.f}, u1,
                                u2);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                if (m <= last) {  // lanes above `last` hold zeros
                    u1 = df_add_fast(u1, shfl_xor_df(u1, m));
                    u2 = df_add_fast(u2, shfl_xor_df(u2, m));
                }
            }
        }
        if (lane == 0) lb->part[warp] = make_float4(u1.hi, u1.lo, u2.hi, u2.lo);
        __syncthreads();
        if (warp == cw) {
            df s1, s2;
            const int nparts = ((fstar < WIN ? fstar : cnt - 1) >> 5) + 1;  // warps that contributed
            if (nparts == 1) {
                const float4 q = lb->part[0];  // Theta^(32*0) = I
                s1 = df{q.x, q.y};
                s2 = df{q.z, q.w};
            } else {
                s1 = df{0.f, 0.f};
                s2 = df{0.f, 0.f};
                if (lane < nparts) {
                    const float4 q = lb->part[lane];
                    dfm_affine_fast(load_theta_hi<REV>(cd, lane), df{q.x, q.y}, df{q.z, q.w},
                                    df{0.f, 0.f}, df{0.f, 0.f}, s1, s2);
                }
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1) {
                    if (m < nparts) {
                        s1 = df_add_fast(s1, shfl_xor_df(s1, m));
                        s2 = df_add_fast(s2, shfl_xor_df(s2, m));
                    }
                }
            }
            if (first_window) {
                acc1 = s1;
                acc2 = s2;
            } else {
                df n1, n2;
                dfm_affine(M, s1, s2, acc1, acc2, n1, n2);  // acc + M * sum
                acc1 = n1;
                acc2 = n2;
            }
            if (fstar >= WIN) M = first_window ? load_theta_hi<REV>(cd, NW)
                                               : dfm_mul(M, load_theta_hi<REV>(cd, NW));
        }
        first_window = false;
        if (fstar < WIN) break;
        // a full window of aggregates: continue NW*32 tiles further back
        base = REV ? base + WIN : base - WIN;
        remaining -= WIN;
    }
    Z1 = acc1;
    Z2 = acc2;
}

}  // namespace sosf
