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

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The look-back words of one section.
struct Words {
    unsigned long long* w;  // words of section k: w[word * cap + tile]
    int64_t cap;
    __device__ __forceinline__ unsigned long long* at(int word, int64_t tile) const {
        return w + word * cap + tile;
    }
};

__device__ __forceinline__ Words section_words(const Params& p, int k) {
    return Words{p.words + (int64_t)k * kWords * p.cap_tiles, p.cap_tiles};
}

__device__ __forceinline__ bool read_inc(const Words& W, int64_t t, uint32_t tag, df& z1, df& z2) {
    const unsigned long long w0 = ld_relaxed_u64(W.at(0, t)), w1 = ld_relaxed_u64(W.at(1, t));
    const unsigned long long w2 = ld_relaxed_u64(W.at(2, t)), w3 = ld_relaxed_u64(W.at(3, t));
    z1 = df{word_value(w0), word_value(w1)};
    z2 = df{word_value(w2), word_value(w3)};
    return word_has(w0, tag) && word_has(w1, tag) && word_has(w2, tag) && word_has(w3, tag);
}

__device__ __forceinline__ bool read_agg(const Words& W, int64_t t, uint32_t tag, float& c1,
                                         float& c2) {
    const unsigned long long w0 = ld_relaxed_u64(W.at(4, t)), w1 = ld_relaxed_u64(W.at(5, t));
    c1 = word_value(w0);
    c2 = word_value(w1);
    return word_has(w0, tag) && word_has(w1, tag);
}

__device__ __forceinline__ void write_inc(const Words& W, int64_t t, uint32_t tag, df z1, df z2) {
    st_relaxed_u64(W.at(0, t), tag_word(z1.hi, tag));
    st_relaxed_u64(W.at(1, t), tag_word(z1.lo, tag));
    st_relaxed_u64(W.at(2, t), tag_word(z2.hi, tag));
    st_relaxed_u64(W.at(3, t), tag_word(z2.lo, tag));
}

__device__ __forceinline__ void write_agg(const Words& W, int64_t t, uint32_t tag, float c1,
                                          float c2) {
    st_relaxed_u64(W.at(4, t), tag_word(c1, tag));
    st_relaxed_u64(W.at(5, t), tag_word(c2, tag));
}

__device__ __forceinline__ df shfl_df0(df v) {
    return df{__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0)};
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

// Incoming state of tile t (global index), section k, which has `npred` >= 1
// predecessors in its channel.  Run by one full warp (uniform control flow);
// every lane returns the same value.
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
// The nearest predecessor is read first (one broadcast read; usually its
// inclusive value is there).  Otherwise the warp reads a window of up to 128
// predecessors, lane l taking 32 j + l for j = 0..3 (coalesced, the words
// are stored structure-of-arrays), folds its own terms with Theta^32 and the
// warp sums Theta^l times them.  A full window without an inclusive value is
// folded with Theta^128 and the walk continues.  All in double-float.
template <bool REV>
__device__ void lookback_warp(const Params& p, int64_t t, int64_t npred, int k, uint32_t epoch,
                              const CoefDF* cd, df& Z1, df& Z2) {
    constexpr int R = 4, WIN = 32 * R;
    const int lane = threadIdx.x & 31;
    const uint32_t tag_inc = (epoch << 2) | kFlagInc, tag_agg = (epoch << 2) | kFlagAgg;
    const Words Wd = section_words(p, k);
    {
        df z1, z2;
        const bool ok = read_inc(Wd, REV ? t + 1 : t - 1, tag_inc, z1, z2);  // same address in all lanes
        if (__all_sync(0xffffffffu, ok)) {
            Z1 = z1;
            Z2 = z2;
            return;
        }
    }
    df acc1 = df{0.f, 0.f}, acc2 = df{0.f, 0.f};
    dfm2 M = dfm_identity();
    bool first_window = true;
    int64_t base = REV ? t + 1 : t - 1;
    int64_t remaining = npred;
    uint32_t spins = 0;
    const uint32_t limit = wait_limit(p.hdr, kSpinLimit);
    for (;;) {
        const int cnt = (int)(remaining < WIN ? remaining : WIN);
        df i1[R], i2[R];
        float c1[R], c2[R];
        uint32_t incm[R], readym[R];
        for (;;) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int g = 32 * j + lane;
                const int64_t tj = REV ? base + g : base - g;
                bool isinc = false, isagg = false;
                i1[j] = df{0.f, 0.f};
                i2[j] = df{0.f, 0.f};
                c1[j] = 0.f;
                c2[j] = 0.f;
                if (g < cnt) {
                    isinc = read_inc(Wd, tj, tag_inc, i1[j], i2[j]);
                    isagg = read_agg(Wd, tj, tag_agg, c1[j], c2[j]);
                }
                incm[j] = __ballot_sync(0xffffffffu, isinc);
                readym[j] = __ballot_sync(0xffffffffu, isinc || isagg);
            }
            int fstar = WIN;
#pragma unroll
            for (int j = R - 1; j >= 0; --j)
                if (incm[j]) fstar = 32 * j + (__ffs(incm[j]) - 1);
            const int need = fstar < WIN ? fstar : cnt;
            bool ok = fstar < cnt || (cnt == WIN && remaining > WIN);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int nl = need - 32 * j;
                if (nl > 0) {
                    const uint32_t m = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
                    if ((readym[j] & m) != m) ok = false;
                }
            }
            if (ok) {
                // this window: sum_{g <= fstar} Theta^g v_g, g = 32 j + lane
                const int last = fstar < WIN ? fstar : cnt - 1;
                df u1 = df{0.f, 0.f}, u2 = df{0.f, 0.f};
                const dfm2 T32 = load_theta<REV>(cd, 32);
#pragma unroll
                for (int j = R - 1; j >= 0; --j) {
                    const int g = 32 * j + lane;
                    df v1 = df{0.f, 0.f}, v2 = df{0.f, 0.f};
                    if (g < fstar) {
                        v1 = df_from(c1[j]);
                        v2 = df_from(c2[j]);
                    } else if (g == fstar) {
                        v1 = i1[j];
                        v2 = i2[j];
                    }
                    if (32 * j <= last) {  // warp-uniform: Horner in Theta^32 over j
                        if (32 * (j + 1) <= last) {
                            df n1, n2;
                            dfm_affine_fast(T32, u1, u2, v1, v2, n1, n2);
                            u1 = n1;
                            u2 = n2;
                        } else {
                            u1 = v1;
                            u2 = v2;
                        }
                    }
                }
                df s1, s2;
                if (last == 0) {
                    s1 = shfl_df0(u1);
                    s2 = shfl_df0(u2);
                } else {
                    dfm_affine_fast(load_theta<REV>(cd, lane), u1, u2, df{0.f, 0.f}, df{0.f, 0.f}, s1,
                                    s2);
                    const int hi = last < 32 ? last : 31;  // highest lane holding a term
#pragma unroll
                    for (int m = 16; m >= 1; m >>= 1) {
                        if (m <= hi) {
                            s1 = df_add_fast(s1, shfl_xor_df(s1, m));
                            s2 = df_add_fast(s2, shfl_xor_df(s2, m));
                        }
                    }
                    // with rounds skipped only lane 0 is sure to hold the
                    // whole sum: every lane takes its value
                    s1 = shfl_df0(s1);
                    s2 = shfl_df0(s2);
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
                if (fstar < WIN) {
                    Z1 = acc1;
                    Z2 = acc2;
                    return;
                }
                M = first_window ? load_theta_hi<REV>(cd, R) : dfm_mul(M, load_theta_hi<REV>(cd, R));
                first_window = false;
                break;  // continue WIN tiles further back
            }
            ++spins;
            if (spins > limit) {
                if (lane == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
                Z1 = acc1;
                Z2 = acc2;
                return;
            }
            if ((spins & 63u) == 0u && ld_volatile_i32(&p.hdr->status) != 0) {
                Z1 = acc1;
                Z2 = acc2;
                return;
            }
            __nanosleep(32);
        }
        base = REV ? base + WIN : base - WIN;
        remaining -= WIN;
    }
}

}  // namespace sosf
