// Forward cascade kernel for sm_103a: stride-N multi-block filtering with the
// PH recursive-stage solver, all K sections fused per tile, and a decoupled
// look-back that carries each section's DF2T state between tiles.
//
// Work decomposition (one persistent CTA of W warps processes one tile of
// T = W * 32 * N samples at a time, tiles handed out in order by an atomic
// counter):
//
//  S2  load: coalesced global loads into a swizzled shared-memory tile, then
//      lane l of warp w reads its contiguous chunk into N registers.  This is
//      the stride-N permutation of Sec. VII-A: register m across the 32
//      lanes is the strided block x_m of Sec. V.
//  per section k (the permutations between sections cancel, Sec. VII-B):
//  S3  non-recursive stage, Eq. feedforward_block_uniform:
//      v_m = x_m + b1 x_{m-1} + b2 x_{m-2} with zero history inside the lane;
//      the history enters later through the DF2T state (z1, z2), which is
//      exactly the paper's pair of scalar corrections to v_0 and v_1.
//  S4  PH recursive stage, Sec. VI-B:
//      (i)   particular solution P w = v (Eq. particular_recurrence) in each
//            lane from zero state, kept only for its two terminal values,
//            which give the lane's zero-state outgoing state s_l;
//      (ii)  terminal-block solve: the lane states obey
//            z_{l+1} = Phi z_l + s_l, a first-order 2x2 recurrence across the
//            32 lanes (the scan of Eq. recursive_doubling_equation, here on
//            DF2T states), solved by a 5-round warp-shuffle scan with the
//            FP64-derived powers Phi^(2^j);
//      (iii) homogeneous correction: each lane re-runs
//            y_m = v_m - a1 y_{m-1} - a2 y_{m-2} from its true incoming state
//            (2 FMAs per sample, like Eq. PH_forward, without a table).
//  S5  cross-warp (shared memory, scan with Psi^(2^r)) and cross-tile
//      (decoupled look-back over FP64 affine maps z -> Theta z + c, the GPU
//      form of the inter-group hand-off of Sec. V) carry of the state.  A
//      channel whose impulse response dies out within half a tile (its
//      memory horizon P, computed by the plan) needs no carry: its tiles
//      overlap by P samples and start from zero state;
//  S7  de-permutation through shared memory and coalesced stores;
//  S8  the lane holding a channel's last sample writes zf.
#include <cmath>

#include "sos_async.cuh"
#include "sos_kernels.cuh"

namespace sosf {

template <int N, int W>
struct FwdKernel {
    static constexpr int kDataThreads = W * 32;
    static constexpr int kThreads = (W + 1) * 32;  // W data warps + 1 coordinator warp
    static constexpr int kTile = W * 32 * N;
    static constexpr int kGran = kTile / 4;
    static constexpr size_t kSmem = 2 * sizeof(float) * kTile;  // two tile buffers
};

// Where a dispatched tile lies.  Tiles of a channel with memory horizon
// P >= 0 overlap by P samples: tile 0 covers [0, T) from zi, tile ti > 0
// computes [T + (ti - 1)(T - P) - P, ...) from zero state and stores all but
// its first P samples.  Other channels' tiles abut and carry the state.
struct TileGeom {
    int64_t ti, t, nt, start;  // index in channel, look-back slot, channel tiles, first sample
    const float* src;          // x of the first sample
    int c, r, skip;            // channel, valid samples, overlap samples not stored
    bool carry;
};

template <int kTile>
__device__ __forceinline__ TileGeom tile_geom(const Params& p, int64_t d, int64_t nrounds) {
    int c;
    int64_t ti;
    if (nrounds > 0) {
        // interleaved: round r = the largest with rp[r] <= d, then the
        // (d - rp[r])-th channel of the sorted order
        int64_t lo = 0, hi = nrounds - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.rp[mid]) <= d) lo = mid; else hi = mid - 1;
        }
        ti = lo;
        c = __ldg(&p.order[d - __ldg(&p.rp[lo])]);
    } else {
        // channel by channel: the largest c with tb[c] <= d
        int lo = 0, hi = p.C - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.tb[mid]) <= d) lo = mid; else hi = mid - 1;
        }
        c = lo;
        ti = d - __ldg(&p.tb[c]);
    }
    const ChanInfo ci = p.chan[c];
    TileGeom g;
    g.c = c;
    g.ti = ti;
    g.t = ci.slot + ti;
    g.nt = ci.ntiles;
    g.carry = ci.horizon < 0;
    g.skip = (!g.carry && ti > 0) ? ci.horizon : 0;
    g.start = g.skip ? kTile + (ti - 1) * (kTile - g.skip) - g.skip : ti * kTile;
    const int64_t rem = ci.len - g.start;
    g.r = (int)(rem < kTile ? rem : kTile);
    g.src = p.x + ci.off + g.start;
    return g;
}


// S2, issued one tile ahead: global -> shared (swizzled) by asynchronous
// copies, zero beyond the channel end; all W + 1 warps take part.
template <int N, int W>
__device__ __forceinline__ void issue_tile_load(const TileGeom& g, float4* buf4, int tid) {
    using KT = FwdKernel<N, W>;
    using S = Swz<N>;
    const bool vec = ((reinterpret_cast<uintptr_t>(g.src) & 15u) == 0) && g.r == KT::kTile;
    if (vec) {
        const float4* s4 = reinterpret_cast<const float4*>(g.src);
#pragma unroll 4
        for (int q = tid; q < KT::kGran; q += KT::kThreads) cp_async16(buf4 + S::g(q), s4 + q);
    } else {
        float* buf = reinterpret_cast<float*>(buf4);
        for (int j = tid; j < KT::kTile; j += KT::kThreads)
            cp_async4(buf + S::e(j), j < g.r ? g.src + j : g.src, j < g.r);
    }
}

// Per-section shared state between the data warps and the coordinator.
template <int W>
struct SectionShared {
    float2 agg[W];  // zero-state state leaving each warp's group
    float2 win[W];  // true state entering each warp's group
};

// Hand-off between consecutive data warps (tiles within a channel's memory
// horizon): the true state leaving warp w's group in section k, passed to
// warp w + 1 through shared memory and an mbarrier of arrival count 1.  The
// producer's arrive releases the value, the consumer's try_wait acquires it;
// a waiting warp is suspended by the hardware instead of polling, so it takes
// no issue slots from the warps it waits for.  Each barrier completes one
// phase per use; every data warp keeps the parity of section k's barriers in
// bit k of its own phase mask (all warps of a tile process the same sections).
template <int W>
struct HandOff {
    float2 val[kMaxSections][W];
    unsigned long long bar[kMaxSections][W];
    uint32_t limit;  // bound on each hand-off wait (polls), read once per launch
};


// One section of the cascade on a data warp's register-resident chunk.
// CHAIN = false: the warp's incoming state comes from the coordinator warp
// (CTA barriers B1/B2, cross-tile look-back).  CHAIN = true (tile within the
// channel's memory horizon, no cross-tile carry): warp 0 starts from the
// tile's own initial state and every other warp waits only for its
// predecessor's hand-off, z_out(w) = Psi z_in(w) + agg(w).
template <int N, int W, bool FACT, bool CHAIN>
__device__ __forceinline__ void data_section(const Params& p, float (&v)[N], int k, int c,
                                             int64_t t, int64_t ti, uint32_t epoch,
                                             const Coef32* cf, const CoefDF* cd,
                                             SectionShared<W>* sh, bool zf_owner, int mq,
                                             float* s_own, HandOff<W>* ho, uint32_t& ph) {
    // position of this data warp's group in the tile (warp 0 of the CTA is
    // the coordinator; CTA warp j holds group W - j, so that the groups the
    // in-tile carry reaches last belong to the oldest warps, which the warp
    // schedulers favour)
    const int lane = threadIdx.x & 31, warp = W - (int)(threadIdx.x >> 5);
    const float4 ab = cf->ab;
    const float a1 = ab.x, a2 = ab.y, b1 = ab.z, b2 = ab.w;
    const float b0 = FACT ? 1.0f : cf->misc.x;
    // (CHAIN) the tile's initial state, needed by warp 0 only: zi / G_k on a
    // channel's first tile, zero state on the others
    float zt1 = 0.f, zt2 = 0.f;
    if (CHAIN && warp == 0 && ti == 0 && p.zi) {
        const float gi = cf->misc.z;
        zt1 = p.zi[((int64_t)c * p.kmax + k) * 2 + 0] * gi;
        zt2 = p.zi[((int64_t)c * p.kmax + k) * 2 + 1] * gi;
    }

    // the section input at the channel's last sample (S8): the owning lane
    // parks its chunk in its own slice of the (idle) tile buffer so that the
    // sample can be picked with a run-time index
    float xq = 0.f, xqm1 = 0.f;
    __syncwarp();  // (N = 16) the owner's slice overlaps a neighbour lane's swizzled chunk
    if (zf_owner) {
#pragma unroll
        for (int m = 0; m < N; ++m) s_own[m] = v[m];
        xq = s_own[mq];
        xqm1 = mq >= 1 ? s_own[mq - 1] : 0.f;
    }

    // S3: non-recursive stage with zero history inside the lane
    const float xl1 = v[N - 1], xl2 = v[N - 2];
#pragma unroll
    for (int m = N - 1; m >= 2; --m)
        v[m] = fmaf(b2, v[m - 2], fmaf(b1, v[m - 1], FACT ? v[m] : b0 * v[m]));
    v[1] = fmaf(b1, v[0], FACT ? v[1] : b0 * v[1]);
    if (!FACT) v[0] = b0 * v[0];

    // S4 (i): particular solution from zero state, terminal values only
    float w0 = v[0], w1 = fmaf(-a1, w0, v[1]);
#pragma unroll
    for (int m = 2; m < N; ++m) {
        const float w2 = fmaf(-a1, w1, fmaf(-a2, w0, v[m]));
        w0 = w1;
        w1 = w2;
    }
    // zero-state DF2T state after the lane chunk
    float S1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, w1, -a2 * w0)));
    float S2 = fmaf(b2, xl1, -a2 * w1);

    // S4 (ii): inclusive scan over lanes, z_{l+1} = Phi z_l + s_l
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int d = 1 << j;
        const float t1 = __shfl_up_sync(0xffffffffu, S1, d);
        const float t2 = __shfl_up_sync(0xffffffffu, S2, d);
        const float4 P = cf->phi_pow[j];
        if (lane >= d) {
            S1 = fmaf(P.x, t1, fmaf(P.y, t2, S1));
            S2 = fmaf(P.z, t1, fmaf(P.w, t2, S2));
        }
    }
    float E1 = __shfl_up_sync(0xffffffffu, S1, 1);
    float E2 = __shfl_up_sync(0xffffffffu, S2, 1);
    if (lane == 0) {
        E1 = 0.f;
        E2 = 0.f;
    }
    float2 Zw;
    if (!CHAIN) {
        if (lane == 31) sh->agg[warp] = make_float2(S1, S2);
        __syncthreads();  // B1: warp aggregates ready for the coordinator
        __syncthreads();  // B2: the coordinator has placed this warp's incoming state
        Zw = sh->win[warp];
    } else {
        // The whole warp waits and the publication is predicated inside one
        // asm block: a branch taken by one lane would leave the warp diverged
        // into the shuffles that follow, which then run several times slower.
        float q1 = zt1, q2 = zt2;
        const unsigned par = (ph >> k) & 1u;
        ph ^= 1u << k;
        if (warp > 0) {
            // bounded wait for the predecessor warp's hand-off
            unsigned long long* b = &ho->bar[k][warp - 1];
            const uint32_t limit = ho->limit;
            for (uint32_t it = 0;; ++it) {
                const bool ok = mbar_try_wait(b, par);
                if (__all_sync(0xffffffffu, ok)) break;
                if (it >= limit) {
                    if (lane == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
                    break;
                }
            }
            const float2 z = ho->val[k][warp - 1];
            q1 = z.x;
            q2 = z.y;
        }
        if (warp < W - 1) {
            // z_out = Psi z_in + agg; the inclusive scan of lane 31 is agg
            const float4 Ps = cf->psi_pow[0];
            const float o1 = fmaf(Ps.x, q1, fmaf(Ps.y, q2, S1));
            const float o2 = fmaf(Ps.z, q1, fmaf(Ps.w, q2, S2));
            mbar_publish(&ho->val[k][warp], o1, o2, &ho->bar[k][warp], lane == 31);
        }
        Zw = make_float2(q1, q2);
    }

    // fold the warp's true incoming state into this lane's
    const float4 Pl = cf->lane_pow[lane];
    const float zin1 = fmaf(Pl.x, Zw.x, fmaf(Pl.y, Zw.y, E1));
    const float zin2 = fmaf(Pl.z, Zw.x, fmaf(Pl.w, Zw.y, E2));

    // S4 (iii): re-run the recursion from the true incoming state
    v[0] = v[0] + zin1;
    v[1] = fmaf(-a1, v[0], v[1] + zin2);
#pragma unroll
    for (int m = 2; m < N; ++m) v[m] = fmaf(-a1, v[m - 1], fmaf(-a2, v[m - 2], v[m]));

    // S8: final state at the channel's last sample
    if (zf_owner) {
#pragma unroll
        for (int m = 0; m < N; ++m) s_own[m] = v[m];
        const float yq = s_own[mq];
        const float yqm1 = mq >= 1 ? s_own[mq - 1] : 0.f;
        float f1;
        if (mq >= 1) {
            f1 = fmaf(b1, xq, fmaf(b2, xqm1, fmaf(-a1, yq, -a2 * yqm1)));
        } else {
            f1 = fmaf(b1, xq, fmaf(-a1, yq, zin2));
        }
        const float f2 = fmaf(b2, xq, -a2 * yq);
        const float G = FACT ? cf->misc.y : 1.0f;
        p.zf[((int64_t)c * p.kmax + k) * 2 + 0] = f1 * G;
        p.zf[((int64_t)c * p.kmax + k) * 2 + 1] = f2 * G;
    }
}

// The coordinator warp's part of one section (S5): scan over the W warp
// aggregates, publication of the tile's aggregate, the look-back (with the
// data warps' help) for the tile's incoming state, publication of its
// outgoing state, and each warp's incoming state.
template <int W>
__device__ __forceinline__ void coord_section(const Params& p, int k, int c, int64_t t, int64_t ti,
                                              int64_t nt, bool carry, uint32_t epoch,
                                              const Coef32* cf, const CoefDF* cd,
                                              SectionShared<W>* sh) {
    const int lane = threadIdx.x & 31;
    // everything this section needs, read while the data warps compute
    float4 Pr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) Pr[r] = cf->psi_pow[r];
    const float4 misc = cf->misc;
    const float4 Pw = cf->psi_w[lane < 16 ? lane : 0];
    const dfm2 Th = load_theta(cd, 1);
    float zi1 = 0.f, zi2 = 0.f;
    if (ti == 0 && p.zi) {
        zi1 = p.zi[((int64_t)c * p.kmax + k) * 2 + 0];
        zi2 = p.zi[((int64_t)c * p.kmax + k) * 2 + 1];
    }
    __syncthreads();  // B1
    float A1 = 0.f, A2 = 0.f;
    if (lane < W) {
        const float2 a = sh->agg[lane];
        A1 = a.x;
        A2 = a.y;
    }
#pragma unroll
    for (int r = 0; (1 << r) < W; ++r) {
        const int d = 1 << r;
        const float t1 = __shfl_up_sync(0xffffffffu, A1, d);
        const float t2 = __shfl_up_sync(0xffffffffu, A2, d);
        if (lane >= d && lane < W) {
            A1 = fmaf(Pr[r].x, t1, fmaf(Pr[r].y, t2, A1));
            A2 = fmaf(Pr[r].z, t1, fmaf(Pr[r].w, t2, A2));
        }
    }
    float WE1 = __shfl_up_sync(0xffffffffu, A1, 1);
    float WE2 = __shfl_up_sync(0xffffffffu, A2, 1);
    if (lane == 0) {
        WE1 = 0.f;
        WE2 = 0.f;
    }
    const float C1 = __shfl_sync(0xffffffffu, A1, W - 1);
    const float C2 = __shfl_sync(0xffffffffu, A2, W - 1);
    const bool has_succ = carry && ti + 1 < nt;
    const Words Wd = section_words(p, k);
    df Z1, Z2;
    if (ti == 0) {
        // zi / G_k, the exact product split into hi + lo
        const float gi = misc.z;
        const float q1 = zi1 * gi, q2 = zi2 * gi;
        Z1 = df{q1, fmaf(zi1, gi, -q1)};
        Z2 = df{q2, fmaf(zi2, gi, -q2)};
    } else if (!carry) {
        // within the channel's memory horizon: the tile started early enough
        // for zero state to be exact to far below FP32 rounding
        Z1 = df{0.f, 0.f};
        Z2 = df{0.f, 0.f};
    } else {
        if (has_succ && lane == 0) write_agg(Wd, t, (epoch << 2) | kFlagAgg, C1, C2);
        lookback_warp<false>(p, t, ti, k, epoch, cd, Z1, Z2);
    }
    if (has_succ && lane == 0) {
        df P1, P2;
        dfm_affine(Th, Z1, Z2, df_from(C1), df_from(C2), P1, P2);
        write_inc(Wd, t, (epoch << 2) | kFlagInc, P1, P2);
    }
    if (lane < W) {
        const float z1 = df_to_float(Z1), z2 = df_to_float(Z2);
        sh->win[lane] = make_float2(fmaf(Pw.x, z1, fmaf(Pw.y, z2, WE1)),
                                    fmaf(Pw.z, z1, fmaf(Pw.w, z2, WE2)));
    }
    __syncthreads();  // B2
}

template <int N, int W, int MINB>
__global__ void __launch_bounds__((W + 1) * 32, MINB) sos_forward_kernel(Params p) {
    using KT = FwdKernel<N, W>;
    using S = Swz<N>;
    extern __shared__ float4 s_tile4[];
    __shared__ SectionShared<W> sh;
    __shared__ HandOff<W> ho;
    __shared__ int64_t s_t;
    // the current channel's coefficient tables, staged once per channel
    __shared__ Coef32 s_c32[kMaxSections];
    __shared__ CoefDF s_cdf[kMaxSections];
    int cur_c = -1;

    // launched early behind the horizon kernel (programmatic dependent
    // launch): the CTAs become resident as that kernel's retire and start
    // once it has completed, without a launch gap in between
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Warp 0 coordinates, warps 1..W hold data.  The coordinator is the CTA's
    // oldest warp: its short, latency-bound path is what every data warp
    // waits for, and the warp schedulers favour older warps.
    const bool coord = warp == 0;
    const uint32_t epoch = *reinterpret_cast<volatile uint32_t*>(&p.hdr->epoch);
    const int64_t total = p.hdr->total_tiles;
    const int64_t nrounds = p.hdr->nrounds;
    // hand-off barriers (made visible to the CTA by the first loop barrier)
    for (int i = tid; i < kMaxSections * W; i += blockDim.x) mbar_init(&ho.bar[0][0] + i, 1);
    if (tid == 0) ho.limit = wait_limit(p.hdr, kHandOffLimit);
    uint32_t ph = 0;  // data warps: hand-off barrier parity per section

    // final states that no tile writes: sections past K[c] are zero, an
    // empty channel keeps its initial state
    if (p.zf) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < (int64_t)p.C * p.kmax;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int c = (int)(i / p.kmax), k = (int)(i % p.kmax);
            const ChanInfo ci = p.chan[c];
            if (k >= ci.K || ci.len == 0) {
                const float z0 = (k < ci.K && p.zi) ? p.zi[i * 2 + 0] : 0.f;
                const float z1 = (k < ci.K && p.zi) ? p.zi[i * 2 + 1] : 0.f;
                p.zf[i * 2 + 0] = z0;
                p.zf[i * 2 + 1] = z1;
            }
        }
    }

    // No carried channel in this call (every channel within its horizon goes
    // through the section pipeline): nothing to dispatch, no slot written, so
    // neither the tile counter nor the look-back epoch has to move.
    if (total == 0) return;

    // Tiles are reserved one ahead: while tile d computes from one buffer,
    // the copies of the next reserved tile fill the other.  A CTA still
    // processes its tiles in dispatch order, and the lowest unfinished tile
    // is always some CTA's current one, so the look-back keeps progressing.
    if (tid == 0) s_t = (int64_t)atomicAdd(&p.hdr->tile_counter, 1u);
    __syncthreads();
    int64_t d = s_t;
    TileGeom gc{};
    if (d < total) {
        gc = tile_geom<KT::kTile>(p, d, nrounds);
        issue_tile_load<N, W>(gc, s_tile4, tid);
    }
    cp_async_commit();
    int cur = 0;
    while (d < total) {
        if (tid == 0) s_t = (int64_t)atomicAdd(&p.hdr->tile_counter, 1u);
        // the reservation is visible, and the previous tile's stores have
        // finished reading the buffer the next copies go to
        __syncthreads();
        const int64_t dn = s_t;
        TileGeom gn{};
        if (dn < total) {
            gn = tile_geom<KT::kTile>(p, dn, nrounds);
            issue_tile_load<N, W>(gn, s_tile4 + (cur ^ 1) * KT::kGran, tid);
        }
        cp_async_commit();
        cp_async_wait1();  // this thread's copies of the current tile

        const int c = gc.c;
        const int64_t ti = gc.ti, t = gc.t, nt = gc.nt, start = gc.start;
        const int r = gc.r, skip = gc.skip;
        const bool carry = gc.carry;
        const ChanInfo ci = p.chan[c];
        float4* buf4 = s_tile4 + cur * KT::kGran;
        float* buf = reinterpret_cast<float*>(buf4);

        if (c != cur_c) {  // CTA-uniform
            constexpr int n32 = sizeof(Coef32) / sizeof(float4), ndf = sizeof(CoefDF) / sizeof(float4);
            const float4* g32 = reinterpret_cast<const float4*>(p.c32 + (int64_t)c * p.kmax);
            const float4* gdf = reinterpret_cast<const float4*>(p.cdf + (int64_t)c * p.kmax);
            for (int i = tid; i < ci.K * n32; i += KT::kThreads)
                reinterpret_cast<float4*>(s_c32)[i] = __ldg(g32 + i);
            for (int i = tid; i < ci.K * ndf; i += KT::kThreads)
                reinterpret_cast<float4*>(s_cdf)[i] = __ldg(gdf + i);
            cur_c = c;
        }
        __syncthreads();  // every thread's copies and the coefficients are in place

        if (coord) {
            if (carry)
                for (int k = 0; k < ci.K; ++k)
                    coord_section<W>(p, k, c, t, ti, nt, carry, epoch, &s_c32[k], &s_cdf[k], &sh);
        } else {
            float v[N];
            const int chunk = (W - warp) * 32 + lane;  // group W - warp of the tile
#pragma unroll
            for (int g = 0; g < N / 4; ++g) {
                const float4 q = buf4[S::g(chunk * (N / 4) + g)];
                v[4 * g + 0] = q.x;
                v[4 * g + 1] = q.y;
                v[4 * g + 2] = q.z;
                v[4 * g + 3] = q.w;
            }
            // owner of the channel's last sample (for zf)
            const bool last = (ti + 1 == nt);
            const int q = r - 1;
            const bool zf_owner = last && p.zf != nullptr && (q / N) == chunk;
            const int mq = q % N;
            // the owner's scratch: its own chunk of the tile buffer, unused
            // while the sections run (plain layout, only that lane touches it)
            float* s_own = buf + chunk * N;
            if (ci.mode) {
                if (carry) {
                    for (int k = 0; k < ci.K; ++k)
                        data_section<N, W, true, false>(p, v, k, c, t, ti, epoch, &s_c32[k],
                                                        &s_cdf[k], &sh, zf_owner, mq, s_own, &ho,
                                                        ph);
                } else {
                    for (int k = 0; k < ci.K; ++k)
                        data_section<N, W, true, true>(p, v, k, c, t, ti, epoch, &s_c32[k],
                                                       &s_cdf[k], &sh, zf_owner, mq, s_own, &ho,
                                                       ph);
                }
                const float G = s_c32[ci.K - 1].misc.y;
#pragma unroll
                for (int m = 0; m < N; ++m) v[m] *= G;
            } else {
                if (carry) {
                    for (int k = 0; k < ci.K; ++k)
                        data_section<N, W, false, false>(p, v, k, c, t, ti, epoch, &s_c32[k],
                                                         &s_cdf[k], &sh, zf_owner, mq, s_own, &ho,
                                                         ph);
                } else {
                    for (int k = 0; k < ci.K; ++k)
                        data_section<N, W, false, true>(p, v, k, c, t, ti, epoch, &s_c32[k],
                                                        &s_cdf[k], &sh, zf_owner, mq, s_own, &ho,
                                                        ph);
                }
            }
            // S7: registers -> shared (swizzled)
            __syncwarp();  // order the zf owner's scratch writes before the lanes' stores
#pragma unroll
            for (int g = 0; g < N / 4; ++g)
                buf4[S::g(chunk * (N / 4) + g)] =
                    make_float4(v[4 * g + 0], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
        }
        __syncthreads();
        // shared -> global, all W + 1 warps (the first `skip` samples are
        // the overlap, already stored by the previous tile; skip % 16 == 0)
        float* dst = p.y + ci.off + start;
        if (((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) && r == KT::kTile) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 4
            for (int g = (skip >> 2) + tid; g < KT::kGran; g += KT::kThreads)
                __stcs(d4 + g, buf4[S::g(g)]);
        } else {
            for (int j = skip + tid; j < r; j += KT::kThreads) __stcs(dst + j, buf[S::e(j)]);
        }
        d = dn;
        gc = gn;
        cur ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");

    // The last CTA to finish opens a new look-back epoch and rewinds the tile
    // counter for the next launch on this workspace (every other CTA has
    // exited, so nobody reads either any more).
    if (tid == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(&p.hdr->done, 1u);
        if (prev == gridDim.x - 1) {
            p.hdr->done = 0;
            p.hdr->tile_counter = 0;
            const uint32_t e = (epoch + 1u) & 0x3fffffffu;
            p.hdr->epoch = e ? e : 1u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------

struct KernelEntry {
    int N, W;
    const void* fn;
    size_t smem;
};

// (N, W, minimum resident CTAs per SM the register allocation must allow)
#define SOSF_ENTRY(N_, W_, B_)                                                              \
    {N_, W_, reinterpret_cast<const void*>(&sos_forward_kernel<N_, W_, B_>),              \
     FwdKernel<N_, W_>::kSmem}

static const KernelEntry kEntries[] = {
    SOSF_ENTRY(16, 8, 3),  SOSF_ENTRY(16, 16, 2), SOSF_ENTRY(32, 4, 4), SOSF_ENTRY(32, 7, 3),
    SOSF_ENTRY(32, 8, 2),  SOSF_ENTRY(32, 16, 1), SOSF_ENTRY(64, 3, 4), SOSF_ENTRY(64, 4, 2),
    SOSF_ENTRY(64, 8, 1),  SOSF_ENTRY(64, 7, 2),
};

bool forward_supported(int N, int W) {
    for (const auto& e : kEntries)
        if (e.N == N && e.W == W) return true;
    return false;
}

cudaError_t launch_forward(const Params& p, int64_t host_tiles, cudaStream_t stream,
                           bool early) {
    const KernelEntry* ke = nullptr;
    for (const auto& e : kEntries)
        if (e.N == p.N && e.W == p.W) ke = &e;
    if (!ke) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    static int s_sms[64] = {0};
    static int s_occ[64][16] = {{0}};
    const int idx = (int)(ke - kEntries);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (s_sms[dev] == 0) {
        err = cudaDeviceGetAttribute(&s_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
    }
    if (s_occ[dev][idx] == 0) {
        err = cudaFuncSetAttribute(ke->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)ke->smem);
        if (err != cudaSuccess) return err;
        int occ = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ke->fn, (p.W + 1) * 32, ke->smem);
        if (err != cudaSuccess) return err;
        s_occ[dev][idx] = occ > 0 ? occ : 1;
    }
    int64_t grid = (int64_t)s_sms[dev] * s_occ[dev][idx];
    if (host_tiles < grid) grid = host_tiles;
    if (grid < 1) return cudaSuccess;
    return launch_params(ke->fn, grid, (p.W + 1) * 32, ke->smem, p, stream, early);
}

}  // namespace sosf
