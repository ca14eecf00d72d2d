// Warp-segment forward kernel for channels within their memory horizon.
//
// The alternative to the section pipeline (pipe.cu) for the same segments:
// one warp runs all K sections of its own segment, group after group, each
// section carrying its DF2T state from one group to the next in registers
// (the paper's group chaining, Sec. V).  A GPU holds a few thousand such
// independent streams and none waits on another warp: there are no
// hand-overs and no pipeline fill, at the price of segments short enough to
// give every warp work, and so a larger share of warm-up (the memory horizon
// P, run from zero state before every segment but a channel's first).
//
// Per warp: two shared-memory slots of one group each (rows padded to N + 4
// floats).  While the sections run on one group in registers, cp.async fills
// the other slot with the next group (of this segment, or the first of the
// warp's next one).  The stride-N permutation in and out is paid once per
// group for the whole cascade (Sec. VII-B).
#include "pipe_section.cuh"
#include "sos_pipe.cuh"

namespace sosf {

constexpr int kWsWarps = 4;  // warps per CTA
constexpr int kWsThreads = kWsWarps * 32;

// CTAs per SM the register budget is sized for (shared memory allows more):
// three, 168 registers per thread.  At four (128 registers) the section
// loop spilled (3.3 local loads per section and group on the band-pass) and
// the kernel ran 16-22 % slower at N = 16 and 32 than at three with room.
template <int N>
constexpr int ws_ctas_per_sm() {
    return 3;
}

template <int N>
struct WsCfg {
    static constexpr int kGroup = 32 * N;
    static constexpr int kGran = kGroup / 4;
    static constexpr int kSlot = 32 * (N + 4);  // floats per slot
    static constexpr size_t kSmem = sizeof(float) * kSlot * 2 * kWsWarps;
};

// the asynchronous copies of one group (rem samples left in the channel)
template <int N>
__device__ __forceinline__ void ws_load(const float* src, int64_t rem, float* slot, int lane) {
    using SL = SlotLayout<N>;
    using WC = WsCfg<N>;
    if (rem >= WC::kGroup && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int q = 0; q < WC::kGran / 32; ++q)
            cp_async16(slot + SL::gran(q * 32 + lane), s4 + q * 32 + lane);
    } else {
        const int r = (int)(rem < WC::kGroup ? rem : WC::kGroup);
        for (int j = lane; j < WC::kGroup; j += 32)
            cp_async4(slot + SL::elem(j), j < r ? src + j : src, j < r);
    }
    cp_async_commit();
}

// Running state of one warp through the groups of its segment.
struct WsCursor {
    const float* src;  // the current group's first input sample
    float* dst;        // its first output sample
    int rem;           // samples of the channel from src on (capped)
    int a, b;          // the segment's own outputs, relative to the group start
};

// Precision class of a channel (ChanInfo::ext), which selects the
// instantiation of the segment code that runs it.
enum WsPrec {
    kPrecF32 = 0,   // every section in FP32
    kPrecSect = 1,  // sections flagged in Coef32::misc.w: 1 = coefficient low
                    // parts in the in-lane recursions, 2 = also the lane scan and
                    // fold in double-float
    kPrecDF = 2     // a range of sections with double-float samples (ChanInfo::dflo..dfhi),
                    // FP32 around it
};

// The section coefficients of a channel run with double-float samples.
__device__ __forceinline__ SecDF load_secdf(const Coef32* cf) {
    const float4 ab = cf->ab, alo = cf->alo, br = cf->braw, bl = cf->blo;
    return SecDF{df{ab.x, alo.x}, df{ab.y, alo.y}, df{br.x, bl.x}, df{br.y, bl.y},
                 df{br.z, bl.z}};
}

// Sections [k0, k1) of a channel run with double-float samples over one
// group (kPrecDF): on entry the lane's row holds its chunk of the range's
// FP32 input, on exit the chunk of its output, rounded once.  Out of line, so
// that its register needs (a double-float section keeps several times the
// temporaries of an FP32 one) do not reach the allocation of the FP32 code
// in the same kernel; the call costs nothing next to the section's work.
template <int N, bool ZF>
__device__ __noinline__ void dfx_group(const Params& p, const Coef32* cf0, int k0, int k1, int c,
                                       float* row, float4* zs, int lane, int owner, int mq) {
    float v[N];
    row_to_chunk<N>(v, row);
    // the low parts live in the lane's row; the input is FP32: they start at
    // zero
#pragma unroll
    for (int b = 0; b < N / 4; ++b)
        reinterpret_cast<float4*>(row)[b] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const Coef32* cf = cf0 + k;
        const SecDF sd = load_secdf(cf);
        const float4 lp = cf->lane_pow[lane], lpl = cf->lane_lo[lane];
        float* zf_dst = ZF ? p.zf + ((int64_t)c * p.kmax + k) * 2 : nullptr;
        const float4 zz = zs[k];
        df z1{zz.x, zz.y}, z2{zz.z, zz.w};
        pipe_section_dfx<N, ZF>(v, row, sd, cf->phi_pow, cf->phi_lo, lp, lpl, z1, z2,
                                lane == owner, mq, zf_dst);
        if (lane == 0) zs[k] = make_float4(z1.hi, z1.lo, z2.hi, z2.lo);
    }
#pragma unroll
    for (int b = 0; b < N / 4; ++b) {
        const float4 l = reinterpret_cast<const float4*>(row)[b];
        reinterpret_cast<float4*>(row)[b] = make_float4(v[4 * b + 0] + l.x, v[4 * b + 1] + l.y,
                                                        v[4 * b + 2] + l.z, v[4 * b + 3] + l.w);
    }
}

// Sections [k0, k1) of a channel over one group in FP32, the chunk v[] in
// registers; zs: their DF2T states (lo parts left zero).  One copy of the
// section code (a rolled loop keeps the kernel's instruction footprint inside
// the instruction cache); plain (L1-cached) loads at the point of use:
// read-only loads would be hoisted out of the group loop, eight sections'
// worth of live registers.  PREC = kPrecSect: each section's level
// (Coef32::misc.w) picks the coefficient low parts or the double-float scan.
// RAW: b0, b1, b2 normalised by a0 only (the double-float range's
// neighbours, whose states are not scaled by the factored gains).
template <int N, bool FACT, bool CR, bool ZF, int PREC, bool RAW>
__device__ __forceinline__ void ws_sections(const Params& p, int c, const Coef32* cf0, int k0,
                                            int k1, float (&v)[N], float* row, float4* zs,
                                            int lane, int owner, int mq) {
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const Coef32* cf = cf0 + k;
        float4 ab = cf->ab;
        float b0 = FACT ? 1.f : cf->misc.x;
        if (RAW) {
            const float4 br = cf->braw;
            ab.z = br.y;
            ab.w = br.z;
            b0 = br.x;
        }
        const float G = (ZF && FACT) ? cf->misc.y : 1.f;
        float* zf_dst = ZF ? p.zf + ((int64_t)c * p.kmax + k) * 2 : nullptr;
        const float4 zz = zs[k];
        float2 z = make_float2(zz.x, zz.z);
        const float lvl = PREC == kPrecSect ? cf->misc.w : 0.f;
        if (CR) {
            pipe_section_cr<N, FACT, ZF>(v, ab, b0, &cf->cr_lv[0], z.x, z.y, lane == owner, mq,
                                         row, zf_dst, G);
        } else if (PREC == kPrecSect && lvl > 1.5f) {
            const float4 lp = cf->lane_pow[lane], lpl = cf->lane_lo[lane], alo = cf->alo;
            pipe_section<N, FACT, ZF, false, true>(v, ab, b0, cf->phi_pow, lp, z.x, z.y,
                                                   lane == owner, mq, row, zf_dst, G, -1, 0.f,
                                                   0.f, cf->phi_lo, lpl,
                                                   make_float2(alo.x, alo.y));
        } else if (PREC == kPrecSect && lvl > 0.5f) {
            const float4 lp = cf->lane_pow[lane], alo = cf->alo;
            pipe_section<N, FACT, ZF, false, false, true>(v, ab, b0, cf->phi_pow, lp, z.x, z.y,
                                                          lane == owner, mq, row, zf_dst, G, -1,
                                                          0.f, 0.f, nullptr,
                                                          make_float4(0.f, 0.f, 0.f, 0.f),
                                                          make_float2(alo.x, alo.y));
        } else {
            const float4 lp = cf->lane_pow[lane];
            pipe_section<N, FACT, ZF>(v, ab, b0, cf->phi_pow, lp, z.x, z.y, lane == owner, mq,
                                      row, zf_dst, G);
        }
        // every lane holds the outgoing state; the writes agree
        if (lane == 0) zs[k] = make_float4(z.x, 0.f, z.y, 0.f);
    }
}

// One group of a segment through all K sections: prefetch the next group,
// filter this one in registers, store the segment's own outputs.  ZF: the
// group holding the channel's last sample, whose final state (zf) is taken at
// element mq of lane `owner`'s chunk; instantiated apart so that the hot
// loop holds no zf code.  PREC: the channel's precision class (WsPrec);
// instantiated apart for the same reason.  zs: the sections' DF2T states
// (z1, z2 as float pairs hi, lo; the lo parts are used by kPrecDF only).
template <int N, bool FACT, bool CR, bool ZF, int PREC>
__device__ __forceinline__ void ws_group(const Params& p, const SegGeom& sg, float* slots,
                                         float4* zs, int lane, int& cur, WsCursor& q, bool last,
                                         bool& pending, const float* nsrc, int64_t nrem,
                                         int owner, int mq) {
    using SL = SlotLayout<N>;
    using WC = WsCfg<N>;
    const int K = sg.K;
    const Coef32* cf0 = p.c32 + (int64_t)sg.c * p.kmax;
    // prefetch: the segment's next group, or the next segment's first
    float* nxt = slots + (cur ^ 1) * WC::kSlot;
    if (!last) {
        ws_load<N>(q.src + WC::kGroup, q.rem - WC::kGroup, nxt, lane);
        cp_async_wait1();
    } else if (nsrc) {
        ws_load<N>(nsrc, nrem, nxt, lane);
        pending = true;
        cp_async_wait1();
    } else {
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncwarp();
    float* slot = slots + cur * WC::kSlot;
    float* row = slot + lane * SL::kRow;
    float v[N];
    if (PREC == kPrecDF) {
        // FP32 sections before and after the double-float range (their b
        // coefficients unfactored, like the range's), the range itself with
        // double-float samples
        const ChanInfo& ci = p.chan[sg.c];
        const int dlo = ci.dflo, dhi = ci.dfhi;
        row_to_chunk<N>(v, row);
        ws_sections<N, false, false, ZF, kPrecSect, true>(p, sg.c, cf0, 0, dlo, v, row, zs,
                                                           lane, owner, mq);
        chunk_to_row<N>(v, row);
        dfx_group<N, ZF>(p, cf0, dlo, dhi + 1, sg.c, row, zs, lane, owner, mq);
        row_to_chunk<N>(v, row);
        ws_sections<N, false, false, ZF, kPrecSect, true>(p, sg.c, cf0, dhi + 1, K, v, row, zs,
                                                           lane, owner, mq);
    } else {
        row_to_chunk<N>(v, row);
        ws_sections<N, FACT, CR, ZF, PREC, false>(p, sg.c, cf0, 0, K, v, row, zs, lane, owner,
                                                  mq);
    }
    if (FACT) {
        const float Gk = cf0[K - 1].misc.y;
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] *= Gk;
    }
    chunk_to_row<N>(v, row);
    __syncwarp();
    // coalesced stores of the segment's own samples of this group
    const int lo = q.a > 0 ? q.a : 0, hi = q.b < WC::kGroup ? q.b : WC::kGroup;
    const bool aligned = (reinterpret_cast<uintptr_t>(q.dst) & 15u) == 0;
    if (lo == 0 && hi == WC::kGroup && aligned) {
        float4* d4 = reinterpret_cast<float4*>(q.dst);
#pragma unroll
        for (int i = 0; i < WC::kGran / 32; ++i)
            __stcs(d4 + i * 32 + lane,
                   *reinterpret_cast<const float4*>(slot + SL::gran(i * 32 + lane)));
    } else if (((lo | hi) & 3) == 0 && aligned) {
        float4* d4 = reinterpret_cast<float4*>(q.dst);
        for (int i = (lo >> 2) + lane; i < (hi >> 2); i += 32)
            __stcs(d4 + i, *reinterpret_cast<const float4*>(slot + SL::gran(i)));
    } else {
        for (int j = lo + lane; j < hi; j += 32) __stcs(q.dst + j, slot[SL::elem(j)]);
    }
    __syncwarp();
    cur ^= 1;
    q.src += WC::kGroup;
    q.dst += WC::kGroup;
    q.rem -= WC::kGroup;
    q.a -= WC::kGroup;
    q.b -= WC::kGroup;
}

// All groups of one segment through all K sections (one warp).  On entry
// slot `cur` holds the segment's first group if `pending`; on exit `cur` is
// the slot of the next segment's first group, and `pending` says whether it
// was issued (nsrc: that group's source, nullptr if none).
template <int N, bool FACT, bool CR, int PREC>
__device__ __forceinline__ void ws_segment(const Params& p, const SegGeom& sg, float* slots,
                                           float4* zs, int lane, int& cur, bool& pending,
                                           const float* nsrc, int64_t nrem) {
    using WC = WsCfg<N>;
    const int K = sg.K;
    const Coef32* cf0 = p.c32 + (int64_t)sg.c * p.kmax;
    // the state entering the segment (zs[k], the same in every lane): zi
    // (scaled by 1/G_k when b0 is factored) on the channel's first segment,
    // zero state after a warm-up
    __syncwarp();
    if (lane < K) {
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sg.si == 0 && p.zi) {
            const float gi = FACT ? __ldg(&cf0[lane].misc.z) : 1.f;
            z.x = __ldg(p.zi + ((int64_t)sg.c * p.kmax + lane) * 2 + 0) * gi;
            z.z = __ldg(p.zi + ((int64_t)sg.c * p.kmax + lane) * 2 + 1) * gi;
        }
        zs[lane] = z;
    }
    __syncwarp();
    WsCursor q;
    q.src = p.x + sg.off + sg.cstart;
    q.dst = p.y + sg.off + sg.cstart;
    q.rem = (int)(sg.len - sg.cstart < 0x40000000 ? sg.len - sg.cstart : 0x40000000);
    q.a = (int)(sg.out_lo - sg.cstart);
    q.b = (int)(sg.out_hi - sg.cstart);
    if (!pending) ws_load<N>(q.src, q.rem, slots + cur * WC::kSlot, lane);
    pending = false;
    // the channel's last sample is in the segment's last group when the
    // segment ends the channel: that group takes the zf path
    const int ng = sg.ngroups;
    const bool zf_last = p.zf && sg.out_hi == sg.len;
    const int ghot = zf_last ? ng - 1 : ng;
    for (int g = 0; g < ghot; ++g)
        ws_group<N, FACT, CR, false, PREC>(p, sg, slots, zs, lane, cur, q, g + 1 == ng, pending,
                                           nsrc, nrem, 0, 0);
    if (zf_last) {
        const int rel = (int)(sg.len - 1 - sg.cstart);
        ws_group<N, FACT, CR, true, PREC>(p, sg, slots, zs, lane, cur, q, true, pending, nsrc,
                                          nrem, (rel % WC::kGroup) / N, rel % N);
    }
}

// One segment of a channel within its memory horizon, in the instantiation
// its channel needs (identity, cyclic reduction, FP32 PH, per-section
// extended precision, or double-float samples).
template <int N, bool CRK>
__device__ __forceinline__ void ws_run_segment(const Params& p, const SegGeom& sg, float* slots,
                                               float4* zs, int lane, int& cur, bool& pending,
                                               const float* nsrc, int64_t nrem) {
    if (sg.K == 0) {
        // identity channel: copy the segment's own samples
        for (int64_t i = sg.out_lo + lane; i < sg.out_hi; i += 32)
            p.y[sg.off + i] = __ldg(p.x + sg.off + i);
    } else {
        const ChanInfo& ci = p.chan[sg.c];
        const bool fact = ci.mode != 0;
        // the channel's precision class (sos_plan_extended): 3 = the whole
        // cascade in double-float, 1..2 = some sections in extended
        // precision, 0 = FP32
        const int ext = ci.ext;
        // cyclic reduction when the call asks for it and every section of
        // the channel is well conditioned for it (FP32 channels only), PH
        // otherwise
        bool cr = CRK && ext == 0;
        for (int k = 0; k < sg.K && cr; ++k)
            cr = __ldg(&p.c32[(int64_t)sg.c * p.kmax + k].cr_misc.w) != 0.f;
        if (ext >= 3)
            ws_segment<N, false, false, kPrecDF>(p, sg, slots, zs, lane, cur, pending,
                                                 nsrc, nrem);
        else if (CRK && fact && cr)
            ws_segment<N, true, CRK, kPrecF32>(p, sg, slots, zs, lane, cur, pending,
                                               nsrc, nrem);
        else if (CRK && cr)
            ws_segment<N, false, CRK, kPrecF32>(p, sg, slots, zs, lane, cur, pending,
                                                nsrc, nrem);
        else if (fact && ext)
            ws_segment<N, true, false, kPrecSect>(p, sg, slots, zs, lane, cur, pending,
                                                  nsrc, nrem);
        else if (fact)
            ws_segment<N, true, false, kPrecF32>(p, sg, slots, zs, lane, cur, pending,
                                                 nsrc, nrem);
        else if (ext)
            ws_segment<N, false, false, kPrecSect>(p, sg, slots, zs, lane, cur, pending,
                                                   nsrc, nrem);
        else
            ws_segment<N, false, false, kPrecF32>(p, sg, slots, zs, lane, cur, pending,
                                                  nsrc, nrem);
    }
}

// CRK: the cyclic-reduction instantiation (algo 2).  The PH one carries no
// cyclic-reduction code, so its register allocation does not pay for it.
template <int N, bool CRK>
__global__ void __launch_bounds__(kWsThreads, ws_ctas_per_sm<N>()) sos_warpseg_kernel(Params p) {
    using WC = WsCfg<N>;
    // the look-back kernel queued behind this one may be launched now (it
    // waits for this kernel's completion before it starts work)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // launched early behind the plan kernel: wait for its completion (and
    // its writes) before the first read of the plan's tables
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ float4 s_ws4[];
    __shared__ float4 s_z[kWsWarps][kMaxSections];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* slots = reinterpret_cast<float*>(s_ws4) + (size_t)w * 2 * WC::kSlot;
    const int64_t total = p.hdr->total_pipe;  // segments of the latest plan
    const int64_t nw = (int64_t)gridDim.x * kWsWarps;
    int cur = 0;
    bool pending = false;
    // segments: the first nw one per warp, the rest handed out in order as
    // warps come free (segments differ in length across uneven channels)
    int64_t d = (int64_t)blockIdx.x * kWsWarps + w;
    SegGeom sg{};
    if (d < total) sg = seg_geom<WC::kGroup>(p, d);
    while (d < total) {
        // the warp's next segment, taken one ahead for the prefetch (only its
        // first group's source is kept live; its geometry is looked up again)
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&p.hdr->seg_next, 1ull);
        const int64_t dn = nw + (int64_t)__shfl_sync(0xffffffffu, t, 0);
        const float* nsrc = nullptr;
        int64_t nrem = 0;
        if (dn < total) {
            const SegGeom nx = seg_geom<WC::kGroup>(p, dn);
            if (nx.K > 0) {
                nsrc = p.x + nx.off + nx.cstart;
                nrem = nx.len - nx.cstart;
            }
        }
        ws_run_segment<N, CRK>(p, sg, slots, s_z[w], lane, cur, pending, nsrc, nrem);
        d = dn;
        if (d < total) sg = seg_geom<WC::kGroup>(p, d);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the last warp to finish resets the hand-out for the next launch (every
    // warp's last atomicAdd on seg_next precedes its arrival here)
    if (lane == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&p.hdr->seg_done, 1u);
        if (prev + 1 == (unsigned)nw) {
            p.hdr->seg_next = 0;
            p.hdr->seg_done = 0;
            __threadfence();
        }
    }
}

// Low-latency streaming: the next block of `chunk` samples of every channel
// (x, y: [C][chunk]) through all K sections, from the state `p.zi` into the
// state `p.zf`, in one launch with the coefficient tables of an earlier
// sos_prepare.  Warp w takes segment w % maxseg of channel w / maxseg: a
// channel within its memory horizon is cut into segments of
// max(seg_len, its shortest allowed segment) samples, each warmed up over the
// horizon from zero state (the first from the incoming state), so that a
// long block is not one warp's sequential walk; other channels are one
// segment.  No plan launch, no hand-out counter, no waits on other warps.
// The paper's real-time scenario: a signal arriving in blocks, the state
// carried from one block to the next (Sec. V's group chaining across calls).
template <int N>
__global__ void __launch_bounds__(kWsThreads, ws_ctas_per_sm<N>())
    sos_stream_kernel(Params p, int64_t chunk, int64_t seg_len, int32_t maxseg, int32_t foreign) {
    using WC = WsCfg<N>;
    extern __shared__ float4 s_ws4[];
    __shared__ float4 s_z[kWsWarps][kMaxSections];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWsWarps + w;
    const int c = (int)(gw / maxseg);
    const int si = (int)(gw % maxseg);
    if (c >= p.C || chunk <= 0) return;
    const ChanInfo ci = p.chan[c];
    int64_t seg = chunk;
    if (ci.horizon >= 0 && ci.K > 0) {
        // the incoming state of a stream is what earlier samples of the same
        // signal left, so its response is part of the impulse-response tail
        // the horizon bounds; a foreign initial state also has to die out
        const int64_t least = foreign ? ci.minseg_z : ci.minseg;
        seg = seg_len > least ? seg_len : least;
        if (seg > chunk) seg = chunk;
    }
    const int nseg = (int)((chunk + seg - 1) / seg);
    if (si >= nseg) return;
    // the channel's coefficient tables into L1 now, all sections at once
    // (each is otherwise a round trip to L2 at the section's first use, one
    // after another: most of a short block's latency)
    {
        const char* cb = reinterpret_cast<const char*>(p.c32 + (int64_t)c * p.kmax);
        const int lines = (int)((sizeof(Coef32) * (size_t)ci.K + 127) / 128);
        for (int i = lane; i < lines; i += 32)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(cb + 128 * (size_t)i));
    }
    // state rows past K (or a channel without sections) pass through
    if (si == 0 && p.zf)
        for (int i = ci.K * 2 + lane; i < p.kmax * 2; i += 32)
            p.zf[(int64_t)c * p.kmax * 2 + i] = p.zi ? p.zi[(int64_t)c * p.kmax * 2 + i] : 0.f;
    float* slots = reinterpret_cast<float*>(s_ws4) + (size_t)w * 2 * WC::kSlot;
    SegGeom sg;
    sg.c = c;
    sg.si = si;
    sg.off = (int64_t)c * chunk;
    sg.len = chunk;
    sg.out_lo = (int64_t)si * seg;
    sg.out_hi = sg.out_lo + seg < chunk ? sg.out_lo + seg : chunk;
    sg.cstart = si == 0 ? 0 : sg.out_lo - ci.horizon;
    sg.ngroups = (int)((sg.out_hi - sg.cstart + WC::kGroup - 1) / WC::kGroup);
    sg.horizon = ci.horizon;
    sg.K = ci.K;
    int cur = 0;
    bool pending = false;
    ws_run_segment<N, false>(p, sg, slots, s_z[w], lane, cur, pending, nullptr, 0);
    asm volatile("cp.async.wait_all;" ::: "memory");
}

#define SOSF_WS(N_, CR_) reinterpret_cast<const void*>(&sos_warpseg_kernel<N_, CR_>)

namespace {
const void* ws_fn(int N, bool cr) {
    if (cr) return N == 16 ? SOSF_WS(16, true) : N == 32 ? SOSF_WS(32, true) : SOSF_WS(64, true);
    return N == 16 ? SOSF_WS(16, false) : N == 32 ? SOSF_WS(32, false) : SOSF_WS(64, false);
}
size_t ws_smem(int N) { return sizeof(float) * 32 * (size_t)(N + 4) * 2 * kWsWarps; }
}  // namespace

// CTAs of the warp-segment kernel (algo 2: the cyclic-reduction one)
// resident per SM (0 on error)
int warpseg_ctas_per_sm(int N, int algo) {
    static int s_occ[2][3] = {{0, 0, 0}, {0, 0, 0}};
    const int idx = N == 16 ? 0 : N == 32 ? 1 : 2, a = algo == 2 ? 1 : 0;
    if (s_occ[a][idx] == 0) {
        const void* fn = ws_fn(N, a == 1);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ws_smem(N)) != cudaSuccess)
            return 0;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kWsThreads, ws_smem(N)) !=
            cudaSuccess)
            return 0;
        s_occ[a][idx] = occ;
    }
    return s_occ[a][idx];
}

int warpseg_warps_per_cta() { return kWsWarps; }

cudaError_t launch_stream(const Params& p, int64_t chunk, int64_t seg_len, int32_t maxseg,
                          int32_t foreign, cudaStream_t stream) {
    const void* fn = p.N == 16 ? reinterpret_cast<const void*>(&sos_stream_kernel<16>)
                   : p.N == 32 ? reinterpret_cast<const void*>(&sos_stream_kernel<32>)
                               : reinterpret_cast<const void*>(&sos_stream_kernel<64>);
    static bool attr[3] = {false, false, false};
    const int idx = p.N == 16 ? 0 : p.N == 32 ? 1 : 2;
    if (!attr[idx]) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem(p.N));
        if (e != cudaSuccess) return e;
        attr[idx] = true;
    }
    void* args[] = {const_cast<Params*>(&p), &chunk, &seg_len, &maxseg, &foreign};
    const int64_t warps = (int64_t)p.C * maxseg;
    const unsigned grid = (unsigned)((warps + kWsWarps - 1) / kWsWarps);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kWsThreads), args, ws_smem(p.N), stream);
}

cudaError_t launch_warpseg(const Params& p, int64_t grid, cudaStream_t stream, bool early) {
    if (warpseg_ctas_per_sm(p.N, p.algo) < 1) return cudaErrorInvalidConfiguration;
    if (grid < 1) return cudaSuccess;
    return launch_params(ws_fn(p.N, p.algo == 2), grid, kWsThreads, ws_smem(p.N), p, stream,
                         early);
}

}  // namespace sosf
