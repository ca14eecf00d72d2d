// Building blocks shared by the forward and adjoint section pipelines:
// segment geometry, the slot layout of the group ring, and the bounded
// mbarrier hand-overs between the pipeline's warps.
#pragma once

#include "sos_async.cuh"
#include "sos_kernels.cuh"

namespace sosf {

constexpr int kPipeRing = 12;                  // group slots per CTA
constexpr int kPipeWarps = kMaxSections + 2;   // loader, sections, storer
constexpr int kPipeThreads = kPipeWarps * 32;
constexpr int kPipeStages = kMaxSections + 1;  // barriers per slot: ready-for stage 0..7, storer

template <int N>
struct PipeCfg {
    static constexpr int kGroup = 32 * N;  // samples per group
    static constexpr int kGran = kGroup / 4;
    static constexpr size_t kSmem = sizeof(float) * 32 * (N + 4) * kPipeRing;
};

// Segment si of channel c: outputs [out_lo, out_hi), computed from cstart.
struct SegGeom {
    int64_t off, len, out_lo, out_hi, cstart;
    int c, si, ngroups, horizon, K;
};

template <int kGroup>
__device__ __forceinline__ SegGeom seg_geom(const Params& p, int64_t d) {
    int lo = 0, hi = p.C - 1;  // the largest position with tbp[pos] <= d
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&p.tbp[mid]) <= d) lo = mid; else hi = mid - 1;
    }
    const int c = __ldg(&p.porder[lo]);
    const ChanInfo ci = p.chan[c];
    SegGeom g;
    g.c = c;
    g.si = (int)(d - __ldg(&p.tbp[lo]));
    g.off = ci.off;
    g.len = ci.len;
    g.K = ci.K;
    g.horizon = ci.horizon;
    g.out_lo = (int64_t)g.si * ci.seg;
    g.out_hi = (ci.single || g.out_lo + ci.seg >= ci.len) ? ci.len : g.out_lo + ci.seg;
    g.cstart = g.si == 0 ? 0 : g.out_lo - ci.horizon;
    g.ngroups = (int)((g.out_hi - g.cstart + kGroup - 1) / kGroup);
    return g;
}

struct PipeShared {
    unsigned long long bar[kPipeRing][kPipeStages];  // slot ready for stage j
    unsigned long long free_[kPipeRing];             // slot free for the loader
    float4 phi[kMaxSections][5];                     // section k's Phi^(2^j), staged by warp 1 + k
    float4 cr[kMaxSections][14];                     // section k's cyclic-reduction coefficients
    uint32_t limit;                                  // bound on each hand-over wait (polls)
};

// Bounded, warp-uniform wait for an mbarrier phase.
// (limit: the workspace's bound, read once per launch)
__device__ __forceinline__ void pipe_wait(const Params& p, unsigned long long* b, unsigned par,
                                          int lane, uint32_t limit) {
    for (uint32_t it = 0;; ++it) {
        const bool ok = mbar_try_wait(b, par);
        if (__all_sync(0xffffffffu, ok)) return;
        if (it >= limit) {
            if (lane == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
            return;
        }
    }
}

// Every lane of the warp arrives on `b` (count 32), so each lane's own
// shared-memory writes are released by its own arrive.
__device__ __forceinline__ void pipe_arrive(unsigned long long* b) { mbar_arrive(b); }

__device__ __forceinline__ void cp_async_arrive_noinc(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

// Slot layout: lane l's chunk of N samples at floats [l (N + 4), l (N + 4) + N)
// of the slot.  The 4-float pad per row makes both the chunk-wise 128-bit
// accesses of the section warps (lane l at 16 (N + 4) l bytes: bank groups
// 4l mod 32, distinct across each quarter-warp) and the row-wise ones of the
// loader and storer bank-conflict free, with compile-time offsets for the
// section warps.
template <int N>
struct SlotLayout {
    static constexpr int kRow = N + 4;           // floats per lane row
    static constexpr int kFloats = 32 * kRow;    // floats per slot
    // granule G (16 bytes) of the group, in sample order -> float offset
    __device__ __forceinline__ static int gran(int G) {
        return (G / (N / 4)) * kRow + (G % (N / 4)) * 4;
    }
    // element j of the group -> float offset
    __device__ __forceinline__ static int elem(int j) { return (j / N) * kRow + (j % N); }
};

}  // namespace sosf
