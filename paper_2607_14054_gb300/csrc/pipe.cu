// Section-pipeline forward kernel for channels within their memory horizon.
//
// A channel whose impulse response dies out within P samples (its memory
// horizon, bounded by the plan) is cut into segments of S samples; segment
// i > 0 is computed from P samples before its start, from zero state, and the
// state it drops changes its outputs by less than 2^-30 relative.  Inside a
// segment the cascade runs exactly as the paper's group chaining (Sec. V):
// the segment is a sequence of groups of N*L samples (L = 32 lanes), and each
// section carries its DF2T state from one group to the next.
//
// One CTA per SM runs two pipelines of warps, each over its own segments:
//   warp 0             loader: global -> a ring of shared-memory slots (one
//                      group each, swizzled), by asynchronous copies;
//   warp 1 + k         section k: for every group, in order, reads the group
//                      (lane l takes samples [lN, lN + N): the stride-N
//                      permutation of Sec. VII-A), runs S3 (non-recursive
//                      stage), S4-PH (particular solution, 5-round lane scan,
//                      re-run from the true lane state) from the state the
//                      previous group left, writes the group back in place
//                      and passes the slot on;
//   warp kMaxSections+1 storer: coalesced stores of finished groups.
// Each slot moves loader -> section 0 -> ... -> section 7 -> storer -> loader,
// every hand-over an mbarrier phase; sections past the channel's K pass the
// slot through.  No warp waits on another's state, only on data, and the
// permutation in and out is paid once per group for the whole cascade
// (Sec. VII-B).
#include <type_traits>

#include "sos_pipe.cuh"
#include "pipe_section.cuh"

namespace sosf {

// The groups of one segment through section k (warp 1 + k).  ZFK: the call
// asks for final states (the zf instantiation of the section is compiled in).
template <int N, bool FACT, bool CR, bool ZFK>
__device__ __forceinline__ void pipe_segment_section(const Params& p, const SegGeom& sg, int k,
                                                     PipeShared& sh, float* ring, int& s,
                                                     unsigned& use, const float4 ab,
                                                     const float4 misc, const float4 lp) {
    using SL = SlotLayout<N>;
    const int lane = threadIdx.x & 31;
    const float4* phi = sh.phi[k];
    // the state entering the segment: zi (scaled by 1/G_k when b0 is
    // factored) for the channel's first segment, zero state otherwise
    float Z1 = 0.f, Z2 = 0.f;
    if (sg.si == 0 && p.zi) {
        const float gi = FACT ? misc.z : 1.f;
        Z1 = p.zi[((int64_t)sg.c * p.kmax + k) * 2 + 0] * gi;
        Z2 = p.zi[((int64_t)sg.c * p.kmax + k) * 2 + 1] * gi;
    }
    const bool last_k = k == sg.K - 1;
    // the group holding the channel's last sample (zf), if in this segment
    int g_last = -1, owner = 0, mq = 0;
    if (ZFK && sg.out_hi == sg.len) {
        const int rel = (int)(sg.len - 1 - sg.cstart);
        g_last = rel / (32 * N);
        owner = (rel % (32 * N)) / N;
        mq = rel % N;
    }
    float* zf_dst = p.zf + ((int64_t)sg.c * p.kmax + k) * 2;
    const float G = misc.y;
    // one group; ZG: the group holding the channel's last sample (the last
    // group of the segment), run after the loop so that the loop's code
    // holds none of the zf selects
    auto group = [&](int g, auto zg) {
        constexpr bool ZG = decltype(zg)::value;
        pipe_wait(p, &sh.bar[s][k], use & 1u, lane, sh.limit);
        float* row = ring + s * SL::kFloats + lane * SL::kRow;
        const bool zf_owner = ZG && lane == owner;
        float v[N];
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(row + 4 * q);
            v[4 * q + 0] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
        if (!CR)
            pipe_section<N, FACT, ZG>(v, ab, misc.x, phi, lp, Z1, Z2, zf_owner, mq, row, zf_dst,
                                      (ZG && FACT) ? G : 1.f);
        else
            pipe_section_cr<N, FACT, ZG>(v, ab, misc.x, sh.cr[k], Z1, Z2, zf_owner, mq, row,
                                         zf_dst, (ZG && FACT) ? G : 1.f);
        if (FACT && last_k) {
#pragma unroll
            for (int m = 0; m < N; ++m) v[m] *= G;
        }
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            *reinterpret_cast<float4*>(row + 4 * q) =
                make_float4(v[4 * q + 0], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        pipe_arrive(&sh.bar[s][k + 1]);
        if (++s == kPipeRing) {
            s = 0;
            ++use;
        }
    };
    const int nplain = g_last >= 0 ? g_last : sg.ngroups;  // g_last = ngroups - 1 if set
    for (int g = 0; g < nplain; ++g) group(g, std::false_type{});
    if (ZFK && g_last >= 0) group(g_last, std::true_type{});
}

template <int N, bool ZFK>
__global__ void __launch_bounds__(2 * kPipeThreads, 1) sos_pipe_kernel(Params p) {
    using PC = PipeCfg<N>;
    using SL = SlotLayout<N>;
    // the look-back kernel queued behind this one may be launched now (it
    // waits for this kernel's completion before it starts work)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // launched early behind the plan kernel: wait for its completion (and
    // its writes) before the first read of the plan's tables
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ float4 s_ring4[];
    __shared__ PipeShared sh2[2];
    const int tid = threadIdx.x, lane = tid & 31, warp2 = tid >> 5;
    // two pipelines per CTA, their warps interleaved (even warps pipeline 0,
    // odd warps pipeline 1): the schedulers then favour neither, where two
    // CTAs of one pipeline each on an SM finished 10-12 us apart
    const int pl = warp2 & 1, warp = warp2 >> 1;
    PipeShared& sh = sh2[pl];
    float* ring = reinterpret_cast<float*>(s_ring4) + (size_t)pl * SL::kFloats * kPipeRing;
    const int64_t total = p.hdr->total_pipe;  // pipeline segments of the latest plan

    for (int i = tid; i < 2 * kPipeRing; i += blockDim.x) {
        // every hand-over is an arrival of all 32 lanes of the handing warp
        // (for the loader: completion of each lane's copies)
        PipeShared& q = sh2[i / kPipeRing];
        for (int j = 0; j < kPipeStages; ++j) mbar_init(&q.bar[i % kPipeRing][j], 32);
        mbar_init(&q.free_[i % kPipeRing], 32);
    }
    if (tid == 0) {
        sh2[0].limit = wait_limit(p.hdr, kHandOffLimit);
        sh2[1].limit = sh2[0].limit;
    }
    __syncthreads();
    const int64_t d0 = 2 * (int64_t)blockIdx.x + pl, dstep = 2 * (int64_t)gridDim.x;

    // ring position of the next group (all warps walk the same sequence):
    // slot s, and the parity of the slot's current use
    int s = 0;
    unsigned use = 0;
    if (warp == 0) {
        // ---- loader ----
        for (int64_t d = d0; d < total; d += dstep) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            const float* src = p.x + sg.off + sg.cstart;
            int rem = (int)(sg.len - sg.cstart < 0x40000000 ? sg.len - sg.cstart : 0x40000000);
            for (int g = 0; g < sg.ngroups; ++g, src += PC::kGroup, rem -= PC::kGroup) {
                if (use > 0) pipe_wait(p, &sh.free_[s], (use - 1) & 1u, lane, sh.limit);
                float* slot = ring + s * SL::kFloats;
                if (rem >= PC::kGroup && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
                    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                    for (int q = 0; q < PC::kGran / 32; ++q)
                        cp_async16(slot + SL::gran(q * 32 + lane), s4 + q * 32 + lane);
                } else {
                    for (int j = lane; j < PC::kGroup; j += 32)
                        cp_async4(slot + SL::elem(j), j < rem ? src + j : src, j < rem);
                }
                cp_async_arrive_noinc(&sh.bar[s][0]);
                if (++s == kPipeRing) {
                    s = 0;
                    ++use;
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kPipeWarps - 1) {
        // ---- storer ----
        for (int64_t d = d0; d < total; d += dstep) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            float* dst = p.y ? p.y + sg.off + sg.cstart : nullptr;
            // group-relative store window [a, b)
            int a = (int)(sg.out_lo - sg.cstart);
            int b = (int)(sg.out_hi - sg.cstart);
            for (int g = 0; g < sg.ngroups; ++g, dst += PC::kGroup, a -= PC::kGroup,
                     b -= PC::kGroup) {
                pipe_wait(p, &sh.bar[s][kMaxSections], use & 1u, lane, sh.limit);
                const float* slot = ring + s * SL::kFloats;
                const int lo = a > 0 ? a : 0;
                const int hi = b < PC::kGroup ? b : PC::kGroup;
                const bool aligned = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
                if (!p.y) {
                } else if (lo == 0 && hi == PC::kGroup && aligned) {
                    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                    for (int q = 0; q < PC::kGran / 32; ++q)
                        __stcs(d4 + q * 32 + lane,
                               *reinterpret_cast<const float4*>(slot + SL::gran(q * 32 + lane)));
                } else if (((lo | hi) & 3) == 0 && aligned) {
                    float4* d4 = reinterpret_cast<float4*>(dst);
                    for (int q = (lo >> 2) + lane; q < (hi >> 2); q += 32)
                        __stcs(d4 + q, *reinterpret_cast<const float4*>(slot + SL::gran(q)));
                } else {
                    for (int j = lo + lane; j < hi; j += 32) __stcs(dst + j, slot[SL::elem(j)]);
                }
                __syncwarp();
                pipe_arrive(&sh.free_[s]);
                if (++s == kPipeRing) {
                    s = 0;
                    ++use;
                }
            }
        }
    } else {
        // ---- section k = warp - 1 ----
        const int k = warp - 1;
        int cur_c = -1;
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f), misc = ab, lp = ab;
        for (int64_t d = d0; d < total; d += dstep) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            if (k < sg.K) {
                if (sg.c != cur_c) {
                    const Coef32* cf = p.c32 + (int64_t)sg.c * p.kmax + k;
                    ab = __ldg(&cf->ab);
                    misc = __ldg(&cf->misc);
                    lp = __ldg(&cf->lane_pow[lane]);
                    __syncwarp();
                    if (lane < 5) sh.phi[k][lane] = __ldg(&cf->phi_pow[lane]);
                    if (lane < 14) sh.cr[k][lane] = __ldg(&cf->cr_lv[0] + lane);
                    __syncwarp();
                    cur_c = sg.c;
                }
                const bool cr = p.algo == 2 && sh.cr[k][13].w != 0.f;
                const bool fact = p.chan[sg.c].mode != 0;
                if (fact && cr)
                    pipe_segment_section<N, true, true, ZFK>(p, sg, k, sh, ring, s, use, ab,
                                                             misc, lp);
                else if (fact)
                    pipe_segment_section<N, true, false, ZFK>(p, sg, k, sh, ring, s, use, ab,
                                                             misc, lp);
                else if (cr)
                    pipe_segment_section<N, false, true, ZFK>(p, sg, k, sh, ring, s, use, ab,
                                                             misc, lp);
                else
                    pipe_segment_section<N, false, false, ZFK>(p, sg, k, sh, ring, s, use, ab,
                                                             misc, lp);
            } else {
                // past the channel's K: pass the groups through
                for (int g = 0; g < sg.ngroups; ++g) {
                    pipe_wait(p, &sh.bar[s][k], use & 1u, lane, sh.limit);
                    pipe_arrive(&sh.bar[s][k + 1]);
                    if (++s == kPipeRing) {
                        s = 0;
                        ++use;
                    }
                }
            }
        }
    }
}

#define SOSF_PIPE(N_, Z_) reinterpret_cast<const void*>(&sos_pipe_kernel<N_, Z_>)

bool pipe_supported(int N) { return N == 16 || N == 32 || N == 64; }

int64_t pipe_group(int N) { return 32LL * N; }

cudaError_t launch_pipe(const Params& p, int64_t grid, cudaStream_t stream, bool early) {
    const bool z = p.zf != nullptr;
    const void* fn = z ? (p.N == 16 ? SOSF_PIPE(16, true) : p.N == 32 ? SOSF_PIPE(32, true)
                                                               : SOSF_PIPE(64, true))
                       : (p.N == 16 ? SOSF_PIPE(16, false) : p.N == 32 ? SOSF_PIPE(32, false)
                                                                : SOSF_PIPE(64, false));
    const size_t smem = 2 * sizeof(float) * 32 * (size_t)(p.N + 4) * kPipeRing;
    static bool attr[2][3] = {{false, false, false}, {false, false, false}};
    const int idx = p.N == 16 ? 0 : p.N == 32 ? 1 : 2;
    if (!attr[z][idx]) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[z][idx] = true;
    }
    if (grid < 1) return cudaSuccess;
    return launch_params(fn, (grid + 1) / 2, 2 * kPipeThreads, smem, p, stream, early);
}

}  // namespace sosf
