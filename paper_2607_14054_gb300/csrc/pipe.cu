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
// One CTA runs a pipeline of warps over its segments:
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
    int lo = 0, hi = p.C - 1;  // the largest c with tbp[c] <= d
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&p.tbp[mid]) <= d) lo = mid; else hi = mid - 1;
    }
    const ChanInfo ci = p.chan[lo];
    SegGeom g;
    g.c = lo;
    g.si = (int)(d - __ldg(&p.tbp[lo]));
    g.off = ci.off;
    g.len = ci.len;
    g.K = ci.K;
    g.horizon = ci.horizon;
    g.out_lo = (int64_t)g.si * p.seg;
    g.out_hi = g.out_lo + p.seg < ci.len ? g.out_lo + p.seg : ci.len;
    g.cstart = g.si == 0 ? 0 : g.out_lo - ci.horizon;
    g.ngroups = (int)((g.out_hi - g.cstart + kGroup - 1) / kGroup);
    return g;
}

struct PipeShared {
    unsigned long long bar[kPipeRing][kPipeStages];  // slot ready for stage j
    unsigned long long free_[kPipeRing];             // slot free for the loader
    float4 phi[kMaxSections][5];                     // section k's Phi^(2^j), staged by warp 1 + k
};

// try_wait with a suspend-time hint: a warp whose slot is not ready yet
// sleeps until the phase completes (or the hint runs out) instead of polling.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Bounded, warp-uniform wait for an mbarrier phase.
__device__ __forceinline__ void pipe_wait(const Params& p, unsigned long long* b, unsigned par,
                                          int lane) {
    for (uint32_t it = 0;; ++it) {
        const bool ok = mbar_try_wait_sleep(b, par);
        if (__all_sync(0xffffffffu, ok)) return;
        if (it >= kHandOffLimit) {
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

// One section over one group, lane chunk v[] in registers, from the group's
// incoming DF2T state (Z1, Z2) (scaled by 1/G_k when b0 is factored); leaves
// the group's outgoing state in (Z1, Z2).
template <int N, bool FACT>
__device__ __forceinline__ void pipe_section(float (&v)[N], const float4 ab, const float b0,
                                             const float4* phi, const float4 lp, float& Z1,
                                             float& Z2, bool zf_owner, int mq, float* s_own,
                                             float* zf_dst, float G) {
    const int lane = threadIdx.x & 31;
    const float a1 = ab.x, a2 = ab.y, b1 = ab.z, b2 = ab.w;

    // S8 support: the section input at the channel's last sample, picked with
    // a run-time index through the owner's scratch
    float xq = 0.f, xqm1 = 0.f;
    __syncwarp();
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
    float S1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, w1, -a2 * w0)));
    float S2 = fmaf(b2, xl1, -a2 * w1);

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
    const float zin1 = fmaf(lp.x, Z1, fmaf(lp.y, Z2, E1));
    const float zin2 = fmaf(lp.z, Z1, fmaf(lp.w, Z2, E2));

    // S4 (iii): re-run the recursion from the true incoming state
    v[0] = v[0] + zin1;
    v[1] = fmaf(-a1, v[0], v[1] + zin2);
#pragma unroll
    for (int m = 2; m < N; ++m) v[m] = fmaf(-a1, v[m - 1], fmaf(-a2, v[m - 2], v[m]));

    // the group's outgoing state, from lane 31's last two inputs and outputs
    const float o1 = fmaf(b1, xl1, fmaf(b2, xl2, fmaf(-a1, v[N - 1], -a2 * v[N - 2])));
    const float o2 = fmaf(b2, xl1, -a2 * v[N - 1]);
    Z1 = __shfl_sync(0xffffffffu, o1, 31);
    Z2 = __shfl_sync(0xffffffffu, o2, 31);

    // S8: final state at the channel's last sample
    if (zf_owner) {
#pragma unroll
        for (int m = 0; m < N; ++m) s_own[m] = v[m];
        const float yq = s_own[mq];
        const float yqm1 = mq >= 1 ? s_own[mq - 1] : 0.f;
        float f1;
        if (mq >= 1) f1 = fmaf(b1, xq, fmaf(b2, xqm1, fmaf(-a1, yq, -a2 * yqm1)));
        else f1 = fmaf(b1, xq, fmaf(-a1, yq, zin2));
        const float f2 = fmaf(b2, xq, -a2 * yq);
        zf_dst[0] = f1 * G;
        zf_dst[1] = f2 * G;
    }
    __syncwarp();
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

// The groups of one segment through section k (warp 1 + k).
template <int N, bool FACT>
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
    if (p.zf && sg.out_hi == sg.len) {
        const int rel = (int)(sg.len - 1 - sg.cstart);
        g_last = rel / (32 * N);
        owner = (rel % (32 * N)) / N;
        mq = rel % N;
    }
    float* zf_dst = p.zf + ((int64_t)sg.c * p.kmax + k) * 2;
    const float G = misc.y;
    for (int g = 0; g < sg.ngroups; ++g) {
        pipe_wait(p, &sh.bar[s][k], use & 1u, lane);
        float* row = ring + s * SL::kFloats + lane * SL::kRow;
        float v[N];
#pragma unroll
        for (int j = 0; j < N / 4; ++j) {
            const float4 t = *reinterpret_cast<const float4*>(row + 4 * j);
            v[4 * j + 0] = t.x;
            v[4 * j + 1] = t.y;
            v[4 * j + 2] = t.z;
            v[4 * j + 3] = t.w;
        }
        const bool zf_owner = g == g_last && lane == owner;
        pipe_section<N, FACT>(v, ab, misc.x, phi, lp, Z1, Z2, zf_owner, mq, row, zf_dst,
                              FACT ? G : 1.f);
        if (FACT && last_k) {
#pragma unroll
            for (int m = 0; m < N; ++m) v[m] *= G;
        }
#pragma unroll
        for (int j = 0; j < N / 4; ++j)
            *reinterpret_cast<float4*>(row + 4 * j) =
                make_float4(v[4 * j + 0], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        __syncwarp();
        pipe_arrive(&sh.bar[s][k + 1]);
        if (++s == kPipeRing) {
            s = 0;
            ++use;
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kPipeThreads, 2) sos_pipe_kernel(Params p) {
    using PC = PipeCfg<N>;
    using SL = SlotLayout<N>;
    extern __shared__ float4 s_ring4[];
    float* ring = reinterpret_cast<float*>(s_ring4);
    __shared__ PipeShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = p.hdr->total_pipe;  // pipeline segments of the latest plan

    for (int i = tid; i < kPipeRing; i += blockDim.x) {
        // every hand-over is an arrival of all 32 lanes of the handing warp
        // (for the loader: completion of each lane's copies)
        for (int j = 0; j < kPipeStages; ++j) mbar_init(&sh.bar[i][j], 32);
        mbar_init(&sh.free_[i], 32);
    }
    __syncthreads();

    // ring position of the next group (all warps walk the same sequence):
    // slot s, and the parity of the slot's current use
    int s = 0;
    unsigned use = 0;
    if (warp == 0) {
        // ---- loader ----
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            const float* src = p.x + sg.off + sg.cstart;
            int rem = (int)(sg.len - sg.cstart < 0x40000000 ? sg.len - sg.cstart : 0x40000000);
            const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
            for (int g = 0; g < sg.ngroups; ++g, src += PC::kGroup, rem -= PC::kGroup) {
                if (use > 0) pipe_wait(p, &sh.free_[s], (use - 1) & 1u, lane);
                float* slot = ring + s * SL::kFloats;
                if (rem >= PC::kGroup && aligned) {
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
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            float* dst = p.y + sg.off + sg.cstart;
            const bool aligned = (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
            // group-relative store window [a, b)
            int a = (int)(sg.out_lo - sg.cstart);
            int b = (int)(sg.out_hi - sg.cstart);
            for (int g = 0; g < sg.ngroups; ++g, dst += PC::kGroup, a -= PC::kGroup,
                     b -= PC::kGroup) {
                pipe_wait(p, &sh.bar[s][kMaxSections], use & 1u, lane);
                const float* slot = ring + s * SL::kFloats;
                const int lo = a > 0 ? a : 0;
                const int hi = b < PC::kGroup ? b : PC::kGroup;
                if (lo == 0 && hi == PC::kGroup && aligned) {
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
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            if (k < sg.K) {
                if (sg.c != cur_c) {
                    const Coef32* cf = p.c32 + (int64_t)sg.c * p.kmax + k;
                    ab = __ldg(&cf->ab);
                    misc = __ldg(&cf->misc);
                    lp = __ldg(&cf->lane_pow[lane]);
                    __syncwarp();
                    if (lane < 5) sh.phi[k][lane] = __ldg(&cf->phi_pow[lane]);
                    __syncwarp();
                    cur_c = sg.c;
                }
                if (p.chan[sg.c].mode)
                    pipe_segment_section<N, true>(p, sg, k, sh, ring, s, use, ab, misc, lp);
                else
                    pipe_segment_section<N, false>(p, sg, k, sh, ring, s, use, ab, misc, lp);
            } else {
                // past the channel's K: pass the groups through
                for (int g = 0; g < sg.ngroups; ++g) {
                    pipe_wait(p, &sh.bar[s][k], use & 1u, lane);
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

#define SOSF_PIPE(N_) reinterpret_cast<const void*>(&sos_pipe_kernel<N_>)

bool pipe_supported(int N) { return N == 16 || N == 32 || N == 64; }

int64_t pipe_group(int N) { return 32LL * N; }

cudaError_t launch_pipe(const Params& p, int64_t grid, cudaStream_t stream) {
    const void* fn = p.N == 16 ? SOSF_PIPE(16) : p.N == 32 ? SOSF_PIPE(32) : SOSF_PIPE(64);
    const size_t smem = sizeof(float) * 32 * (size_t)(p.N + 4) * kPipeRing;
    static bool attr[3] = {false, false, false};
    const int idx = p.N == 16 ? 0 : p.N == 32 ? 1 : 2;
    if (!attr[idx]) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[idx] = true;
    }
    if (grid < 1) return cudaSuccess;
    void* args[] = {const_cast<Params*>(&p)};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kPipeThreads), args, smem, stream);
}

}  // namespace sosf
