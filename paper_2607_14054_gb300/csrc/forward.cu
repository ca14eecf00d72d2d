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
//      form of the inter-group hand-off of Sec. V) carry of the state;
//  S7  de-permutation through shared memory and coalesced stores;
//  S8  the lane holding a channel's last sample writes zf.
#include <cmath>

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

__device__ __forceinline__ double2 compose_horner(const double th[4], double u1, double u2,
                                                  double c1, double c2) {
    // Theta * u + c
    return make_double2(fma(th[0], u1, fma(th[1], u2, c1)), fma(th[2], u1, fma(th[3], u2, c2)));
}

// Incoming DF2T state of tile t (global index), section k, whose channel-local
// index is ti >= 1.  Run by one full warp; every lane returns the same value.
// Predecessor tiles publish either their aggregate c (zero-state outgoing
// state) or their inclusive value P (true outgoing state); the state entering
// tile t is Z_t = sum_{i<f} Theta^i c_{t-1-i} + Theta^f P_{t-1-f}, formed by
// Horner's rule from the nearest inclusive predecessor f.  Windows of 32
// aggregates without an inclusive value are folded with Theta^32.
__device__ double2 lookback(const Params& p, int64_t t, int64_t ti, int k, uint32_t epoch,
                            const Coef64* cc) {
    const int lane = threadIdx.x & 31;
    double th[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) th[i] = cc->theta[i];
    double acc1 = 0.0, acc2 = 0.0;
    double M[4] = {1.0, 0.0, 0.0, 1.0};
    int64_t base = t - 1;
    int64_t remaining = ti;
    const uint32_t* fl = p.flags + (int64_t)k * p.cap_tiles;
    const double2* ag = p.agg + (int64_t)k * p.cap_tiles;
    const double2* ic = p.inc + (int64_t)k * p.cap_tiles;
    for (;;) {
        const int cnt = (int)(remaining < 32 ? remaining : 32);
        const int64_t j = base - lane;
        const bool valid = lane < cnt;
        uint32_t incm = 0;
        int first = 32;
        uint32_t spins = 0;
        for (;;) {
            const uint32_t st = valid ? ld_acquire_u32(fl + j) : 0u;
            const bool ok = valid && (st >> 2) == epoch && (st & 3u) != 0u;
            const bool isinc = ok && (st & 3u) == kFlagInc;
            incm = __ballot_sync(0xffffffffu, isinc);
            const uint32_t readym = __ballot_sync(0xffffffffu, ok);
            if (incm) {
                first = __ffs(incm) - 1;
                const uint32_t need = first == 0 ? 0u : (0xffffffffu >> (32 - first));
                if ((readym & need) == need) break;
            } else if (cnt == 32 && readym == 0xffffffffu) {
                first = 32;
                break;
            }
            ++spins;
            if (spins > kSpinLimit) {
                if (lane == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
                return make_double2(0.0, 0.0);
            }
            if ((spins & 63u) == 0u && ld_volatile_i32(&p.hdr->status) != 0)
                return make_double2(0.0, 0.0);
            __nanosleep(64);
        }
        double2 val = make_double2(0.0, 0.0);
        if (lane < first && valid) val = ld_relaxed_f64x2(ag + j);
        if (incm && lane == first) val = ld_relaxed_f64x2(ic + j);
        double u1 = 0.0, u2 = 0.0;
        int top = 31;
        if (incm) {
            u1 = __shfl_sync(0xffffffffu, val.x, first);
            u2 = __shfl_sync(0xffffffffu, val.y, first);
            top = first - 1;
        }
        for (int i = top; i >= 0; --i) {
            const double c1 = __shfl_sync(0xffffffffu, val.x, i);
            const double c2 = __shfl_sync(0xffffffffu, val.y, i);
            const double2 n = compose_horner(th, u1, u2, c1, c2);
            u1 = n.x;
            u2 = n.y;
        }
        // Z = acc + M u
        acc1 = fma(M[0], u1, fma(M[1], u2, acc1));
        acc2 = fma(M[2], u1, fma(M[3], u2, acc2));
        if (incm) return make_double2(acc1, acc2);
        // no inclusive value in this window: go 32 tiles further back
        const double* t32 = cc->theta32;
        const double m0 = M[0] * t32[0] + M[1] * t32[2], m1 = M[0] * t32[1] + M[1] * t32[3];
        const double m2 = M[2] * t32[0] + M[3] * t32[2], m3 = M[2] * t32[1] + M[3] * t32[3];
        M[0] = m0; M[1] = m1; M[2] = m2; M[3] = m3;
        base -= 32;
        remaining -= 32;
        if (remaining <= 0) {  // cannot happen: a channel's first tile is always inclusive
            if (lane == 0) set_status(p.hdr, SOS_ERR_TIMEOUT);
            return make_double2(acc1, acc2);
        }
    }
}

template <int N, int W>
struct FwdKernel {
    static constexpr int kThreads = W * 32;
    static constexpr int kTile = W * 32 * N;
    static constexpr int kGran = kTile / 4;
    static constexpr size_t kSmem = sizeof(float) * kTile;
};

// One section of the cascade on the register-resident chunk v[0..N).
template <int N, int W, bool FACT>
__device__ __forceinline__ void run_section(const Params& p, float (&v)[N], int k, int c,
                                            int64_t t, int64_t ti, int64_t nt, uint32_t epoch,
                                            float2* s_agg, double2* s_Z, bool zf_owner, int mq,
                                            float* zf_out, float* s_own) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Coef32* cf = p.c32 + ((int64_t)c * p.kmax + k);
    const float4 ab = __ldg(&cf->ab);
    const float a1 = ab.x, a2 = ab.y, b1 = ab.z, b2 = ab.w;
    const float b0 = FACT ? 1.0f : __ldg(&cf->misc).x;

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
        const float4 P = __ldg(&cf->phi_pow[j]);
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
    if (lane == 31) s_agg[warp] = make_float2(S1, S2);
    __syncthreads();

    // S5: scan over the W warp aggregates (every warp redundantly)
    float A1 = 0.f, A2 = 0.f;
    if (lane < W) {
        const float2 a = s_agg[lane];
        A1 = a.x;
        A2 = a.y;
    }
#pragma unroll
    for (int r = 0; (1 << r) < W; ++r) {
        const int d = 1 << r;
        const float t1 = __shfl_up_sync(0xffffffffu, A1, d);
        const float t2 = __shfl_up_sync(0xffffffffu, A2, d);
        const float4 P = __ldg(&cf->psi_pow[r]);
        if (lane >= d && lane < W) {
            A1 = fmaf(P.x, t1, fmaf(P.y, t2, A1));
            A2 = fmaf(P.z, t1, fmaf(P.w, t2, A2));
        }
    }
    // zero-state state entering this warp (exclusive) and leaving the tile
    float WE1 = __shfl_sync(0xffffffffu, A1, warp > 0 ? warp - 1 : 0);
    float WE2 = __shfl_sync(0xffffffffu, A2, warp > 0 ? warp - 1 : 0);
    if (warp == 0) {
        WE1 = 0.f;
        WE2 = 0.f;
    }

    if (warp == 0) {
        const float C1 = __shfl_sync(0xffffffffu, A1, W - 1);
        const float C2 = __shfl_sync(0xffffffffu, A2, W - 1);
        const Coef64* cc = p.c64 + ((int64_t)c * p.kmax + k);
        const bool has_succ = ti + 1 < nt;
        const size_t slot = (size_t)k * p.cap_tiles + (size_t)t;
        double2 Z;
        if (ti == 0) {
            Z = make_double2(0.0, 0.0);
            if (p.zi) {
                const double gi = cc->Ginv;
                Z.x = (double)p.zi[((int64_t)c * p.kmax + k) * 2 + 0] * gi;
                Z.y = (double)p.zi[((int64_t)c * p.kmax + k) * 2 + 1] * gi;
            }
        } else {
            if (has_succ && lane == 0) {
                st_relaxed_f64x2(p.agg + slot, make_double2((double)C1, (double)C2));
                st_release_u32(p.flags + slot, (epoch << 2) | kFlagAgg);
            }
            Z = lookback(p, t, ti, k, epoch, cc);
        }
        if (has_succ && lane == 0) {
            const double2 P = compose_horner(cc->theta, Z.x, Z.y, (double)C1, (double)C2);
            st_relaxed_f64x2(p.inc + slot, P);
            st_release_u32(p.flags + slot, (epoch << 2) | kFlagInc);
        }
        if (lane == 0) *s_Z = Z;
    }
    __syncthreads();
    const double2 Zt = *s_Z;

    // fold: state entering this warp, then this lane
    const float z1 = (float)Zt.x, z2 = (float)Zt.y;
    const float4 Pw = __ldg(&cf->psi_w[warp]);
    const float Zw1 = fmaf(Pw.x, z1, fmaf(Pw.y, z2, WE1));
    const float Zw2 = fmaf(Pw.z, z1, fmaf(Pw.w, z2, WE2));
    const float4 Pl = __ldg(&cf->lane_pow[lane]);
    const float zin1 = fmaf(Pl.x, Zw1, fmaf(Pl.y, Zw2, E1));
    const float zin2 = fmaf(Pl.z, Zw1, fmaf(Pl.w, Zw2, E2));

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
        float f1, f2;
        if (mq >= 1) {
            f1 = fmaf(b1, xq, fmaf(b2, xqm1, fmaf(-a1, yq, -a2 * yqm1)));
        } else {
            f1 = fmaf(b1, xq, fmaf(-a1, yq, zin2));
        }
        f2 = fmaf(b2, xq, -a2 * yq);
        const float G = FACT ? __ldg(&cf->misc).y : 1.0f;
        zf_out[((int64_t)c * p.kmax + k) * 2 + 0] = f1 * G;
        zf_out[((int64_t)c * p.kmax + k) * 2 + 1] = f2 * G;
    }
}

template <int N, int W>
__global__ void __launch_bounds__(W * 32) sos_forward_kernel(Params p) {
    using KT = FwdKernel<N, W>;
    using S = Swz<N>;
    extern __shared__ float4 s_tile4[];
    float* s_tile = reinterpret_cast<float*>(s_tile4);
    __shared__ float2 s_agg[W];
    __shared__ double2 s_Z;
    __shared__ int64_t s_t;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t epoch = *reinterpret_cast<volatile uint32_t*>(&p.hdr->epoch);
    const int64_t total = p.hdr->total_tiles;

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

    for (;;) {
        if (tid == 0) s_t = (int64_t)atomicAdd(&p.hdr->tile_counter, 1u);
        __syncthreads();
        const int64_t t = s_t;
        if (t >= total) break;

        // channel of tile t: the largest c with tb[c] <= t
        int lo = 0, hi = p.C - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.tb[mid]) <= t) lo = mid; else hi = mid - 1;
        }
        const int c = lo;
        const ChanInfo ci = p.chan[c];
        const int64_t ti = t - __ldg(&p.tb[c]);
        const int64_t nt = ci.ntiles;
        const int64_t start = ti * KT::kTile;
        const int64_t rem = ci.len - start;
        const int r = (int)(rem < KT::kTile ? rem : KT::kTile);  // valid samples
        const float* src = p.x + ci.off + start;

        // S2: global -> shared (swizzled), zero beyond the channel end
        const bool vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && r == KT::kTile;
        if (vec) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll 4
            for (int g = tid; g < KT::kGran; g += KT::kThreads) s_tile4[S::g(g)] = __ldcs(s4 + g);
        } else {
            for (int j = tid; j < KT::kTile; j += KT::kThreads)
                s_tile[S::e(j)] = j < r ? __ldcs(src + j) : 0.0f;
        }
        __syncthreads();
        float v[N];
        const int chunk = warp * 32 + lane;
#pragma unroll
        for (int g = 0; g < N / 4; ++g) {
            const float4 q = s_tile4[S::g(chunk * (N / 4) + g)];
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

        // the owner's scratch: its own chunk of the tile buffer, unused while
        // the sections run (plain layout, only that lane touches it)
        float* s_own = s_tile + chunk * N;
        if (ci.mode) {
            for (int k = 0; k < ci.K; ++k)
                run_section<N, W, true>(p, v, k, c, t, ti, nt, epoch, s_agg, &s_Z, zf_owner, mq,
                                        p.zf, s_own);
            const float G = __ldg(&p.c32[(int64_t)c * p.kmax + ci.K - 1].misc).y;
#pragma unroll
            for (int m = 0; m < N; ++m) v[m] *= G;
        } else {
            for (int k = 0; k < ci.K; ++k)
                run_section<N, W, false>(p, v, k, c, t, ti, nt, epoch, s_agg, &s_Z, zf_owner, mq,
                                         p.zf, s_own);
        }

        // S7: registers -> shared (swizzled) -> global
        __syncwarp();  // order the zf owner's scratch writes before the lanes' stores
#pragma unroll
        for (int g = 0; g < N / 4; ++g)
            s_tile4[S::g(chunk * (N / 4) + g)] =
                make_float4(v[4 * g + 0], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
        __syncthreads();
        float* dst = p.y + ci.off + start;
        if (((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) && r == KT::kTile) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 4
            for (int g = tid; g < KT::kGran; g += KT::kThreads) __stcs(d4 + g, s_tile4[S::g(g)]);
        } else {
            for (int j = tid; j < r; j += KT::kThreads) __stcs(dst + j, s_tile[S::e(j)]);
        }
        __syncthreads();
    }

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

#define SOSF_ENTRY(N_, W_) \
    {N_, W_, reinterpret_cast<const void*>(&sos_forward_kernel<N_, W_>), FwdKernel<N_, W_>::kSmem}

static const KernelEntry kEntries[] = {
    SOSF_ENTRY(16, 8), SOSF_ENTRY(16, 16), SOSF_ENTRY(32, 4), SOSF_ENTRY(32, 8),
    SOSF_ENTRY(32, 16), SOSF_ENTRY(64, 4), SOSF_ENTRY(64, 8),
};

bool forward_supported(int N, int W) {
    for (const auto& e : kEntries)
        if (e.N == N && e.W == W) return true;
    return false;
}

cudaError_t launch_forward(const Params& p, int64_t host_tiles, cudaStream_t stream) {
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
        if (ke->smem > 48 * 1024) {
            err = cudaFuncSetAttribute(ke->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ke->smem);
            if (err != cudaSuccess) return err;
        }
        int occ = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ke->fn, p.W * 32, ke->smem);
        if (err != cudaSuccess) return err;
        s_occ[dev][idx] = occ > 0 ? occ : 1;
    }
    int64_t grid = (int64_t)s_sms[dev] * s_occ[dev][idx];
    if (host_tiles < grid) grid = host_tiles;
    if (grid < 1) return cudaSuccess;
    void* args[] = {const_cast<Params*>(&p)};
    return cudaLaunchKernel(ke->fn, dim3((unsigned)grid), dim3(p.W * 32), args, ke->smem, stream);
}

}  // namespace sosf
