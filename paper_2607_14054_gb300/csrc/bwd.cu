// Backward (adjoint) of the cascade: gradients of a loss L with respect to
// x, zi and every coefficient, given dL/dy and dL/dzf.
//
// Per normalised section (b0, b1, b2, a1, a2; DF2T state s, input u, output
// y) the forward step is s_{n+1} = A s_n + B u_n, y_n = s1_n + b0 u_n with
// A = [[-a1, 1], [-a2, 0]] (the banded-Toeplitz recurrence of Eq.
// recursive_equation_block_form).  Its transpose runs backwards in time: with
// g = dL/dy, the adjoint state mu_n = A^T mu_{n+1} + (g_n, 0), mu_T = dL/dzf,
// whose components are (lambda_n, lambda_{n+1}) for the time-reversed
// all-pole recursion lambda_n = g_n - a1 lambda_{n+1} - a2 lambda_{n+2}.  Then
//   dL/du_n = b0 lambda_n + b1 lambda_{n+1} + b2 lambda_{n+2}   (reversed FIR),
//   dL/db_j = sum_n lambda_{n+j} u_n,  dL/da_j = -sum_n lambda_{n+j} y_n,
//   dL/dzi  = mu_0 = (lambda_0, lambda_1),
// with lambda_T = dzf_1 and lambda_{T+1} = dzf_2.  Section k's dL/du is
// section k-1's dL/dy; section 0's is dL/dx.
//
// In reversed time m = T - 1 - n both recursions are forward ones: lambda
// is the all-pole part of the section run on the reversed g, and dL/du is the
// whole section (zeros first, then poles, like the forward pass) run on the
// reversed g from the DF2T state e = M dL/dzf, M = [[c1, c2], [c2, a1 c2 -
// a2 c1]], c_j = b_j - a_j b0.  Running the zeros first matters: the all-pole
// part alone can have a gain of 1e4 and more, and applying the zeros to its
// output afterwards would cancel most of the digits.
//
// One warp per segment (the warp-segment scheme of the forward), in two
// passes.  The forward pass runs the segment's groups through the cascade and
// keeps only each section's DF2T state at the start of every group the
// segment owns (checkpoints, 8 bytes per section and group).  The reverse
// pass walks the groups from the top of time down: per group it recomputes
// the K + 1 section signals from the checkpoint into shared memory, then runs
// the adjoint cascade on the reversed group (section K-1 first), accumulating
// the coefficient sums against the recomputed u and y and writing dL/dx.  No
// per-section intermediate leaves the SM.  A channel within its memory
// horizon needs the adjoint from P samples above each segment (zero state
// there: the adjoint's impulse response is the forward's, reversed) and the
// forward from P samples below; a channel without one is a single segment.
//
// Groups are anchored at the segment's top (the channel's end, or the end of
// the adjoint warm-up), so dL/dzf enters at a group boundary.  The channel's
// first group may then start before sample 0: its inputs there are zero and
// zi enters at the group-relative position of sample 0 (pipe_section's INJ).
#include "pipe_section.cuh"
#include "sos_pipe.cuh"

namespace sosf {

constexpr int kBwWarps = 1;  // warps per CTA (one: shared memory, not threads, bounds the CTAs per SM)
constexpr int kBwThreads = kBwWarps * 32;

template <int N>
struct BwCfg {
    static constexpr int kGroup = 32 * N;
    static constexpr int kRow = N + 4;
    static constexpr int kSlot = 32 * kRow;                  // floats per group slot
    static constexpr int kSig = (kMaxSections + 1) * kSlot;  // the K + 1 section signals
    static constexpr int kAcc = kMaxSections * 5 * 32;       // per-lane coefficient sums
    static constexpr int kWarpFloats = kSig + kSlot + kAcc;
    static constexpr size_t kSmem = sizeof(float) * (size_t)kWarpFloats * kBwWarps;
};

// Segment geometry of the backward: groups [top - (i + 1) G, top - i G),
// i = 0 .. n - 1, cover the forward warm-up below the segment, its own
// samples [out_lo, out_hi) and the adjoint warm-up above.
struct BwGeom {
    int64_t top;  // one past the highest sample of the top group
    int n;        // groups
    bool at_end;  // top is the channel's end: the adjoint starts from dL/dzf
};

template <int kGroup>
__device__ __forceinline__ BwGeom bw_geom(const SegGeom& sg) {
    BwGeom b;
    const int64_t t = sg.out_hi + sg.horizon;
    b.at_end = sg.out_hi == sg.len || t >= sg.len;
    b.top = b.at_end ? sg.len : t;
    const int64_t fstart = sg.si == 0 ? 0 : sg.out_lo - sg.horizon;  // forward warm-up start
    b.n = (int)((b.top - fstart + kGroup - 1) / kGroup);
    return b;
}

// Checkpoint slot of (channel c, segment si, group start gb > -G): distinct
// across channels (floor((off + gb + G) / G) + 2c grows by at least one from
// a channel's last group to the next channel's first) and between adjacent
// segments of one channel (parity of si), the only ones whose own groups
// meet.
template <int kGroup>
__device__ __forceinline__ int64_t ck_slot(const SegGeom& sg, int64_t gb) {
    return 2 * ((sg.off + gb + kGroup) / kGroup + 2 * (int64_t)sg.c) + (sg.si & 1);
}

// Asynchronous copies of the group [gb, gb + G) of one channel's array into a
// slot in forward layout (lane l's row holds samples [lN, lN + N)), zeros
// outside [0, len).
template <int N>
__device__ __forceinline__ void bw_load(const float* chan, int64_t gb, int64_t len, float* slot,
                                        int lane) {
    using BC = BwCfg<N>;
    const float* src = chan + gb;
    if (gb >= 0 && gb + BC::kGroup <= len && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int q = 0; q < BC::kGroup / 128; ++q) {
            const int g4 = q * 32 + lane;  // 16-byte granule in sample order
            cp_async16(slot + (g4 / (N / 4)) * BC::kRow + (g4 % (N / 4)) * 4, s4 + g4);
        }
    } else {
        for (int j = lane; j < BC::kGroup; j += 32) {
            const int64_t n = gb + j;
            const bool ok = n >= 0 && n < len;
            cp_async4(slot + (j / N) * BC::kRow + (j % N), ok ? chan + n : chan, ok);
        }
    }
    cp_async_commit();
}

// a lane row read back to front: the reversed chunk of the mirrored lane
template <int N>
__device__ __forceinline__ void row_load_rev(const float* row, float (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
        const float4 t = *reinterpret_cast<const float4*>(row + 4 * q);
        v[N - 1 - (4 * q + 0)] = t.x;
        v[N - 1 - (4 * q + 1)] = t.y;
        v[N - 1 - (4 * q + 2)] = t.z;
        v[N - 1 - (4 * q + 3)] = t.w;
    }
}

template <int N>
__device__ __forceinline__ void row_store_scaled(float* row, const float (&v)[N], float scale) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
        *reinterpret_cast<float4*>(row + 4 * q) =
            make_float4(v[4 * q + 0] * scale, v[4 * q + 1] * scale, v[4 * q + 2] * scale,
                        v[4 * q + 3] * scale);
}

template <int N>
__device__ __forceinline__ void row_store_rev(float* row, const float (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
        *reinterpret_cast<float4*>(row + 4 * q) =
            make_float4(v[N - 1 - (4 * q + 0)], v[N - 1 - (4 * q + 1)], v[N - 1 - (4 * q + 2)],
                        v[N - 1 - (4 * q + 3)]);
}

// The K sections forward over the group in sig[0] (a lane row each), from
// the states zs (left at the group's outgoing states); the true output of
// section k goes to sig[k + 1] when `keep`.  INJ: the channel's first group,
// zi entering at group-relative position pinj.
template <int N, bool FACT, bool INJ>
__device__ __forceinline__ void bw_forward_group(const Params& p, const SegGeom& sg, float* sig,
                                                 float2* zs, int lane, bool keep, int pinj) {
    using BC = BwCfg<N>;
    const Coef32* cf0 = p.c32 + (int64_t)sg.c * p.kmax;
    float v[N];
    row_to_chunk<N>(v, sig + lane * BC::kRow);
#pragma unroll 1
    for (int k = 0; k < sg.K; ++k) {
        const Coef32* cf = cf0 + k;
        const float4 ab = cf->ab;
        const float b0 = FACT ? 1.f : cf->misc.x;
        const float4 lp = cf->lane_pow[lane];
        float2 z = zs[k];
        if (INJ) {
            float zi1 = 0.f, zi2 = 0.f;
            if (p.zi) {
                const float gi = FACT ? cf->misc.z : 1.f;
                zi1 = p.zi[((int64_t)sg.c * p.kmax + k) * 2 + 0] * gi;
                zi2 = p.zi[((int64_t)sg.c * p.kmax + k) * 2 + 1] * gi;
            }
            pipe_section<N, FACT, false, true>(v, ab, b0, cf->phi_pow, lp, z.x, z.y, false, 0,
                                               nullptr, nullptr, 1.f, pinj, zi1, zi2);
        } else {
            pipe_section<N, FACT, false>(v, ab, b0, cf->phi_pow, lp, z.x, z.y, false, 0, nullptr,
                                         nullptr, 1.f);
        }
        __syncwarp();
        if (lane == 0) zs[k] = z;
        if (keep)
            row_store_scaled<N>(sig + (k + 1) * BC::kSlot + lane * BC::kRow, v,
                                FACT ? cf->misc.y : 1.f);
    }
    __syncwarp();
}

template <int N>
__device__ __forceinline__ void bw_forward_group_any(const Params& p, const SegGeom& sg,
                                                     float* sig, float2* zs, int lane, bool keep,
                                                     bool fact, bool inj, int pinj) {
    if (fact) {
        if (inj) bw_forward_group<N, true, true>(p, sg, sig, zs, lane, keep, pinj);
        else bw_forward_group<N, true, false>(p, sg, sig, zs, lane, keep, 0);
    } else {
        if (inj) bw_forward_group<N, false, true>(p, sg, sig, zs, lane, keep, pinj);
        else bw_forward_group<N, false, false>(p, sg, sig, zs, lane, keep, 0);
    }
}

template <int N>
__global__ void __launch_bounds__(kBwThreads) sos_adjoint_kernel(Params p) {
    using BC = BwCfg<N>;
    constexpr int G = BC::kGroup;
    extern __shared__ float4 s_bw4[];
    __shared__ float2 s_zf[kBwWarps][kMaxSections];     // forward states
    __shared__ float s_za[kBwWarps][kMaxSections][6];   // adjoint: lambda, dL/du states; lambda above
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* base = reinterpret_cast<float*>(s_bw4) + (size_t)w * BC::kWarpFloats;
    float* sig = base;                  // [K + 1][32][N + 4]
    float* gslot = base + BC::kSig;     // dL/dy of the group, then dL/dx
    float* acc = gslot + BC::kSlot;     // [kMaxSections][5][32]
    float2* zs = s_zf[w];
    const int64_t total = p.hdr->total_pipe;
    const int64_t nw = (int64_t)gridDim.x * kBwWarps;

    int64_t d = (int64_t)blockIdx.x * kBwWarps + w;
    while (d < total) {
        const SegGeom sg = seg_geom<G>(p, d);
        const BwGeom bg = bw_geom<G>(sg);
        const int K = sg.K;
        const float* xc = p.x + sg.off;
        const float* gc = p.gy + sg.off;
        float* dxc = p.gx + sg.off;
        const bool fact = p.chan[sg.c].mode != 0;
        const int64_t gb_low = bg.top - (int64_t)bg.n * G;  // the lowest group's start
        if (K == 0) {
            // identity channel: dL/dx = dL/dy on the segment's own samples
            for (int64_t i = sg.out_lo + lane; i < sg.out_hi; i += 32) dxc[i] = __ldg(gc + i);
        } else {
            // ---- forward pass: checkpoints at the start of every own group ----
            __syncwarp();
            if (lane < K) zs[lane] = make_float2(0.f, 0.f);
            __syncwarp();
            for (int i = bg.n - 1; i >= 0; --i) {
                const int64_t gb = bg.top - (int64_t)(i + 1) * G;
                if (gb >= sg.out_hi) break;  // above the own samples: adjoint warm-up only
                bw_load<N>(xc, gb, sg.len, sig, lane);
                if (gb + G > sg.out_lo && lane < K) {
                    float2* ck = reinterpret_cast<float2*>(p.ck) + ck_slot<G>(sg, gb) * p.kmax;
                    ck[lane] = zs[lane];
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                __syncwarp();
                bw_forward_group_any<N>(p, sg, sig, zs, lane, false, fact,
                                        sg.si == 0 && gb == gb_low, (int)-gb);
            }
            // ---- reverse pass ----
            for (int i = lane; i < kMaxSections * 5 * 32; i += 32) acc[i] = 0.f;
            if (lane < K) {
                const Coef32* cf = p.c32 + (int64_t)sg.c * p.kmax + lane;
                const float a1 = cf->ab.x, a2 = cf->ab.y;
                const float b0 = cf->braw.x, b1 = cf->braw.y, b2 = cf->braw.z;
                float g1 = 0.f, g2 = 0.f;
                if (bg.at_end && p.gzf) {
                    g1 = p.gzf[((int64_t)sg.c * p.kmax + lane) * 2 + 0];
                    g2 = p.gzf[((int64_t)sg.c * p.kmax + lane) * 2 + 1];
                }
                const float c1 = fmaf(-a1, b0, b1), c2 = fmaf(-a2, b0, b2);
                float* za = s_za[w][lane];
                za[0] = fmaf(-a1, g1, -a2 * g2);  // lambda's reversed DF2T state
                za[1] = -a2 * g1;
                za[2] = fmaf(c1, g1, c2 * g2);    // dL/du's: M dL/dzf
                za[3] = fmaf(c2, g1, fmaf(a1 * c2, g2, -a2 * c1 * g2));
                za[4] = g1;                       // lambda at the two samples above
                za[5] = g2;
            }
            __syncwarp();
            float* gzi_c = p.gzi ? p.gzi + (int64_t)sg.c * p.kmax * 2 : nullptr;
            for (int i = 0; i < bg.n; ++i) {
                const int64_t gb = bg.top - (int64_t)(i + 1) * G;
                const bool own = gb < sg.out_hi && gb + G > sg.out_lo;
                bw_load<N>(gc, gb, sg.len, gslot, lane);
                if (own) bw_load<N>(xc, gb, sg.len, sig, lane);
                if (own && lane < K) {
                    const float2* ck =
                        reinterpret_cast<const float2*>(p.ck) + ck_slot<G>(sg, gb) * p.kmax;
                    zs[lane] = ck[lane];
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                __syncwarp();
                // the K + 1 section signals of this group, from its checkpoint
                if (own)
                    bw_forward_group_any<N>(p, sg, sig, zs, lane, true, fact,
                                            sg.si == 0 && gb == gb_low, (int)-gb);
                // reversed lane l is the forward row 31 - l read back to front:
                // its element m is sample n = nb - m
                const int mirror = 31 - lane;
                const int64_t nb = gb + G - 1 - (int64_t)lane * N;
                const int64_t mlo = nb - (sg.out_hi - 1), mhi = nb - sg.out_lo;  // own m
                float v[N];
                row_load_rev<N>(gslot + mirror * BC::kRow, v);
#pragma unroll 1
                for (int k = K - 1; k >= 0; --k) {
                    const Coef32* cf = p.c32 + (int64_t)sg.c * p.kmax + k;
                    const float4 ab = cf->ab;
                    const float4 br = cf->braw;
                    const float4 lp = cf->lane_pow[lane];
                    float* za = s_za[w][k];
                    float zl1 = za[0], zl2 = za[1], zu1 = za[2], zu2 = za[3];
                    const float q1 = za[4], q2 = za[5];
                    float lw[N];
#pragma unroll
                    for (int m = 0; m < N; ++m) lw[m] = v[m];
                    // lambda (reversed): all-pole part; dL/du (reversed): the
                    // whole section; one fused pass
                    pipe_section_dual<N>(lw, v, ab.x, ab.y, br.x, br.y, br.z, cf->phi_pow, lp,
                                         zl1, zl2, zu1, zu2);
                    // lambda_{n+1}, lambda_{n+2} of element m are elements m-1,
                    // m-2, the first two from the lane (or group) before
                    float p1 = __shfl_up_sync(0xffffffffu, lw[N - 1], 1);
                    float p2 = __shfl_up_sync(0xffffffffu, lw[N - 2], 1);
                    if (lane == 0) {
                        p1 = q1;
                        p2 = q2;
                    }
                    const float nq1 = __shfl_sync(0xffffffffu, lw[N - 1], 31);
                    const float nq2 = __shfl_sync(0xffffffffu, lw[N - 2], 31);
                    if (own) {
                        float u[N], y[N];
                        row_load_rev<N>(sig + k * BC::kSlot + mirror * BC::kRow, u);
                        row_load_rev<N>(sig + (k + 1) * BC::kSlot + mirror * BC::kRow, y);
                        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
                        for (int m = 0; m < N; ++m) {
                            if (m >= mlo && m <= mhi) {
                                const float l0 = lw[m];
                                const float l1 = m >= 1 ? lw[m - 1] : p1;
                                const float l2 = m >= 2 ? lw[m - 2] : (m == 1 ? p1 : p2);
                                s0 = fmaf(l0, u[m], s0);
                                s1 = fmaf(l1, u[m], s1);
                                s2 = fmaf(l2, u[m], s2);
                                s3 = fmaf(-l1, y[m], s3);
                                s4 = fmaf(-l2, y[m], s4);
                            }
                        }
                        float* a = acc + k * 5 * 32 + lane;
                        a[0] += s0;
                        a[32] += s1;
                        a[64] += s2;
                        a[96] += s3;
                        a[128] += s4;
                    }
                    // dL/dzi = (lambda_0, lambda_1): sample 0 is element nb of
                    // the lane with 0 <= nb < N
                    if (gzi_c && sg.si == 0 && nb >= 0 && nb < N) {
                        const int m0 = (int)nb;
                        float l0, l1;
                        pick_pair<N>(lw, m0, l0, l1);
                        gzi_c[k * 2 + 0] = l0;
                        gzi_c[k * 2 + 1] = m0 >= 1 ? l1 : p1;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        za[0] = zl1;
                        za[1] = zl2;
                        za[2] = zu1;
                        za[3] = zu2;
                        za[4] = nq1;
                        za[5] = nq2;
                    }
                    __syncwarp();
                }
                // dL/dx of the own samples: back into the slot in forward
                // order, then coalesced stores
                if (own) {
                    row_store_rev<N>(gslot + mirror * BC::kRow, v);
                    __syncwarp();
                    const int64_t a0 = sg.out_lo - gb, b0 = sg.out_hi - gb;
                    const int lo = (int)(a0 > 0 ? a0 : 0), hi = (int)(b0 < G ? b0 : G);
                    for (int j = lo + lane; j < hi; j += 32)
                        __stcs(dxc + gb + j, gslot[(j / N) * BC::kRow + (j % N)]);
                }
                __syncwarp();
            }
            // the segment's share of the coefficient sums
            for (int k = 0; k < K; ++k) {
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    float a = acc[(k * 5 + q) * 32 + lane];
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    if (lane == 0)
                        atomicAdd(&p.gacc[((int64_t)sg.c * p.kmax + k) * 5 + q], (double)a);
                }
            }
            __syncwarp();
        }
        // the next segment, as warps come free
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&p.hdr->seg_next, 1ull);
        d = nw + (int64_t)__shfl_sync(0xffffffffu, t, 0);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the last warp to finish resets the hand-out for the next launch
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

// dL/d(raw sos row) from the sums for the normalised coefficients (b_j =
// B_j / A0, a_j = A_j / A0), zero for sections past K; dL/dzi of sections
// past K is zero, and an empty channel passes dL/dzf through to dL/dzi.
__global__ void adjoint_finalize_kernel(Params p, double* grad_sos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)p.C * p.kmax) return;
    const int c = (int)(i / p.kmax), k = (int)(i % p.kmax);
    const ChanInfo ci = p.chan[c];
    double* g = grad_sos + i * 6;
    const bool on = k < ci.K && ci.len > 0;
    if (on) {
        const double* r = p.sos + i * 6;
        const double ia0 = 1.0 / r[3];
        const double* a = p.gacc + i * 5;
        const double b0 = r[0] * ia0, b1 = r[1] * ia0, b2 = r[2] * ia0;
        const double a1 = r[4] * ia0, a2 = r[5] * ia0;
        g[0] = a[0] * ia0;
        g[1] = a[1] * ia0;
        g[2] = a[2] * ia0;
        g[4] = a[3] * ia0;
        g[5] = a[4] * ia0;
        g[3] = -(b0 * a[0] + b1 * a[1] + b2 * a[2] + a1 * a[3] + a2 * a[4]) * ia0;
    } else {
        for (int q = 0; q < 6; ++q) g[q] = 0.0;
    }
    if (p.gzi && !on) {
        const bool pass = k < ci.K && ci.len == 0 && p.gzf;
        p.gzi[i * 2 + 0] = pass ? p.gzf[i * 2 + 0] : 0.f;
        p.gzi[i * 2 + 1] = pass ? p.gzf[i * 2 + 1] : 0.f;
    }
}

#define SOSF_ADJ(N_) reinterpret_cast<const void*>(&sos_adjoint_kernel<N_>)

namespace {
const void* adj_fn(int N) { return N == 16 ? SOSF_ADJ(16) : N == 32 ? SOSF_ADJ(32) : SOSF_ADJ(64); }
size_t adj_smem(int N) {
    return N == 16 ? BwCfg<16>::kSmem : N == 32 ? BwCfg<32>::kSmem : BwCfg<64>::kSmem;
}
}  // namespace

// warps of the adjoint kernel resident on the device (0 on error)
int64_t adjoint_warps(int N, int sms) {
    static int s_occ[3] = {0, 0, 0};
    const int idx = N == 16 ? 0 : N == 32 ? 1 : 2;
    if (s_occ[idx] == 0) {
        if (cudaFuncSetAttribute(adj_fn(N), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)adj_smem(N)) != cudaSuccess)
            return 0;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adj_fn(N), kBwThreads,
                                                          adj_smem(N)) != cudaSuccess)
            return 0;
        s_occ[idx] = occ;
    }
    return (int64_t)sms * s_occ[idx] * kBwWarps;
}

// checkpoint slots the adjoint kernel may use (see ck_slot)
int64_t adjoint_ck_slots(int N, int64_t total_len, int32_t C) {
    const int64_t G = 32LL * N;
    return 2 * ((total_len + 2 * G) / G + 2 * (int64_t)C + 2);
}

cudaError_t launch_adjoint(const Params& p, int sms, double* grad_sos, cudaStream_t stream) {
    const int64_t warps = adjoint_warps(p.N, sms);
    if (warps < 1) return cudaErrorInvalidConfiguration;
    if (p.total > 0) {
        const cudaError_t e = launch_params(adj_fn(p.N), warps / kBwWarps, kBwThreads,
                                            adj_smem(p.N), p, stream, false);
        if (e != cudaSuccess) return e;
    }
    const int64_t n = (int64_t)p.C * p.kmax;
    adjoint_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(p, grad_sos);
    return cudaGetLastError();
}

}  // namespace sosf
