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
// output afterwards would cancel most of the digits.  So the adjoint pipeline
// walks each segment's groups from the top of time down, the loader reverses
// every group into its slot, and each section's stage runs the forward
// section code twice (lambda and dL/du) with the forward tables.  The segment's
// u and y of every section come from the forward pass that the backward call
// runs first (the section pipeline with `inter` set).  A channel within its
// memory horizon needs the adjoint from P samples above each segment (zero
// state there, the same horizon: the adjoint's impulse response is the
// forward's, reversed); a channel without one is a single segment.
#include "sos_pipe.cuh"
#include "pipe_section.cuh"

namespace sosf {

// Segment geometry of the backward walk: groups tile [.., top) downwards.
struct BwdGeom {
    int64_t top;  // one past the highest sample computed
    int ngroups;
    bool at_end;  // top is the channel's end: the adjoint starts from dL/dzf
};

template <int kGroup>
__device__ __forceinline__ BwdGeom bwd_geom(const SegGeom& sg) {
    BwdGeom b;
    const int64_t t = sg.out_hi + sg.horizon;
    b.at_end = sg.out_hi == sg.len || t >= sg.len;
    b.top = b.at_end ? sg.len : t;
    b.ngroups = (int)((b.top - sg.out_lo + kGroup - 1) / kGroup);
    return b;
}

template <int N>
__global__ void __launch_bounds__(kPipeThreads, 2) sos_adjoint_kernel(Params p) {
    using PC = PipeCfg<N>;
    using SL = SlotLayout<N>;
    extern __shared__ float4 s_ring4[];
    float* ring = reinterpret_cast<float*>(s_ring4);
    __shared__ PipeShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = p.hdr->total_pipe;

    for (int i = tid; i < kPipeRing; i += blockDim.x) {
        for (int j = 0; j < kPipeStages; ++j) mbar_init(&sh.bar[i][j], 32);
        mbar_init(&sh.free_[i], 32);
    }
    __syncthreads();

    int s = 0;
    unsigned use = 0;
    if (warp == 0) {
        // ---- loader: dL/dy of the groups, top down ----
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            const BwdGeom bg = bwd_geom<PC::kGroup>(sg);
            for (int g = 0; g < bg.ngroups; ++g) {
                if (use > 0) pipe_wait(p, &sh.free_[s], (use - 1) & 1u, lane);
                // the group [gb, gb + G) goes into the slot reversed: slot
                // element i holds sample gb + G - 1 - i
                const int64_t gb = bg.top - (int64_t)(g + 1) * PC::kGroup;
                float* slot = ring + s * SL::kFloats;
                const float* src = p.gy + sg.off + gb;
                for (int i = lane; i < PC::kGroup; i += 32) {
                    const int j = PC::kGroup - 1 - i;
                    const bool ok = gb + j >= 0;
                    cp_async4(slot + SL::elem(i), ok ? src + j : p.gy + sg.off, ok);
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
        // ---- storer: dL/dx of the segment's own samples ----
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            const BwdGeom bg = bwd_geom<PC::kGroup>(sg);
            for (int g = 0; g < bg.ngroups; ++g) {
                pipe_wait(p, &sh.bar[s][kMaxSections], use & 1u, lane);
                const int64_t gb = bg.top - (int64_t)(g + 1) * PC::kGroup;
                const int64_t a0 = sg.out_lo - gb, b0 = sg.out_hi - gb;
                const int lo = (int)(a0 > 0 ? a0 : 0);
                const int hi = (int)(b0 < PC::kGroup ? b0 : PC::kGroup);
                const float* slot = ring + s * SL::kFloats;
                float* dst = p.gx + sg.off + gb;
                for (int j = lo + lane; j < hi; j += 32)
                    __stcs(dst + j, slot[SL::elem(PC::kGroup - 1 - j)]);
                __syncwarp();
                pipe_arrive(&sh.free_[s]);
                if (++s == kPipeRing) {
                    s = 0;
                    ++use;
                }
            }
        }
    } else {
        // ---- stage j = warp - 1: section k = 7 - j (the top section first) ----
        const int j = warp - 1;
        const int k = kMaxSections - 1 - j;
        int cur_c = -1;
        float4 ab = make_float4(0.f, 0.f, 0.f, 0.f), br = ab, lp = ab;
        for (int64_t d = blockIdx.x; d < total; d += gridDim.x) {
            const SegGeom sg = seg_geom<PC::kGroup>(p, d);
            const BwdGeom bg = bwd_geom<PC::kGroup>(sg);
            if (k >= sg.K) {
                for (int g = 0; g < bg.ngroups; ++g) {
                    pipe_wait(p, &sh.bar[s][j], use & 1u, lane);
                    pipe_arrive(&sh.bar[s][j + 1]);
                    if (++s == kPipeRing) {
                        s = 0;
                        ++use;
                    }
                }
                continue;
            }
            if (sg.c != cur_c) {
                const Coef32* cf = p.c32 + (int64_t)sg.c * p.kmax + k;
                ab = __ldg(&cf->ab);
                br = __ldg(&cf->braw);
                lp = __ldg(&cf->lane_pow[lane]);
                __syncwarp();
                if (lane < 5) sh.phi[k][lane] = __ldg(&cf->phi_pow[lane]);
                __syncwarp();
                cur_c = sg.c;
            }
            const float a1 = ab.x, a2 = ab.y, b0 = br.x, b1 = br.y, b2 = br.z;
            const float4 ab_l = make_float4(a1, a2, 0.f, 0.f);  // all-pole part
            const float4 ab_u = make_float4(a1, a2, b1, b2);    // whole section
            // reversed-time DF2T states at the top: from dL/dzf at the
            // channel's end, zero at the top of a warm-up.  lambda's previous
            // two values (lambda_{n+1}, lambda_{n+2} of the first sample) are
            // dL/dzf there too.
            float g1 = 0.f, g2 = 0.f;
            if (bg.at_end && p.gzf) {
                g1 = p.gzf[((int64_t)sg.c * p.kmax + k) * 2 + 0];
                g2 = p.gzf[((int64_t)sg.c * p.kmax + k) * 2 + 1];
            }
            float Zl1 = fmaf(-a1, g1, -a2 * g2), Zl2 = -a2 * g1;
            const float c1 = fmaf(-a1, b0, b1), c2 = fmaf(-a2, b0, b2);
            float Zu1 = fmaf(c1, g1, c2 * g2);
            float Zu2 = fmaf(c2, g1, fmaf(a1 * c2, g2, -a2 * c1 * g2));
            float q1 = g1, q2 = g2;  // lambda at the two reversed samples before the group
            float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            const float* u_base =
                (k == 0 ? p.x : p.inter + (int64_t)(k - 1) * p.total) + sg.off;
            const float* y_base = p.inter + (int64_t)k * p.total + sg.off;
            float* gzi_dst = p.gzi ? p.gzi + ((int64_t)sg.c * p.kmax + k) * 2 : nullptr;
            for (int g = 0; g < bg.ngroups; ++g) {
                pipe_wait(p, &sh.bar[s][j], use & 1u, lane);
                const int64_t gb = bg.top - (int64_t)(g + 1) * PC::kGroup;
                float* row = ring + s * SL::kFloats + lane * SL::kRow;
                float v[N], w[N];
#pragma unroll
                for (int q = 0; q < N / 4; ++q) {
                    const float4 t = *reinterpret_cast<const float4*>(row + 4 * q);
                    v[4 * q + 0] = t.x;
                    v[4 * q + 1] = t.y;
                    v[4 * q + 2] = t.z;
                    v[4 * q + 3] = t.w;
                }
#pragma unroll
                for (int m = 0; m < N; ++m) w[m] = v[m];
                // lambda (reversed): all-pole part; dL/du (reversed): section
                pipe_section<N, true>(w, ab_l, 1.f, sh.phi[k], lp, Zl1, Zl2, false, 0, row,
                                      nullptr, 1.f);
                pipe_section<N, false>(v, ab_u, b0, sh.phi[k], lp, Zu1, Zu2, false, 0, row,
                                       nullptr, 1.f);
                // reversed element m of this lane is sample n = nb - m; there
                // lambda_{n+1}, lambda_{n+2} are the reversed elements m-1,
                // m-2, the first two taken from the lane (or group) before
                const int64_t nb = gb + PC::kGroup - 1 - (int64_t)lane * N;
                float p1 = __shfl_up_sync(0xffffffffu, w[N - 1], 1);
                float p2 = __shfl_up_sync(0xffffffffu, w[N - 2], 1);
                if (lane == 0) {
                    p1 = q1;
                    p2 = q2;
                }
                q1 = __shfl_sync(0xffffffffu, w[N - 1], 31);
                q2 = __shfl_sync(0xffffffffu, w[N - 2], 31);
                const int64_t mlo = nb - (sg.out_hi - 1), mhi = nb - sg.out_lo;  // m in [mlo, mhi]
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    if (m >= mlo && m <= mhi) {
                        const float l0 = w[m];
                        const float l1 = m >= 1 ? w[m - 1] : p1;
                        const float l2 = m >= 2 ? w[m - 2] : (m == 1 ? p1 : p2);
                        const float u = __ldg(u_base + nb - m), y = __ldg(y_base + nb - m);
                        acc[0] = fmaf(l0, u, acc[0]);
                        acc[1] = fmaf(l1, u, acc[1]);
                        acc[2] = fmaf(l2, u, acc[2]);
                        acc[3] = fmaf(-l1, y, acc[3]);
                        acc[4] = fmaf(-l2, y, acc[4]);
                    }
                }
                // dL/dzi = (lambda_0, lambda_1): sample 0 is reversed element
                // m0 = nb of the lane holding it, sample 1 is m0 - 1
                if (gzi_dst && sg.si == 0 && nb >= 0 && nb < N) {
                    const int m0 = (int)nb;
#pragma unroll
                    for (int m = 0; m < N; ++m) row[m] = w[m];
                    gzi_dst[0] = row[m0];
                    gzi_dst[1] = m0 >= 1 ? row[m0 - 1] : p1;
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < N / 4; ++q)
                    *reinterpret_cast<float4*>(row + 4 * q) =
                        make_float4(v[4 * q + 0], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                __syncwarp();
                pipe_arrive(&sh.bar[s][j + 1]);
                if (++s == kPipeRing) {
                    s = 0;
                    ++use;
                }
            }
            // the segment's share of the coefficient sums
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                float a = acc[i];
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) atomicAdd(&p.gacc[((int64_t)sg.c * p.kmax + k) * 5 + i], (double)a);
            }
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

cudaError_t launch_adjoint(const Params& p, int64_t grid, double* grad_sos, cudaStream_t stream) {
    const void* fn = p.N == 16 ? SOSF_ADJ(16) : p.N == 32 ? SOSF_ADJ(32) : SOSF_ADJ(64);
    const size_t smem = sizeof(float) * 32 * (size_t)(p.N + 4) * kPipeRing;
    static bool attr[3] = {false, false, false};
    const int idx = p.N == 16 ? 0 : p.N == 32 ? 1 : 2;
    if (!attr[idx]) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[idx] = true;
    }
    if (grid >= 1) {
        void* args[] = {const_cast<Params*>(&p)};
        const cudaError_t e =
            cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kPipeThreads), args, smem, stream);
        if (e != cudaSuccess) return e;
    }
    const int64_t n = (int64_t)p.C * p.kmax;
    adjoint_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(p, grad_sos);
    return cudaGetLastError();
}

}  // namespace sosf
