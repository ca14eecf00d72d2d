// The comparison algorithms of the paper's evaluation (Sec. VIII) on the
// same segmentation as the method: each channel cut into segments of
// seg_len outputs, each segment computed from its channel's memory horizon P
// earlier (zero state there; the channel's zi for its first segment), so
// that all four algorithms (scalar, block, PH, cyclic reduction) share the
// parallel decomposition and differ only in how a segment is filtered.
//
//  * scalar (Sec. II, Eq. complex_second_order): one thread per segment, the
//    sections' transposed-direct-form-II recursions sample by sample (the
//    sequential dependency chain of depth equal to the segment length);
//  * block filtering (Sec. IV, Eq. block_filtering_equation): one warp per
//    segment, blocks of L = 32 samples (one per lane); per block and section
//    y_n = H x_n + H_b xbar_{n-1} - H_a ybar_{n-1}, H the lower-triangular
//    Toeplitz matrix of the section's first L impulse-response samples, the
//    boundary terms from the previous block's last two inputs and outputs:
//    L + 4 block FMAs per block, each lane computing its own row.
#include "sos_common.cuh"

namespace sosf {

struct CmpSeg {
    int64_t off, len, out_lo, out_hi, cstart;
    int c, K;
    bool first, last;
};

// segment s of channel c (false if c has fewer segments)
__device__ __forceinline__ bool cmp_seg(const Params& p, int c, int64_t s, int64_t seg_len,
                                        CmpSeg& g) {
    const ChanInfo ci = p.chan[c];
    const int64_t P = ci.horizon;
    const int64_t L = ci.len;
    const int64_t sl = P < 0 ? (L > 0 ? L : 1) : seg_len;  // no horizon: one segment
    const int64_t ns = L > 0 ? (L + sl - 1) / sl : 1;      // an empty channel: one empty one
    if (s >= ns) return false;
    g.c = c;
    g.off = ci.off;
    g.len = L;
    g.K = ci.K;
    g.out_lo = s * sl;
    g.out_hi = g.out_lo + sl < L ? g.out_lo + sl : L;
    // warm-up from zero state P samples early; with an initial state, a
    // segment whose warm-up would start within the plan's first segment of
    // the channel (which the plan made long enough for the initial state's
    // response to die out) starts at the channel's start from zi instead
    g.cstart = s == 0 ? 0 : g.out_lo - P;
    g.first = s == 0;
    if (g.cstart < 0) g.cstart = 0;
    if (p.zi && s > 0 && g.cstart < ci.seg) {
        g.cstart = 0;
        g.first = true;
    }
    g.last = g.out_hi == L;
    return true;
}

// ---------------------------------------------------------------------------
// scalar: one thread per segment
// ---------------------------------------------------------------------------
__global__ void sos_scalar_kernel(Params p, int64_t seg_len) {
    const int c = blockIdx.y;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    CmpSeg g;
    if (!cmp_seg(p, c, s, seg_len, g)) return;
    const Coef32* cf = p.c32 + (int64_t)c * p.kmax;
    float b0[kMaxSections], b1[kMaxSections], b2[kMaxSections], a1[kMaxSections],
        a2[kMaxSections], z1[kMaxSections], z2[kMaxSections];
#pragma unroll
    for (int k = 0; k < kMaxSections; ++k) {
        if (k < g.K) {
            const float4 br = cf[k].braw, ab = cf[k].ab;
            b0[k] = br.x;
            b1[k] = br.y;
            b2[k] = br.z;
            a1[k] = ab.x;
            a2[k] = ab.y;
            z1[k] = g.first && p.zi ? p.zi[((int64_t)c * p.kmax + k) * 2 + 0] : 0.f;
            z2[k] = g.first && p.zi ? p.zi[((int64_t)c * p.kmax + k) * 2 + 1] : 0.f;
        } else {
            b0[k] = 1.f;
            b1[k] = b2[k] = a1[k] = a2[k] = z1[k] = z2[k] = 0.f;
        }
    }
    const float* x = p.x + g.off;
    float* y = p.y + g.off;
    for (int64_t n = g.cstart; n < g.out_hi; ++n) {
        float v = __ldg(x + n);
#pragma unroll
        for (int k = 0; k < kMaxSections; ++k) {
            if (k < g.K) {
                const float o = fmaf(b0[k], v, z1[k]);
                z1[k] = fmaf(b1[k], v, fmaf(-a1[k], o, z2[k]));
                z2[k] = fmaf(b2[k], v, -a2[k] * o);
                v = o;
            }
        }
        if (n >= g.out_lo) y[n] = v;
    }
    // the final state (sections past K: zero; an empty channel keeps zi)
    if (g.last && p.zf)
#pragma unroll
        for (int k = 0; k < kMaxSections; ++k) {
            if (k >= p.kmax) break;
            p.zf[((int64_t)c * p.kmax + k) * 2 + 0] = k < g.K ? z1[k] : 0.f;
            p.zf[((int64_t)c * p.kmax + k) * 2 + 1] = k < g.K ? z2[k] : 0.f;
        }
}

// ---------------------------------------------------------------------------
// block filtering: one warp per segment, L = 32
// ---------------------------------------------------------------------------
constexpr int kBlkWarps = 4;

__global__ void __launch_bounds__(kBlkWarps * 32) sos_block_kernel(Params p, int64_t seg_len) {
    // per warp and section the section's first L impulse-response samples
    // behind L zeros, hpad[k][32 + i] = h[i]: lane l reads column j of H,
    // h[l - j], at hpad[k][32 + l - j] (consecutive lanes, consecutive words)
    extern __shared__ float s_blk[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.y;
    const int64_t s = (int64_t)blockIdx.x * kBlkWarps + w;
    CmpSeg g;
    if (!cmp_seg(p, c, s, seg_len, g)) return;
    float* hpad = s_blk + (size_t)w * kMaxSections * 64;
    const Coef32* cf = p.c32 + (int64_t)c * p.kmax;
    // H_b, H_a rows and the all-pole response g[l], g[l - 1] of this lane,
    // per section: g from the recursion (lane 0, 32 steps), shared through
    // the first column slot, then h[l - j] for every column
    float hb0[kMaxSections], hb1[kMaxSections], ha0[kMaxSections], ha1[kMaxSections],
        g0[kMaxSections], g1[kMaxSections];
#pragma unroll
    for (int k = 0; k < kMaxSections; ++k) {
        hb0[k] = hb1[k] = ha0[k] = ha1[k] = g0[k] = g1[k] = 0.f;
        if (k >= g.K) continue;
        const float4 br = cf[k].braw, ab = cf[k].ab;
        float* hk = hpad + k * 64;
        if (lane == 0) {
            float q2 = 0.f, q1 = 0.f;  // g[n-2], g[n-1]
            for (int n = 0; n < 32; ++n) {
                const float gn = fmaf(-ab.x, q1, fmaf(-ab.y, q2, n == 0 ? 1.f : 0.f));
                hk[32 + n] = gn;  // g for now
                q2 = q1;
                q1 = gn;
            }
        }
        __syncwarp();
        const float gl = hk[32 + lane], glm1 = lane >= 1 ? hk[31 + lane] : 0.f,
                    glm2 = lane >= 2 ? hk[30 + lane] : 0.f;
        __syncwarp();
        // h[l] = b0 g[l] + b1 g[l-1] + b2 g[l-2]
        hk[lane] = 0.f;
        hk[32 + lane] = fmaf(br.x, gl, fmaf(br.y, glm1, br.z * glm2));
        // boundary terms: x[-2] -> b2 g[l]; x[-1] -> b1 g[l] + b2 g[l-1];
        // y[-2] -> a2 g[l]; y[-1] -> a1 g[l] + a2 g[l-1]
        hb0[k] = br.z * gl;
        hb1[k] = fmaf(br.y, gl, br.z * glm1);
        ha0[k] = ab.y * gl;
        ha1[k] = fmaf(ab.x, gl, ab.y * glm1);
        g0[k] = gl;
        g1[k] = glm1;
    }
    __syncwarp();
    // block recurrence state per section: the previous block's last two
    // inputs and outputs; the first block of the channel takes zi instead
    float px2[kMaxSections], px1[kMaxSections], py2[kMaxSections], py1[kMaxSections];
    float zi1[kMaxSections], zi2[kMaxSections];
#pragma unroll
    for (int k = 0; k < kMaxSections; ++k) {
        px2[k] = px1[k] = py2[k] = py1[k] = 0.f;
        zi1[k] = zi2[k] = 0.f;
        if (k < g.K && g.first && p.zi) {
            zi1[k] = p.zi[((int64_t)c * p.kmax + k) * 2 + 0];
            zi2[k] = p.zi[((int64_t)c * p.kmax + k) * 2 + 1];
        }
    }
    const float* x = p.x + g.off;
    float* y = p.y + g.off;
    bool first_block = true;
    // the channel's last sample, for the final state: its block-relative lane
    const int64_t nlast = g.len - 1;
    float zf1[kMaxSections], zf2[kMaxSections];
#pragma unroll
    for (int k = 0; k < kMaxSections; ++k) {
        zf1[k] = zi1[k];
        zf2[k] = zi2[k];
    }
    for (int64_t b0i = g.cstart; b0i < g.out_hi; b0i += 32) {
        const int64_t n = b0i + lane;
        float v = n < g.len ? __ldg(x + n) : 0.f;
        const bool has_last = g.last && nlast >= b0i && nlast < b0i + 32;
        const int lq = (int)(nlast - b0i);
#pragma unroll
        for (int k = 0; k < kMaxSections; ++k) {
            if (k >= g.K) break;
            const float* hk = hpad + k * 64 + 32 + lane;
            // H x_n: cumulative sum of the columns, x_j broadcast to the warp
            float acc = 0.f;
#pragma unroll 8
            for (int j = 0; j < 32; ++j)
                acc = fmaf(hk[-j], __shfl_sync(0xffffffffu, v, j), acc);
            // boundary: + H_b xbar - H_a ybar (or the channel's initial state,
            // which enters as z1 g[l] + z2 g[l-1])
            if (first_block && g.first) {
                acc = fmaf(zi1[k], g0[k], fmaf(zi2[k], g1[k], acc));
            } else {
                acc = fmaf(hb0[k], px2[k], fmaf(hb1[k], px1[k], acc));
                acc = fmaf(-ha0[k], py2[k], fmaf(-ha1[k], py1[k], acc));
            }
            if (has_last) {
                // DF2T state after sample nlast from the section's inputs and
                // outputs at nlast and nlast - 1 (the previous block's last
                // ones when nlast opens this block)
                const float xm1 = __shfl_sync(0xffffffffu, v, (lq - 1) & 31);
                const float ym1 = __shfl_sync(0xffffffffu, acc, (lq - 1) & 31);
                const bool open = lq == 0;
                const float xp = open ? (first_block && g.first ? 0.f : px1[k]) : xm1;
                const float yp = open ? (first_block && g.first ? 0.f : py1[k]) : ym1;
                const float4 br = cf[k].braw, ab = cf[k].ab;
                // at the channel's very first sample the previous "input" and
                // "output" are carried by zi itself: z1 = b1 x - a1 y + z2_in
                float f1 = fmaf(br.y, v, fmaf(br.z, xp, fmaf(-ab.x, acc, -ab.y * yp)));
                if (open && first_block && g.first) f1 = fmaf(br.y, v, fmaf(-ab.x, acc, zi2[k]));
                const float f2 = fmaf(br.z, v, -ab.y * acc);
                zf1[k] = __shfl_sync(0xffffffffu, f1, lq);
                zf2[k] = __shfl_sync(0xffffffffu, f2, lq);
            }
            px2[k] = __shfl_sync(0xffffffffu, v, 30);
            px1[k] = __shfl_sync(0xffffffffu, v, 31);
            py2[k] = __shfl_sync(0xffffffffu, acc, 30);
            py1[k] = __shfl_sync(0xffffffffu, acc, 31);
            v = acc;
        }
        first_block = false;
        if (n >= g.out_lo && n < g.out_hi) y[n] = v;
    }
    if (g.last && p.zf && lane == 0)
#pragma unroll
        for (int k = 0; k < kMaxSections; ++k) {
            if (k >= p.kmax) break;
            p.zf[((int64_t)c * p.kmax + k) * 2 + 0] = k < g.K ? zf1[k] : 0.f;
            p.zf[((int64_t)c * p.kmax + k) * 2 + 1] = k < g.K ? zf2[k] : 0.f;
        }
}

cudaError_t launch_compare(const Params& p, int algo, int64_t seg_len, int64_t max_segs,
                           cudaStream_t stream) {
    if (max_segs <= 0) return cudaSuccess;
    if (algo == 0) {
        const int threads = 128;
        const unsigned gx = (unsigned)((max_segs + threads - 1) / threads);
        sos_scalar_kernel<<<dim3(gx, (unsigned)p.C), threads, 0, stream>>>(p, seg_len);
    } else {
        const size_t smem = sizeof(float) * kBlkWarps * kMaxSections * 64;
        static bool attr = false;
        if (!attr) {
            const cudaError_t e = cudaFuncSetAttribute(
                sos_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const unsigned gx = (unsigned)((max_segs + kBlkWarps - 1) / kBlkWarps);
        sos_block_kernel<<<dim3(gx, (unsigned)p.C), kBlkWarps * 32, smem, stream>>>(p, seg_len);
    }
    return cudaGetLastError();
}

}  // namespace sosf
