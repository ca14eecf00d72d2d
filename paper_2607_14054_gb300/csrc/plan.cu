// Plan kernel: per-call set-up of the workspace, entirely on the device so
// that a call never synchronises and can be captured into a CUDA graph.
//
//  * block C (the last one): channel offsets and tile prefix (exclusive scans
//    of the lengths) and the status word;
//  * block c < C: the coefficient tables of channel c, one warp per section.
//
// Coefficient tables (paper Sec. VI-B, "pre-computed before filtering"):
// the rows are normalised by a0; when every b0 of the channel is nonzero the
// common factor prod_k b0_k is split off (Sec. II, Eq. simple_second_order)
// and section k's state is carried scaled by 1/G_k, G_k = b0_1 ... b0_k.
// The DF2T transition A = [[-a1, 1], [-a2, 0]] is raised to the lane step
// Phi = A^N, the warp step Psi = A^(NL) and the tile step Theta = A^T by
// repeated squaring, then the per-lane tables Phi^l, Psi^w and Theta^d by
// binary powering, each lane forming its own entry.  All of it runs in
// double-float arithmetic (about 48 significand bits) on the FP32 pipe:
// GB300's FP64 FMA is 1/64 of its FP32 rate with a 64-cycle latency.  The
// per-sample tables are rounded once to FP32; the Theta^d used by the
// cross-tile look-back stay double-float.
#include <cfloat>
#include <cmath>

#include "sos_common.cuh"

namespace sosf {

__device__ __forceinline__ df df_of_double(double v) {
    const float hi = (float)v;
    return df{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ float4 to_f4(const dfm2& m) {
    return make_float4(df_to_float(m.a), df_to_float(m.b), df_to_float(m.c), df_to_float(m.d));
}

__device__ __forceinline__ bool finite_row(const double* r) {
    for (int i = 0; i < 6; ++i)
        if (!isfinite(r[i])) return false;
    return true;
}

// Blocks 0..C-1: coefficients.  Block C: channel table.  256 threads.
__global__ void __launch_bounds__(256) plan_kernel(Params p) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = p.C, kmax = p.kmax;

    if ((int)blockIdx.x == C) {
        // ---- channel table: exclusive scans of lengths and tile counts ----
        const int64_t T = (int64_t)p.W * kLanes * p.N;
        __shared__ int64_t s_wsum_len[8], s_wsum_til[8];
        __shared__ int64_t s_carry_len, s_carry_til;
        if (tid == 0) {
            s_carry_len = 0;
            s_carry_til = 0;
            p.hdr->status = 0;
            p.hdr->nchan = C;
        }
        __syncthreads();
        for (int base = 0; base < C; base += 256) {
            const int c = base + tid;
            int64_t len = 0, nt = 0;
            int32_t K = 0;
            if (c < C) {
                len = p.lengths[c];
                K = p.K[c];
                if (len < 0 || K < 0 || K > kmax) {
                    set_status(p.hdr, SOS_ERR_ARG);
                    len = 0;
                    K = 0;
                }
                nt = len > 0 ? (len + T - 1) / T : 0;
            }
            // inclusive warp scans
            int64_t il = len, it = nt;
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t ol = __shfl_up_sync(0xffffffffu, il, d);
                const int64_t ot = __shfl_up_sync(0xffffffffu, it, d);
                if (lane >= d) {
                    il += ol;
                    it += ot;
                }
            }
            if (lane == 31) {
                s_wsum_len[warp] = il;
                s_wsum_til[warp] = it;
            }
            __syncthreads();
            int64_t wl = 0, wt = 0;
            for (int w = 0; w < warp; ++w) {
                wl += s_wsum_len[w];
                wt += s_wsum_til[w];
            }
            const int64_t cl = s_carry_len, ct = s_carry_til;
            if (c < C) {
                // mode and err belong to the coefficient block of channel c
                p.chan[c].off = cl + wl + il - len;
                p.chan[c].len = len;
                p.chan[c].K = K;
                p.chan[c].ntiles = (int32_t)nt;
                p.tb[c] = ct + wt + it - nt;
            }
            __syncthreads();
            if (tid == 255) {
                s_carry_len = cl + wl + il;
                s_carry_til = ct + wt + it;
            }
            __syncthreads();
        }
        if (tid == 0) {
            const int64_t total = s_carry_til;
            p.tb[C] = total;
            if (total > p.cap_tiles) set_status(p.hdr, SOS_ERR_WORKSPACE);
            p.hdr->total_tiles = total > p.cap_tiles ? 0 : total;
        }
        return;
    }

    // ---- coefficient tables of channel c ----
    const int c = blockIdx.x;
    __shared__ double s_b0[kMaxSections];
    __shared__ int s_mode;
    __shared__ double s_G[kMaxSections];
    // [0..4] Phi^(2^j); [5..9] Psi^(2^r); [10..19] Theta^(2^i)
    __shared__ dfm2 s_chain[kMaxSections][20];

    if (tid == 0) p.chan[c].err = 0;
    __syncthreads();
    const int K = p.K[c];
    const bool valid_K = (K >= 0 && K <= kmax);
    const int Kc = valid_K ? K : 0;
    const int k = warp;
    double row[6] = {0, 0, 0, 1, 0, 0};
    bool active = k < Kc;
    if (active) {
        const double* r = p.sos + ((int64_t)c * kmax + k) * 6;
        for (int i = 0; i < 6; ++i) row[i] = r[i];
        bool ok = finite_row(row) && row[3] != 0.0;
        if (!ok) {
            if (lane == 0) atomicCAS(&p.chan[c].err, 0, (int)SOS_ERR_COEF);
            row[0] = 0; row[1] = 0; row[2] = 0; row[3] = 1; row[4] = 0; row[5] = 0;
        }
    }
    const double ia0 = 1.0 / row[3];
    const double b0 = row[0] * ia0, b1 = row[1] * ia0, b2 = row[2] * ia0;
    const double a1 = row[4] * ia0, a2 = row[5] * ia0;
    if (active && (p.flags_opt & SOS_FLAG_CHECK_STABLE)) {
        // both roots of z^2 + a1 z + a2 strictly inside the unit circle
        // (Jury: |a2| < 1 and |a1| < 1 + a2)
        if (!(fabs(a2) < 1.0 && fabs(a1) < 1.0 + a2) && lane == 0)
            atomicCAS(&p.chan[c].err, 0, (int)SOS_ERR_UNSTABLE);
    }
    if (lane == 0 && k < kMaxSections) s_b0[k] = b0;
    __syncthreads();
    if (tid == 0) {
        // factor b0 out of every section when that keeps the scaled signal in
        // a safe FP32 range: every b0 nonzero and 2^-60 < |G_k| < 2^60
        int mode = Kc > 0 ? 1 : 0;
        double G = 1.0;
        for (int j = 0; j < Kc; ++j) {
            G *= s_b0[j];
            if (!(s_b0[j] != 0.0) || !(fabs(G) > 0x1p-60) || !(fabs(G) < 0x1p60)) mode = 0;
        }
        G = 1.0;
        for (int j = 0; j < kMaxSections; ++j) {
            if (j < Kc && mode) G *= s_b0[j];
            s_G[j] = mode ? G : 1.0;
        }
        s_mode = mode;
        p.chan[c].mode = mode;
    }
    __syncthreads();
    const int mode = s_mode;

    if (!active) return;

    // ---- double-float squaring chain (lane 0) ----
    const int N = p.N, W = p.W;
    if (lane == 0) {
        const dfm2 A{df_of_double(-a1), df{1.f, 0.f}, df_of_double(-a2), df{0.f, 0.f}};
        dfm2 P = A;
        for (int n = 1; n < N; n <<= 1) P = dfm_mul(P, P);  // A^N (N a power of two)
        s_chain[k][0] = P;
        for (int j = 1; j < 5; ++j) s_chain[k][j] = dfm_mul(s_chain[k][j - 1], s_chain[k][j - 1]);
        s_chain[k][5] = dfm_mul(s_chain[k][4], s_chain[k][4]);  // Psi = Phi^32
        for (int r = 1; r < 5; ++r) s_chain[k][5 + r] = dfm_mul(s_chain[k][4 + r], s_chain[k][4 + r]);
        dfm2 Th = dfm_identity();  // Theta = Psi^W, any W <= 31
        for (int r = 0; r < 5; ++r)
            if ((W >> r) & 1) Th = dfm_mul(Th, s_chain[k][5 + r]);
        s_chain[k][10] = Th;
        for (int i = 1; i < 10; ++i) s_chain[k][10 + i] = dfm_mul(s_chain[k][9 + i], s_chain[k][9 + i]);
    }
    __syncwarp();

    Coef32* out32 = p.c32 + ((int64_t)c * kmax + k);
    CoefDF* outdf = p.cdf + ((int64_t)c * kmax + k);
    {
        // Phi^lane, Theta^lane and Theta^(32 lane) by binary powering
        dfm2 P = dfm_identity(), Q = dfm_identity(), R = dfm_identity();
        for (int j = 0; j < 5; ++j)
            if ((lane >> j) & 1) {
                P = dfm_mul(P, s_chain[k][j]);
                Q = dfm_mul(Q, s_chain[k][10 + j]);
                R = dfm_mul(R, s_chain[k][15 + j]);
            }
        out32->lane_pow[lane] = to_f4(P);
        outdf->theta_pow[lane][0] = make_float4(Q.a.hi, Q.a.lo, Q.b.hi, Q.b.lo);
        outdf->theta_pow[lane][1] = make_float4(Q.c.hi, Q.c.lo, Q.d.hi, Q.d.lo);
        if (lane < 18) {
            outdf->theta_hi[lane][0] = make_float4(R.a.hi, R.a.lo, R.b.hi, R.b.lo);
            outdf->theta_hi[lane][1] = make_float4(R.c.hi, R.c.lo, R.d.hi, R.d.lo);
        }
        if (lane == 0) {
            const dfm2 T32 = s_chain[k][15];
            outdf->theta_pow[32][0] = make_float4(T32.a.hi, T32.a.lo, T32.b.hi, T32.b.lo);
            outdf->theta_pow[32][1] = make_float4(T32.c.hi, T32.c.lo, T32.d.hi, T32.d.lo);
        }
    }
    if (lane < 16) {
        dfm2 P = dfm_identity();
        for (int r = 0; r < 4; ++r)
            if ((lane >> r) & 1) P = dfm_mul(P, s_chain[k][5 + r]);
        out32->psi_w[lane] = to_f4(P);
    }
    if (lane < 5) out32->phi_pow[lane] = to_f4(s_chain[k][lane]);
    if (lane < 4) out32->psi_pow[lane] = to_f4(s_chain[k][5 + lane]);
    if (lane == 0) {
        const double sb = mode ? 1.0 / b0 : 1.0;
        out32->ab = make_float4((float)a1, (float)a2, (float)(b1 * sb), (float)(b2 * sb));
        const double G = s_G[k];
        out32->misc = make_float4((float)b0, (float)G, (float)(1.0 / G), 0.0f);
    }
}

// Interleaved dispatch order (one CTA of 1024 threads, runs after
// plan_kernel).  Tiles are handed out round by round: round r holds tile r of
// every channel that has more than r tiles.  Then a tile's predecessor in its
// own channel was dispatched a whole round earlier and has usually finished,
// so the look-back finds its outgoing state at once.  Channels are sorted by
// decreasing tile count (bitonic sort in shared memory), which makes each
// round a prefix of that order.  With more than kMaxSortChannels channels the
// kernel leaves nrounds = 0 and tiles go channel by channel.
__global__ void __launch_bounds__(1024) order_kernel(Params p) {
    extern __shared__ unsigned long long s_key[];
    const int tid = threadIdx.x, C = p.C;
    if (C > kMaxSortChannels) {
        if (tid == 0) p.hdr->nrounds = 0;
        return;
    }
    int n = 1;
    while (n < C) n <<= 1;
    for (int i = tid; i < n; i += blockDim.x) {
        // ascending sort of (MAX - ntiles, channel): decreasing tile count,
        // then increasing channel index; padding sorts last
        const unsigned long long nt = i < C ? (unsigned long long)p.chan[i].ntiles : 0ull;
        s_key[i] = i < C ? (((0xffffffffull - nt) << 32) | (unsigned)i) : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = s_key[i], b = s_key[j];
                    if ((a > b) == up) {
                        s_key[i] = b;
                        s_key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < C; i += blockDim.x) p.order[i] = (int32_t)(s_key[i] & 0xffffffffu);
    const int64_t nrounds = C > 0 ? (int64_t)(0xffffffffull - (s_key[0] >> 32)) : 0;
    // rp[r] = sum over rounds q < r of (channels with more than q tiles)
    __shared__ int64_t s_carry;
    __shared__ int64_t s_wsum[32];
    if (tid == 0) s_carry = 0;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int64_t base = 0; base <= nrounds; base += blockDim.x) {
        const int64_t r = base + tid;
        int64_t cnt = 0;
        if (r < nrounds) {
            // channels with ntiles > r: a prefix of the sorted order (binary search)
            int lo = 0, hi = C;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const int64_t nt = (int64_t)(0xffffffffull - (s_key[mid] >> 32));
                if (nt > r) lo = mid + 1; else hi = mid;
            }
            cnt = lo;
        }
        int64_t inc = cnt;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        int64_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        const int64_t carry = s_carry;
        if (r <= nrounds) p.rp[r] = carry + wpre + inc - cnt;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = carry + wpre + inc;
        __syncthreads();
    }
    if (tid == 0) p.hdr->nrounds = nrounds;
}

}  // namespace sosf

namespace sosf {
cudaError_t launch_plan(const Params& p, cudaStream_t stream) {
    plan_kernel<<<p.C + 1, 256, 0, stream>>>(p);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    int n = 1;
    while (n < p.C && n < kMaxSortChannels) n <<= 1;
    const size_t smem = p.C <= kMaxSortChannels ? sizeof(unsigned long long) * (size_t)n : 0;
    static bool attr_set = false;
    if (!attr_set) {
        err = cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(unsigned long long) * kMaxSortChannels));
        if (err != cudaSuccess) return err;
        attr_set = true;
    }
    order_kernel<<<1, 1024, smem, stream>>>(p);
    return cudaGetLastError();
}
}  // namespace sosf
