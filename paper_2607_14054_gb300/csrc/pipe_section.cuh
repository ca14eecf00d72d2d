// One section of the cascade over one group of 32 N samples held as lane
// chunks in registers: S3 non-recursive stage, S4-PH (particular solution,
// lane scan, re-run from the true lane state), the group's outgoing DF2T
// state, and S8 (zf) for the lane holding the channel's last sample.  Used
// by the forward section pipeline and, on time-reversed data, by the adjoint.
#pragma once

#include "sos_pipe.cuh"

namespace sosf {

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

}  // namespace sosf
