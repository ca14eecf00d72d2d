// Time reversal of packed channels, for zero-phase (forward-backward)
// filtering: channel c's samples [off_c, off_c + len_c) of src are written
// reversed into the same positions of dst.  Grid: (blocks over samples,
// channels); reads and writes are both coalesced (neighbouring threads touch
// neighbouring addresses, one run ascending and one descending).
#include "sos_common.cuh"

namespace sosf {

__global__ void reverse_kernel(const float* __restrict__ src, float* __restrict__ dst,
                               const ChanInfo* __restrict__ chan, int32_t C) {
    const int c = blockIdx.y;
    if (c >= C) return;
    const int64_t off = chan[c].off, len = chan[c].len;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[off + i] = __ldg(src + off + len - 1 - i);
}

cudaError_t launch_reverse(const float* src, float* dst, const Params& p, int64_t max_len,
                           cudaStream_t stream) {
    if (max_len <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t bx = (max_len + threads - 1) / threads;
    if (bx > 1024) bx = 1024;
    reverse_kernel<<<dim3((unsigned)bx, (unsigned)p.C), threads, 0, stream>>>(src, dst, p.chan, p.C);
    return cudaGetLastError();
}

}  // namespace sosf
