// sos_filter_host: the whole call from host memory to host memory.
//
// A caller whose signal lives in (pinned) host memory pays two copies per
// call, each several times the filter's own time.  This entry point cuts the
// packed signal into blocks and runs, for each block, the copy in, the
// filter and the copy out on three streams, two device buffers per
// direction, so that block i's filter and block i-1's copy out overlap block
// i+1's copy in: the call then takes about as long as the two copies run
// side by side instead of one after the other.  The filtering is sos_filter
// itself, block by block, on the caller's stream: whole channels grouped up
// to the block size, and a channel longer than that in time pieces whose
// DF2T states are handed from piece to piece on the device (the state
// hand-off of Sec. V between calls).
#include <algorithm>
#include <mutex>
#include <vector>

#include "sos_common.cuh"

namespace sosf {

namespace {

constexpr int kMaxDevices = 64;

// per device: the two copy streams and the hand-over events (slot 0, 1 for
// copied-in, filtered, copied-out), made once and kept; calls that enqueue
// at the same time take turns (the mutex), their work may interleave on the
// shared copy streams but each waits only on its own hand-overs or on
// earlier, finished ones
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr}, ev_start = nullptr, ev_join[2] = {nullptr, nullptr};
};
std::mutex g_host_mu;
HostPipe g_pipes[kMaxDevices];

cudaError_t host_pipe(int dev, HostPipe** hp) {
    HostPipe& h = g_pipes[dev];
    if (!h.in) {
        cudaError_t e = cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&h.ev_in[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev_comp[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev_out[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.ev_start, cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&h.ev_join[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            h.in = nullptr;
            return e;
        }
    }
    *hp = &h;
    return cudaSuccess;
}

__global__ void set_length_kernel(int64_t* cell, int64_t value) { *cell = value; }

// One block of the call: channels [c0, c1) whole, or (c1 = c0 + 1, piece
// >= 0) samples [t0, t0 + len) of channel c0.
struct Block {
    int32_t c0, c1;
    int64_t off;   // first sample in the packed arrays
    int64_t len;   // samples
    int64_t t0;    // time piece: first sample within the channel
    bool piece, first, last;
};

std::vector<Block> plan_blocks(int32_t C, const int64_t* lh, int64_t block) {
    std::vector<Block> v;
    int64_t off = 0;
    int32_t c = 0;
    while (c < C) {
        const int64_t n = lh[c];
        if (n > block) {
            for (int64_t t = 0; t < n; t += block) {
                const int64_t len = std::min(block, n - t);
                v.push_back(Block{c, c + 1, off + t, len, t, true, t == 0, t + len == n});
            }
            off += n;
            ++c;
            continue;
        }
        // whole channels while they fit (the first always does: lh[c] <= block)
        Block b{c, c, off, 0, 0, false, true, true};
        while (c < C && lh[c] <= block && b.len + lh[c] <= block) {
            b.len += lh[c];
            off += lh[c];
            ++c;
        }
        b.c1 = c;
        v.push_back(b);
    }
    return v;
}

int64_t default_block(int64_t total) {
    int64_t b = (total + 7) / 8;
    b = (b + 4095) / 4096 * 4096;
    return std::max<int64_t>(b, int64_t(1) << 20);
}

// The blocks' copies in, filters and copies out, in order (see sos_filter_host).
sos_status enqueue_blocks(const std::vector<Block>& blocks, HostPipe* hp, cudaStream_t st,
                          const float* x_host, const double* sos, const int32_t* K, int32_t kmax,
                          const int64_t* lengths, const int64_t* lengths_host, const float* zi,
                          float* y_host, float* zf, void* workspace, size_t ws_bytes,
                          float* const* dx, float* const* dy, float* const* carry,
                          int64_t* const* lcell, const sos_tuning* tuning, void* stream) {
    sos_status s = SOS_OK;
    int pc = 0;  // carry buffer holding the state entering the next piece
    for (size_t i = 0; i < blocks.size(); ++i) {
        const Block& b = blocks[i];
        const int sl = (int)(i & 1);
        const size_t bytes = sizeof(float) * (size_t)b.len;
        // copy in (after block i - 2's filter has released this buffer)
        if (cudaStreamWaitEvent(hp->in, hp->ev_comp[sl], 0) != cudaSuccess) return SOS_ERR_CUDA;
        if (b.len > 0 &&
            cudaMemcpyAsync(dx[sl], x_host + b.off, bytes, cudaMemcpyHostToDevice, hp->in) !=
                cudaSuccess)
            return SOS_ERR_CUDA;
        if (cudaEventRecord(hp->ev_in[sl], hp->in) != cudaSuccess) return SOS_ERR_CUDA;
        // filter on the caller's stream (after the copy in, and after block
        // i - 2's copy out has released the output buffer)
        if (cudaStreamWaitEvent(st, hp->ev_in[sl], 0) != cudaSuccess) return SOS_ERR_CUDA;
        if (cudaStreamWaitEvent(st, hp->ev_out[sl], 0) != cudaSuccess) return SOS_ERR_CUDA;
        if (b.piece) {
            const int32_t c = b.c0;
            const int64_t len = b.len;
            set_length_kernel<<<1, 1, 0, st>>>(lcell[sl], len);
            if (cudaGetLastError() != cudaSuccess) return SOS_ERR_CUDA;
            const float* zin = b.first ? (zi ? zi + (int64_t)c * kmax * 2 : nullptr) : carry[pc];
            float* zout = b.last ? (zf ? zf + (int64_t)c * kmax * 2 : nullptr) : carry[pc ^ 1];
            s = sos_filter(dx[sl], sos + (int64_t)c * kmax * 6, K + c, 1, kmax, lcell[sl], &len,
                           zin, dy[sl], zout, workspace, ws_bytes, tuning, stream);
            if (s != SOS_OK) return s;
            if (!b.first || !b.last) pc ^= 1;
        } else {
            const int32_t c = b.c0, n = b.c1 - b.c0;
            s = sos_filter(dx[sl], sos + (int64_t)c * kmax * 6, K + c, n, kmax, lengths + c,
                           lengths_host + c, zi ? zi + (int64_t)c * kmax * 2 : nullptr, dy[sl],
                           zf ? zf + (int64_t)c * kmax * 2 : nullptr, workspace, ws_bytes, tuning,
                           stream);
            if (s != SOS_OK) return s;
        }
        if (cudaEventRecord(hp->ev_comp[sl], st) != cudaSuccess) return SOS_ERR_CUDA;
        // copy out
        if (cudaStreamWaitEvent(hp->out, hp->ev_comp[sl], 0) != cudaSuccess) return SOS_ERR_CUDA;
        if (b.len > 0 &&
            cudaMemcpyAsync(y_host + b.off, dy[sl], bytes, cudaMemcpyDeviceToHost, hp->out) !=
                cudaSuccess)
            return SOS_ERR_CUDA;
        if (cudaEventRecord(hp->ev_out[sl], hp->out) != cudaSuccess) return SOS_ERR_CUDA;
    }
    return SOS_OK;
}

}  // namespace

}  // namespace sosf

using namespace sosf;

extern "C" sos_status sos_filter_host_sizes(int32_t n_channels, int32_t kmax,
                                            const int64_t* lengths_host, int64_t block,
                                            const sos_tuning* tuning, size_t* ws_bytes,
                                            size_t* staging_bytes, int64_t* block_used) {
    if (n_channels < 1 || kmax < 1 || kmax > kMaxSections || !lengths_host) return SOS_ERR_ARG;
    int64_t total = 0;
    for (int32_t c = 0; c < n_channels; ++c) {
        if (lengths_host[c] < 0) return SOS_ERR_ARG;
        total += lengths_host[c];
    }
    if (block <= 0) block = default_block(total);
    block = (block + 3) / 4 * 4;
    size_t ws = 0;
    for (const Block& b : plan_blocks(n_channels, lengths_host, block)) {
        const int64_t one = b.len;
        const size_t need = b.piece ? sos_workspace_size(1, kmax, &one, tuning)
                                    : sos_workspace_size(b.c1 - b.c0, kmax, lengths_host + b.c0,
                                                         tuning);
        if (need == 0) return SOS_ERR_ARG;
        ws = std::max(ws, need);
    }
    if (ws == 0) ws = sos_workspace_size(1, kmax, &block, tuning);
    if (ws_bytes) *ws_bytes = ws;
    // two input and two output buffers of a block, two state buffers, two
    // length cells
    if (staging_bytes)
        *staging_bytes = 4 * sizeof(float) * (size_t)block + 2 * 256 + 2 * 256;
    if (block_used) *block_used = block;
    return SOS_OK;
}

extern "C" sos_status sos_filter_host(const float* x_host, const double* sos, const int32_t* K,
                                      int32_t n_channels, int32_t kmax, const int64_t* lengths,
                                      const int64_t* lengths_host, const float* zi,
                                      float* y_host, float* zf, void* workspace, size_t ws_bytes,
                                      void* staging, size_t staging_bytes, int64_t block,
                                      const sos_tuning* tuning, void* stream) {
    size_t ws_need = 0, st_need = 0;
    int64_t blk = 0;
    sos_status s = sos_filter_host_sizes(n_channels, kmax, lengths_host, block, tuning, &ws_need,
                                         &st_need, &blk);
    if (s != SOS_OK) return s;
    if (!sos || !K || !lengths || !workspace || !staging) return SOS_ERR_ARG;
    if (ws_bytes < ws_need || staging_bytes < st_need) return SOS_ERR_WORKSPACE;
    if (kmax * 2 * sizeof(float) > 256) return SOS_ERR_ARG;
    int64_t total = 0;
    for (int32_t c = 0; c < n_channels; ++c) total += lengths_host[c];
    if (total > 0 && (!x_host || !y_host)) return SOS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SOS_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SOS_ERR_ARG;  // host-side blocking steps
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SOS_ERR_CUDA;

    char* base = static_cast<char*>(staging);
    float* dx[2] = {reinterpret_cast<float*>(base),
                    reinterpret_cast<float*>(base) + blk};
    float* dy[2] = {reinterpret_cast<float*>(base) + 2 * blk,
                    reinterpret_cast<float*>(base) + 3 * blk};
    char* tail = base + 4 * sizeof(float) * (size_t)blk;
    float* carry[2] = {reinterpret_cast<float*>(tail), reinterpret_cast<float*>(tail + 256)};
    int64_t* lcell[2] = {reinterpret_cast<int64_t*>(tail + 512),
                         reinterpret_cast<int64_t*>(tail + 768)};

    const std::vector<Block> blocks = plan_blocks(n_channels, lengths_host, blk);
    std::lock_guard<std::mutex> lock(g_host_mu);
    HostPipe* hp = nullptr;
    if (host_pipe(dev, &hp) != cudaSuccess) return SOS_ERR_CUDA;
    // the copies in may overwrite the staging buffers only after the
    // caller's earlier work on `stream` (an earlier call's filters) is done
    if (cudaEventRecord(hp->ev_start, st) != cudaSuccess) return SOS_ERR_CUDA;
    if (cudaStreamWaitEvent(hp->in, hp->ev_start, 0) != cudaSuccess) return SOS_ERR_CUDA;
    if (cudaStreamWaitEvent(hp->out, hp->ev_start, 0) != cudaSuccess) return SOS_ERR_CUDA;
    // the call is complete on `stream` when everything enqueued on the copy
    // streams is: the last copies out, or, after an error part way, whatever
    // was enqueued before it (so that the caller may free the buffers once
    // `stream` is done)
    const sos_status se = enqueue_blocks(blocks, hp, st, x_host, sos, K, kmax, lengths,
                                         lengths_host, zi, y_host, zf, workspace, ws_bytes, dx,
                                         dy, carry, lcell, tuning, stream);
    cudaError_t e = cudaEventRecord(hp->ev_join[0], hp->in);
    if (e == cudaSuccess) e = cudaEventRecord(hp->ev_join[1], hp->out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp->ev_join[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, hp->ev_join[1], 0);
    if (se != SOS_OK) return se;
    return e == cudaSuccess ? SOS_OK : SOS_ERR_CUDA;
}
