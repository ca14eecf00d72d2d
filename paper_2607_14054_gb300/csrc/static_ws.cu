// sos_filter_static: sos_filter with its scratch memory in a fixed, library-
// owned device array instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory at all: real-time audio or
// control callbacks where cudaMalloc's latency and implicit device
// synchronisation are not allowed, plug-ins running inside a host application
// that owns the device allocator, and code that must not grow the memory
// footprint after start-up.  They still pass their own input and output
// buffers; only the scratch (channel table, coefficient tables, look-back
// words) moves into this array.
#include <mutex>

#include "sos_common.cuh"

namespace sosf {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device

// File-scope device scratch.  In host code `g_static_scratch` names a host-side
// stand-in, not device memory: only the address obtained from
// cudaGetSymbolAddress (per device, with that device current) may be given to
// a kernel.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
}  // namespace

}  // namespace sosf

using namespace sosf;

extern "C" sos_status sos_filter_static(const float* x, const double* sos, const int32_t* K,
                                        int32_t n_channels, int32_t kmax, const int64_t* lengths,
                                        const int64_t* lengths_host, const float* zi, float* y,
                                        float* zf, const sos_tuning* tuning, void* stream,
                                        int32_t* device_status) {
    if (n_channels < 1 || kmax < 1 || !lengths_host) return SOS_ERR_ARG;
    const size_t need = sos_workspace_size(n_channels, kmax, lengths_host, tuning);
    if (need == 0) return SOS_ERR_ARG;
    if (need > kStaticScratchBytes) return SOS_ERR_WORKSPACE;  // beyond the fixed maximum
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SOS_ERR_CUDA;
    // reading the device status waits for the stream, which a capture forbids
    if (cap != cudaStreamCaptureStatusNone && device_status) return SOS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SOS_ERR_CUDA;
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            // first call on this device: find the array's device address and
            // zero it once (the look-back epoch and the tile counter must start
            // at zero; later calls keep them consistent themselves).  The
            // zeroing is ordered on the caller's stream and waited for here, so
            // that it has finished before this or any later call, on any
            // stream, touches the array.  A stream being captured cannot be
            // waited for: the first call must come before any capture.
            if (cap != cudaStreamCaptureStatusNone) return SOS_ERR_ARG;
            void* a = nullptr;
            if (cudaGetSymbolAddress(&a, g_static_scratch) != cudaSuccess || !a) return SOS_ERR_CUDA;
            if (cudaMemsetAsync(a, 0, kStaticScratchBytes, st) != cudaSuccess) return SOS_ERR_CUDA;
            if (cudaStreamSynchronize(st) != cudaSuccess) return SOS_ERR_CUDA;
            g_addr[dev] = a;
        }
        ws = g_addr[dev];
    }
    const sos_status s = sos_filter(x, sos, K, n_channels, kmax, lengths, lengths_host, zi, y, zf,
                                    ws, kStaticScratchBytes, tuning, stream);
    if (s != SOS_OK || !device_status) return s;
    *device_status = (int32_t)sos_device_status(ws, stream);  // waits for the stream
    return SOS_OK;
}
