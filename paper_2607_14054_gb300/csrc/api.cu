// C ABI of the library (declared in include/sosfilt.h): argument checks,
// workspace carving and the two launches of one call (plan, forward).
#include <cstring>
#include <vector>

#include "sos_common.cuh"

namespace sosf {
cudaError_t launch_plan(const Params& p, cudaStream_t stream);
cudaError_t launch_forward(const Params& p, int64_t host_tiles, cudaStream_t stream, bool early);
cudaError_t launch_pipe(const Params& p, int64_t grid, cudaStream_t stream, bool early);
bool forward_supported(int N, int W);
bool pipe_supported(int N);
cudaError_t launch_warpseg(const Params& p, int64_t grid, cudaStream_t stream, bool early);
int warpseg_ctas_per_sm(int N, int algo);
int warpseg_warps_per_cta();
cudaError_t launch_stream(const Params& p, int64_t chunk, int64_t seg_len, int32_t maxseg,
                          int32_t foreign, cudaStream_t stream);
cudaError_t launch_reverse(const float* src, float* dst, const Params& p, int64_t max_len,
                           cudaStream_t stream);
cudaError_t launch_compare(const Params& p, int algo, int64_t seg_len, int64_t max_segs,
                           cudaStream_t stream);
}  // namespace sosf

using namespace sosf;

namespace {

constexpr int32_t kAbiVersion = 1;

struct Tune {
    int N, W, algo, flags;
};

bool resolve_tuning(const sos_tuning* t, Tune* out) {
    Tune r{32, 8, 1, 0};
    if (t) {
        if (t->n_blocks) r.N = t->n_blocks;
        if (t->warps) r.W = t->warps;
        if (t->algo) r.algo = t->algo;
        r.flags = t->flags;
    }
    if (r.algo != 1 && r.algo != 2) return false;
    if (!forward_supported(r.N, r.W) || !pipe_supported(r.N)) return false;
    *out = r;
    return true;
}

// SMs of the current device (cached per device); 0 if unknown.
int device_sms() {
    static int s_sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (s_sms[dev] == 0 &&
        cudaDeviceGetAttribute(&s_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return s_sms[dev];
}

constexpr int kPipeCtasPerSm = 2;

// Segment length: long enough that the warm-up before each segment is a small
// fraction of it, short enough that the segments of the whole call keep every
// consumer busy: each pipeline CTA (between 8 and 64 groups of 32 N), or, for
// the warp-segment kernel, each resident warp (at least 8192 samples, so that
// horizons up to 4096 samples qualify as with the pipeline, and at most 64
// groups).
// CTAs per SM of a warp-segment launch: the tuning's request (flag bits
// 8..11), at most as many as fit; 0 = as many as fit.
int warpseg_ctas(int N, int algo, int flags) {
    const int fit = warpseg_ctas_per_sm(N, algo);
    const int req = (flags >> 8) & 15;
    return req > 0 && req < fit ? req : fit;
}

int64_t segment_length(int64_t total_len, int N, int algo, int flags, bool warp_segments) {
    const int64_t group = 32LL * N;
    const int sms = device_sms() > 0 ? device_sms() : 148;
    int64_t units = (int64_t)sms * kPipeCtasPerSm, gmin = 8;
    if (warp_segments) {
        const int occ = warpseg_ctas(N, algo, flags);
        units = (int64_t)sms * (occ > 0 ? occ : 1) * warpseg_warps_per_cta();
        gmin = (8192 + group - 1) / group;
    }
    int64_t g = (total_len + units * group - 1) / (units * group);
    if (g < gmin) g = gmin;
    if (g > 64) g = 64;
    return g * group;
}

int64_t count_tiles(int32_t C, const int64_t* lengths_host, int64_t T, bool* ok) {
    int64_t total = 0;
    *ok = true;
    for (int32_t c = 0; c < C; ++c) {
        const int64_t n = lengths_host[c];
        if (n < 0) {
            *ok = false;
            return 0;
        }
        total += (n + T - 1) / T;
    }
    return total;
}

}  // namespace

extern "C" {

int32_t sos_abi_version(void) { return kAbiVersion; }

const char* sos_status_str(sos_status s) {
    switch (s) {
        case SOS_OK: return "SOS_OK";
        case SOS_ERR_ARG: return "SOS_ERR_ARG";
        case SOS_ERR_UNSTABLE: return "SOS_ERR_UNSTABLE";
        case SOS_ERR_CUDA: return "SOS_ERR_CUDA";
        case SOS_ERR_TIMEOUT: return "SOS_ERR_TIMEOUT";
        case SOS_ERR_WORKSPACE: return "SOS_ERR_WORKSPACE";
        case SOS_ERR_UNSUPPORTED: return "SOS_ERR_UNSUPPORTED";
        case SOS_ERR_COEF: return "SOS_ERR_COEF";
    }
    return "SOS_ERR_UNKNOWN";
}

size_t sos_workspace_size(int32_t n_channels, int32_t kmax, const int64_t* lengths_host,
                          const sos_tuning* tuning) {
    Tune tu;
    if (n_channels < 1 || kmax < 1 || kmax > kMaxSections || !lengths_host) return 0;
    if (!resolve_tuning(tuning, &tu)) return 0;
    bool ok = true;
    const int64_t tiles = count_tiles(n_channels, lengths_host, (int64_t)tu.W * kLanes * tu.N, &ok);
    if (!ok) return 0;
    return ws_layout(n_channels, kmax, tiles).total;
}

sos_status sos_workspace_init(void* workspace, size_t ws_bytes, void* stream) {
    if (!workspace || ws_bytes < sizeof(WsHeader)) return SOS_ERR_ARG;
    if (cudaMemsetAsync(workspace, 0, ws_bytes, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SOS_ERR_CUDA;
    return SOS_OK;
}

}  // extern "C"

namespace {

// Validates the shared arguments and fills the workspace part of Params.
sos_status setup(int32_t n_channels, int32_t kmax, const int64_t* lengths_host, void* workspace,
                 size_t ws_bytes, const sos_tuning* tuning, Params* p, int64_t* tiles_out,
                 int64_t* total_len_out) {
    if (!lengths_host || !workspace) return SOS_ERR_ARG;
    if (n_channels < 1 || kmax < 1) return SOS_ERR_ARG;
    if (kmax > kMaxSections) return SOS_ERR_UNSUPPORTED;
    Tune tu;
    if (!resolve_tuning(tuning, &tu)) return SOS_ERR_UNSUPPORTED;
    bool ok = true;
    const int64_t T = (int64_t)tu.W * kLanes * tu.N;
    const int64_t tiles = count_tiles(n_channels, lengths_host, T, &ok);
    if (!ok) return SOS_ERR_ARG;
    int64_t total_len = 0;
    for (int32_t c = 0; c < n_channels; ++c) total_len += lengths_host[c];
    const WsLayout L = ws_layout(n_channels, kmax, tiles);
    if (ws_bytes < L.total) return SOS_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    p->hdr = reinterpret_cast<WsHeader*>(ws + L.hdr);
    p->chan = reinterpret_cast<ChanInfo*>(ws + L.chan);
    p->tb = reinterpret_cast<int64_t*>(ws + L.tb);
    p->tbp = reinterpret_cast<int64_t*>(ws + L.tbp);
    p->order = reinterpret_cast<int32_t*>(ws + L.order);
    p->porder = reinterpret_cast<int32_t*>(ws + L.porder);
    p->rp = reinterpret_cast<int64_t*>(ws + L.rp);
    p->c32 = reinterpret_cast<Coef32*>(ws + L.c32);
    p->cdf = reinterpret_cast<CoefDF*>(ws + L.cdf);
    p->key = reinterpret_cast<unsigned char*>(ws + L.key);
    p->words = reinterpret_cast<unsigned long long*>(ws + L.slots);
    p->cap_tiles = tiles;
    p->C = n_channels;
    p->kmax = kmax;
    p->N = tu.N;
    p->W = tu.W;
    p->flags_opt = tu.flags;
    p->algo = tu.algo;
    p->seg = segment_length(total_len, tu.N, tu.algo, tu.flags,
                            (tu.flags & SOS_FLAG_SECTION_PIPELINE) == 0);
    p->total = total_len;
    *tiles_out = tiles;
    *total_len_out = total_len;
    return SOS_OK;
}

}  // namespace

extern "C" {

sos_status sos_prepare(const double* sos, const int32_t* K, int32_t n_channels, int32_t kmax,
                       const int64_t* lengths, const int64_t* lengths_host, void* workspace,
                       size_t ws_bytes, const sos_tuning* tuning, void* stream) {
    if (!sos || !K || !lengths) return SOS_ERR_ARG;
    Params p{};
    int64_t tiles = 0, total = 0;
    const sos_status s = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p,
                               &tiles, &total);
    if (s != SOS_OK) return s;
    p.sos = sos;
    p.K = K;
    p.lengths = lengths;
    if (launch_plan(p, static_cast<cudaStream_t>(stream)) != cudaSuccess) return SOS_ERR_CUDA;
    return SOS_OK;
}

}  // extern "C"

namespace {

// which of the two filtering launches a call enqueues
enum ApplyParts { kPartPipe = 1, kPartCarry = 2 };

sos_status apply_parts(const float* x, int32_t n_channels, int32_t kmax,
                       const int64_t* lengths_host, const float* zi, float* y, float* zf,
                       void* workspace, size_t ws_bytes, const sos_tuning* tuning, void* stream,
                       int parts) {
    Params p{};
    int64_t tiles = 0, total = 0;
    const sos_status s = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p,
                               &tiles, &total);
    if (s != SOS_OK) return s;
    if (total > 0 && (!x || !y)) return SOS_ERR_ARG;
    if (x && y && total > 0) {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t bytes = sizeof(float) * (size_t)total;
        if (xb < yb + bytes && yb < xb + bytes) return SOS_ERR_ARG;  // no overlap
    }
    p.x = x;
    p.y = y;
    p.zi = zi;
    p.zf = zf;
    // the warp-segment kernel (or the section pipeline) for the channels
    // within their memory horizon, then the look-back kernel for the others
    // (which also writes the final states of empty channels and unused
    // sections: at least one CTA), launched early so that it starts without a
    // launch gap once the first has completed
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool early = false;
    if (total > 0 && (parts & kPartPipe)) {
        const int64_t sms = device_sms() > 0 ? device_sms() : 1;
        cudaError_t e;
        // launched early (programmatic dependent launch): its CTAs become
        // resident while the preceding kernel (normally the plan) finishes,
        // and wait for that kernel's completion on the device
        if (p.flags_opt & SOS_FLAG_SECTION_PIPELINE)
            e = launch_pipe(p, sms * kPipeCtasPerSm, st, true);
        else
            e = launch_warpseg(p, sms * warpseg_ctas(p.N, p.algo, p.flags_opt), st, true);
        if (e != cudaSuccess) return SOS_ERR_CUDA;
        early = true;
    }
    if (parts & kPartCarry) {
        const int64_t launch_tiles = tiles > 0 ? tiles : 1;
        if (launch_forward(p, launch_tiles, st, early) != cudaSuccess) return SOS_ERR_CUDA;
    }
    return SOS_OK;
}

}  // namespace

extern "C" {

sos_status sos_apply(const float* x, int32_t n_channels, int32_t kmax,
                     const int64_t* lengths_host, const float* zi, float* y, float* zf,
                     void* workspace, size_t ws_bytes, const sos_tuning* tuning, void* stream) {
    return apply_parts(x, n_channels, kmax, lengths_host, zi, y, zf, workspace, ws_bytes, tuning,
                       stream, kPartPipe | kPartCarry);
}

sos_status sos_apply_pipeline(const float* x, int32_t n_channels, int32_t kmax,
                              const int64_t* lengths_host, const float* zi, float* y, float* zf,
                              void* workspace, size_t ws_bytes, const sos_tuning* tuning,
                              void* stream) {
    return apply_parts(x, n_channels, kmax, lengths_host, zi, y, zf, workspace, ws_bytes, tuning,
                       stream, kPartPipe);
}

sos_status sos_apply_carried(const float* x, int32_t n_channels, int32_t kmax,
                             const int64_t* lengths_host, const float* zi, float* y, float* zf,
                             void* workspace, size_t ws_bytes, const sos_tuning* tuning,
                             void* stream) {
    return apply_parts(x, n_channels, kmax, lengths_host, zi, y, zf, workspace, ws_bytes, tuning,
                       stream, kPartCarry);
}

sos_status sos_filter(const float* x, const double* sos, const int32_t* K, int32_t n_channels,
                      int32_t kmax, const int64_t* lengths, const int64_t* lengths_host,
                      const float* zi, float* y, float* zf, void* workspace, size_t ws_bytes,
                      const sos_tuning* tuning, void* stream) {
    // check everything the second half checks before enqueuing the first
    Params p{};
    int64_t tiles = 0, total = 0;
    sos_status s = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p, &tiles,
                         &total);
    if (s != SOS_OK) return s;
    if (!sos || !K || !lengths) return SOS_ERR_ARG;
    if (total > 0 && (!x || !y)) return SOS_ERR_ARG;
    if (x && y && total > 0) {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t bytes = sizeof(float) * (size_t)total;
        if (xb < yb + bytes && yb < xb + bytes) return SOS_ERR_ARG;
    }
    s = sos_prepare(sos, K, n_channels, kmax, lengths, lengths_host, workspace, ws_bytes, tuning,
                    stream);
    if (s != SOS_OK) return s;
    return sos_apply(x, n_channels, kmax, lengths_host, zi, y, zf, workspace, ws_bytes, tuning,
                     stream);
}

sos_status sos_stream(const float* x, float* y, const float* zi, float* zf, int32_t n_channels,
                      int32_t kmax, int64_t chunk, uint32_t flags, void* workspace,
                      size_t ws_bytes, const sos_tuning* tuning, void* stream) {
    if (chunk < 0 || n_channels < 1 || (flags & ~SOS_STREAM_FOREIGN_STATE)) return SOS_ERR_ARG;
    if (chunk > 0 && (!x || !y)) return SOS_ERR_ARG;
    // the workspace was carved by sos_prepare for n_channels channels of
    // `chunk` samples each: carve it the same way
    std::vector<int64_t> lh((size_t)n_channels, chunk);
    Params p{};
    int64_t tiles = 0, total = 0;
    const sos_status s = setup(n_channels, kmax, lh.data(), workspace, ws_bytes, tuning, &p,
                               &tiles, &total);
    if (s != SOS_OK) return s;
    if (x && y && total > 0) {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t bytes = sizeof(float) * (size_t)total;
        if (xb < yb + bytes && yb < xb + bytes) return SOS_ERR_ARG;
    }
    if (zi && zf) {
        // different warps of one channel read zi and write zf
        const char* a = reinterpret_cast<const char*>(zi);
        const char* b = reinterpret_cast<const char*>(zf);
        const size_t bytes = sizeof(float) * 2 * (size_t)kmax * (size_t)n_channels;
        if (a < b + bytes && b < a + bytes) return SOS_ERR_ARG;
    }
    p.x = x;
    p.y = y;
    p.zi = zi;
    p.zf = zf;
    if (chunk == 0) return SOS_OK;
    // segments: enough for every resident warp of the device to take one
    // when the channels alone do not fill it; each channel's own memory
    // horizon may lengthen its segments on the device
    const int64_t group = 32LL * p.N;
    const int sms = device_sms() > 0 ? device_sms() : 148;
    const int occ = warpseg_ctas(p.N, 1, 0);
    const int64_t warps = (int64_t)sms * (occ > 0 ? occ : 1) * warpseg_warps_per_cta();
    int64_t per = warps / n_channels;
    if (per < 1) per = 1;
    int64_t seg = (chunk + per - 1) / per;
    seg = (seg + group - 1) / group * group;
    const int64_t maxseg = (chunk + seg - 1) / seg;
    const int32_t foreign = (flags & SOS_STREAM_FOREIGN_STATE) && zi ? 1 : 0;
    if (launch_stream(p, chunk, seg, (int32_t)maxseg, foreign,
                      static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SOS_ERR_CUDA;
    return SOS_OK;
}

sos_status sos_apply_baseline(int32_t algorithm, const float* x, int32_t n_channels,
                              int32_t kmax, const int64_t* lengths_host, const float* zi, float* y,
                              float* zf, int64_t seg_len, void* workspace, size_t ws_bytes,
                              const sos_tuning* tuning, void* stream) {
    if (algorithm != 0 && algorithm != 1) return SOS_ERR_ARG;
    if (seg_len < 32) return SOS_ERR_ARG;
    Params p{};
    int64_t tiles = 0, total = 0;
    const sos_status s = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p,
                               &tiles, &total);
    if (s != SOS_OK) return s;
    if (total > 0 && (!x || !y)) return SOS_ERR_ARG;
    if (x && y && total > 0) {
        const char* xb = reinterpret_cast<const char*>(x);
        const char* yb = reinterpret_cast<const char*>(y);
        const size_t bytes = sizeof(float) * (size_t)total;
        if (xb < yb + bytes && yb < xb + bytes) return SOS_ERR_ARG;
    }
    // segments per channel: at most ceil(len / seg_len) (channels without a
    // horizon are one segment)
    int64_t max_segs = 1;
    for (int32_t c = 0; c < n_channels; ++c) {
        const int64_t ns = (lengths_host[c] + seg_len - 1) / seg_len;
        if (ns > max_segs) max_segs = ns;
    }
    p.x = x;
    p.y = y;
    p.zi = zi;
    p.zf = zf;
    if (launch_compare(p, algorithm, seg_len, max_segs, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return SOS_ERR_CUDA;
    return SOS_OK;
}

sos_status sos_filtfilt(const float* x, const double* sos, const int32_t* K, int32_t n_channels,
                        int32_t kmax, const int64_t* lengths, const int64_t* lengths_host, float* y,
                        float* tmp, void* workspace, size_t ws_bytes, const sos_tuning* tuning,
                        void* stream) {
    Params p{};
    int64_t tiles = 0, total = 0;
    sos_status s = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p, &tiles,
                         &total);
    if (s != SOS_OK) return s;
    if (!sos || !K || !lengths) return SOS_ERR_ARG;
    if (total > 0 && (!x || !y || !tmp)) return SOS_ERR_ARG;
    if (total > 0) {
        const size_t bytes = sizeof(float) * (size_t)total;
        const char* b[3] = {reinterpret_cast<const char*>(x), reinterpret_cast<const char*>(y),
                            reinterpret_cast<const char*>(tmp)};
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (b[i] < b[j] + bytes && b[j] < b[i] + bytes) return SOS_ERR_ARG;
    }
    int64_t max_len = 0;
    for (int32_t c = 0; c < n_channels; ++c) max_len = lengths_host[c] > max_len ? lengths_host[c] : max_len;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // forward pass (zero state), reversal, forward pass of the reversed
    // signal, reversal: y = R H R H x
    s = sos_prepare(sos, K, n_channels, kmax, lengths, lengths_host, workspace, ws_bytes, tuning,
                    stream);
    if (s != SOS_OK) return s;
    s = sos_apply(x, n_channels, kmax, lengths_host, nullptr, tmp, nullptr, workspace, ws_bytes,
                  tuning, stream);
    if (s != SOS_OK) return s;
    if (launch_reverse(tmp, y, p, max_len, st) != cudaSuccess) return SOS_ERR_CUDA;
    s = sos_apply(y, n_channels, kmax, lengths_host, nullptr, tmp, nullptr, workspace, ws_bytes,
                  tuning, stream);
    if (s != SOS_OK) return s;
    if (launch_reverse(tmp, y, p, max_len, st) != cudaSuccess) return SOS_ERR_CUDA;
    return SOS_OK;
}

sos_status sos_device_status(void* workspace, void* stream) {
    if (!workspace) return SOS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SOS_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOS_ERR_CUDA;
    int32_t result = h.status;
    if (result == 0 && h.nchan > 0) {
        // channel table sits right after the header (see ws_layout); read it in
        // fixed-size pieces (no host allocation)
        const WsLayout L = ws_layout(h.nchan, 1, 1);
        ChanInfo buf[128];
        for (int32_t c0 = 0; c0 < h.nchan && result == 0; c0 += 128) {
            const int32_t n = h.nchan - c0 < 128 ? h.nchan - c0 : 128;
            if (cudaMemcpy(buf, static_cast<char*>(workspace) + L.chan + sizeof(ChanInfo) * c0,
                           sizeof(ChanInfo) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                return SOS_ERR_CUDA;
            for (int32_t i = 0; i < n; ++i)
                if (buf[i].err) {
                    result = buf[i].err;
                    break;
                }
        }
    }
    const int32_t zero = 0;
    if (cudaMemcpy(&static_cast<WsHeader*>(workspace)->status, &zero, sizeof(zero),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return SOS_ERR_CUDA;
    return static_cast<sos_status>(result);
}

sos_status sos_plan_query(void* workspace, int32_t first, int32_t count, int32_t* horizon,
                          int32_t* tiles, void* stream) {
    if (!workspace || first < 0 || count < 0) return SOS_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SOS_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOS_ERR_CUDA;
    if ((int64_t)first + count > h.nchan) return SOS_ERR_ARG;
    const WsLayout L = ws_layout(h.nchan, 1, 1);
    ChanInfo buf[128];
    for (int32_t c0 = 0; c0 < count; c0 += 128) {
        const int32_t n = count - c0 < 128 ? count - c0 : 128;
        if (cudaMemcpy(buf,
                       static_cast<char*>(workspace) + L.chan + sizeof(ChanInfo) * (first + c0),
                       sizeof(ChanInfo) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SOS_ERR_CUDA;
        for (int32_t i = 0; i < n; ++i) {
            if (horizon) horizon[c0 + i] = buf[i].horizon;
            if (tiles) tiles[c0 + i] = buf[i].ntiles;
        }
    }
    return SOS_OK;
}

sos_status sos_plan_extended(void* workspace, int32_t first, int32_t count, int32_t* extended,
                             void* stream) {
    if (!workspace || !extended || first < 0 || count < 0) return SOS_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SOS_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOS_ERR_CUDA;
    if ((int64_t)first + count > h.nchan) return SOS_ERR_ARG;
    const WsLayout L = ws_layout(h.nchan, 1, 1);
    ChanInfo buf[128];
    for (int32_t c0 = 0; c0 < count; c0 += 128) {
        const int32_t n = count - c0 < 128 ? count - c0 : 128;
        if (cudaMemcpy(buf,
                       static_cast<char*>(workspace) + L.chan + sizeof(ChanInfo) * (first + c0),
                       sizeof(ChanInfo) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
            return SOS_ERR_CUDA;
        for (int32_t i = 0; i < n; ++i) extended[c0 + i] = buf[i].ext;
    }
    return SOS_OK;
}

sos_status sos_workspace_set_wait_limit(void* workspace, uint32_t limit, void* stream) {
    if (!workspace) return SOS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t v = limit;
    if (cudaMemcpyAsync(&static_cast<WsHeader*>(workspace)->spin_limit, &v, sizeof(v),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SOS_ERR_CUDA;
    // the source is a local: the copy must have read it before returning
    if (cudaStreamSynchronize(st) != cudaSuccess) return SOS_ERR_CUDA;
    return SOS_OK;
}

sos_status sos_plan_recomputed(void* workspace, int32_t* channels, void* stream) {
    if (!workspace || !channels) return SOS_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SOS_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOS_ERR_CUDA;
    *channels = h.last_recomputed;
    return SOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

namespace sosf {
cudaError_t launch_adjoint(const Params& p, int sms, double* grad_sos, cudaStream_t stream);
int64_t adjoint_warps(int N, int sms);
int64_t adjoint_ck_slots(int N, int64_t total_len, int32_t C);
}  // namespace sosf

namespace {

struct BwdLayout {
    size_t ck, gacc, total;
};

// the backward's scratch after the forward workspace: forward-state
// checkpoints of the adjoint kernel and the FP64 coefficient sums
BwdLayout bwd_layout(size_t base, int32_t C, int32_t kmax, int64_t total_len, int N) {
    BwdLayout L;
    size_t o = align_up(base, 256);
    L.ck = o;
    o = align_up(o + sizeof(float) * 2 * (size_t)kmax * (size_t)adjoint_ck_slots(N, total_len, C),
                 256);
    L.gacc = o;
    o = align_up(o + sizeof(double) * 5 * (size_t)C * (size_t)kmax, 256);
    L.total = o;
    return L;
}

// Backward segment length, in whole groups (at least 8, at most 64): from
// the call's samples over the adjoint kernel's resident warps upwards, the
// length whose segments (whole channels cut at it) take the fewest group
// steps on the warps, rounds x groups per segment, so that a channel's last
// partial segment does not start a second round on a few warps; a horizon
// of up to half a segment fits.
int64_t backward_segment_length(const int64_t* lengths_host, int32_t C, int64_t total_len,
                                int N) {
    const int64_t group = 32LL * N;
    const int sms = device_sms() > 0 ? device_sms() : 148;
    int64_t units = adjoint_warps(N, sms);
    if (units < 1) units = 1;
    int64_t g0 = (total_len + units * group - 1) / (units * group);
    if (g0 < 8) g0 = 8;
    if (g0 > 64) g0 = 64;
    int64_t best = g0, best_cost = -1;
    for (int64_t g = g0; g <= 64 && g <= 2 * g0; ++g) {
        const int64_t seg = g * group;
        int64_t nseg = 0;
        for (int32_t c = 0; c < C; ++c) nseg += (lengths_host[c] + seg - 1) / seg;
        const int64_t cost = (nseg + units - 1) / units * g;
        if (best_cost < 0 || cost < best_cost) {
            best = g;
            best_cost = cost;
        }
    }
    return best * group;
}

}  // namespace

extern "C" {

size_t sos_backward_workspace_size(int32_t n_channels, int32_t kmax, const int64_t* lengths_host,
                                   const sos_tuning* tuning) {
    const size_t base = sos_workspace_size(n_channels, kmax, lengths_host, tuning);
    if (base == 0) return 0;
    Tune tu;
    if (!resolve_tuning(tuning, &tu)) return 0;
    int64_t total = 0;
    for (int32_t c = 0; c < n_channels; ++c) total += lengths_host[c];
    return bwd_layout(base, n_channels, kmax, total, tu.N).total;
}

sos_status sos_filter_backward(const float* x, const double* sos, const int32_t* K,
                               int32_t n_channels, int32_t kmax, const int64_t* lengths,
                               const int64_t* lengths_host, const float* zi, const float* grad_y,
                               const float* grad_zf, float* grad_x, double* grad_sos,
                               float* grad_zi, void* workspace, size_t ws_bytes,
                               const sos_tuning* tuning, void* stream) {
    Params p{};
    int64_t tiles = 0, total = 0;
    sos_status st = setup(n_channels, kmax, lengths_host, workspace, ws_bytes, tuning, &p, &tiles,
                          &total);
    if (st != SOS_OK) return st;
    if (!sos || !K || !lengths || !grad_sos) return SOS_ERR_ARG;
    if (total > 0 && (!x || !grad_y || !grad_x)) return SOS_ERR_ARG;
    const size_t base = ws_layout(n_channels, kmax, tiles).total;
    const BwdLayout BL = bwd_layout(base, n_channels, kmax, total, p.N);
    if (ws_bytes < BL.total) return SOS_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    p.sos = sos;
    p.K = K;
    p.lengths = lengths;
    // the backward plan: no look-back (a channel without a memory horizon is
    // one segment), segments sized for the adjoint kernel's warps
    p.flags_opt |= kFlagBackwardPlan;
    p.seg = backward_segment_length(lengths_host, n_channels, total, p.N);
    p.ck = reinterpret_cast<float*>(ws + BL.ck);
    p.gacc = reinterpret_cast<double*>(ws + BL.gacc);
    if (launch_plan(p, sm) != cudaSuccess) return SOS_ERR_CUDA;
    if (cudaMemsetAsync(p.gacc, 0, sizeof(double) * 5 * (size_t)n_channels * kmax, sm) !=
        cudaSuccess)
        return SOS_ERR_CUDA;
    p.x = x;
    p.y = nullptr;
    p.zi = zi;
    p.zf = nullptr;
    p.gy = grad_y;
    p.gzf = grad_zf;
    p.gx = grad_x;
    p.gzi = grad_zi;
    const int sms = device_sms() > 0 ? device_sms() : 1;
    if (launch_adjoint(p, sms, grad_sos, sm) != cudaSuccess) return SOS_ERR_CUDA;
    return SOS_OK;
}

}  // extern "C"
