// Shared definitions of the sm_103a cascaded-biquad kernels: workspace
// layout, per-section coefficient tables, and small PTX helpers.
//
// Notation follows the paper: L = 32 lanes (the block size, Sec. IV, "the
// warp width on a GPU"), N samples per lane per group (the number of blocks,
// Sec. V), a group of N*L samples per warp, W warps per tile.  Lane l of a
// warp holds samples [l*N, l*N + N) of its group in registers v[0..N), so
// register m of all lanes is the paper's strided block x_m (Sec. V,
// Eq. recursive_equation_multi_block_form) and the stride-N permutation of
// Sec. VII-A is the shared-memory transpose done on load.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sosfilt.h"
#include "sos_df.cuh"

namespace sosf {

constexpr int kLanes = 32;
constexpr int kMaxSections = SOS_MAX_SECTIONS;
constexpr uint32_t kFlagAgg = 1;   // tile aggregate of one section published
constexpr uint32_t kFlagInc = 2;   // tile inclusive state (outgoing state) published
constexpr uint32_t kSpinLimit = 1u << 21;
constexpr int kMaxSortChannels = 8192;  // interleaved dispatch up to this many channels

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

struct WsHeader {
    uint32_t epoch;         // bumped by the plan kernel once per call
    uint32_t tile_counter;  // in-order tile dispatch
    int32_t status;         // device-side status of the latest call (sos_status)
    uint32_t plan_done;     // blocks of the running plan launch that have finished
    int64_t total_tiles;    // tiles of the latest call (device view)
    int32_t nchan;          // channels of the latest call
    uint32_t done;          // CTAs of the running filter launch that have finished
    int64_t nrounds;        // interleaved dispatch: rounds (longest channel's tiles); 0 = channel-major
    int64_t total_pipe;     // segments of the section pipeline (channels within their horizon)
    unsigned long long seg_next;  // warp-segment kernel: segments handed out past the first round
    uint32_t seg_done;      // warp-segment kernel: warps of the running launch that have finished
    uint32_t spin_limit;    // bound on each device-side wait (0 = the compiled default)
    // plan cache: the call-level inputs of the latest complete plan on this
    // workspace (key_valid = 1), so that the next plan can tell whether a
    // channel's tables are still those of its inputs
    int32_t key_valid, key_N, key_W, key_algo, key_flags, key_kmax, key_C;
    uint32_t plan_changed;  // channels recomputed by the running plan launch
    int64_t key_seg, key_cap;
    int32_t last_recomputed;  // channels the latest plan recomputed
    uint32_t pad2[3];
};
static_assert(sizeof(WsHeader) == 128, "header size");

// Per-channel record of the plan cache: the raw sos rows (bit patterns), K
// and length from which the channel's tables were last built.
struct ChanKeyHead {
    int64_t len;
    int32_t K;
    int32_t valid;
};
__host__ __device__ inline size_t chan_key_stride(int32_t kmax) {
    return sizeof(ChanKeyHead) + sizeof(double) * 6 * (size_t)kmax;
}

struct ChanInfo {
    int64_t off;      // first sample of the channel in the packed arrays
    int64_t len;      // samples
    int32_t K;        // sections used
    int32_t mode;     // 1: b0 factored out of every section (Sec. II, Eq. simple_second_order)
    int32_t ntiles;   // tiles of this channel (dispatch)
    int32_t err;      // coefficient error found by the plan kernel (sos_status), 0 if none
    int64_t slot;     // first look-back slot of the channel (ceil(len / T) slots)
    int32_t horizon;  // >= 0: memory horizon P (segments start P samples early, no
                      // carry); -1: the state is carried by the look-back
    int16_t single;   // 1: the whole channel is one segment (backward plans)
    int16_t ext;      // precision class: 0 FP32; 1, 2: the largest section level
                      // (Coef32::misc.w); 3: double-float samples throughout
    int64_t seg;      // segment length of a channel with a horizon (a multiple of 32 N,
                      // at least 2 P)
    int32_t minseg;   // the shortest segment length the horizon allows (P, whole
                      // groups), 0 without a horizon
    int32_t minseg_z; // the same, also long enough for the response of an arbitrary
                      // initial state to die out
    int16_t dflo, dfhi;  // precision class 3: sections dflo..dfhi run with double-float
                         // samples, the others in FP32
    int32_t pad;
};
static_assert(sizeof(ChanInfo) == 72, "channel table entry");

// A channel's memory horizon P is the shortest warm-up after which the
// cascade's impulse-response tail, summed in absolute value, is below
// kHorizonEps times a lower bound of the response's L2 norm (and the
// initial state's contribution past the first tile is below the same
// bound).  Tiles of such a channel start P samples early from zero state;
// the state they drop changes the output by less than kHorizonEps relative,
// far below FP32 rounding.  Longer memories (P > T / 2, poles on or near the
// unit circle, coincident poles) keep the decoupled look-back.
constexpr float kHorizonEps = 0x1p-30f;

// Cyclic reduction divides by e_i at every level (c_i = e_i - f_i / e_i);
// a section whose |f_i / e_i| exceeds this at some level keeps PH, which
// divides by nothing.
constexpr double kCrKappaMax = 100.0;

// Internal plan flag (above the public SOS_FLAG_* bits): the plan of a
// backward call, where channels without a horizon become single segments.
constexpr int32_t kFlagBackwardPlan = 1 << 16;

// Per (channel, section) FP32 coefficients and transition-matrix powers.
// The DF2T state transition of one sample is A = [[-a1, 1], [-a2, 0]];
// Phi = A^N advances one lane chunk, Psi = A^{N L} one warp group.  All
// powers are formed in FP64 and rounded once to FP32.  2x2 matrices are
// stored row-major in a float4 (m00, m01, m10, m11).
struct __align__(16) Coef32 {
    float4 ab;            // a1, a2, b1, b2  (b1, b2 divided by b0 when factored)
    float4 misc;          // b0, G_k (cumulative gain), 1/G_k, 1 if extended precision
    float4 braw;          // b0, b1, b2 normalised by a0 only (the adjoint's FIR)
    float4 phi_pow[5];    // Phi^(2^j), j = 0..4 (lane scan)
    float4 psi_pow[4];    // Psi^(2^r), r = 0..3 (warp scan)
    float4 psi_w[16];     // Psi^w, w = 0..15 (fold the tile state into warp w)
    float4 lane_pow[32];  // Phi^l, l = 0..31 (fold the warp state into lane l)
    // cyclic reduction (Sec. VI-C), built when the call asks for it: level i
    // of log2 N has (e_i, f_i, g_i = f_i / e_i, c_i = e_i - g_i) and
    // d_i = -f_i g_i (Eq. cr_coeff_update); the terminal recurrence across
    // lanes Y_l + e_n Y_{l-1} + f_n Y_{l-2} = V_l (Eq. cr_terminal_block) is
    // scanned with the powers C^(2^j) of C = [[-e_n, -f_n], [1, 0]].
    float4 cr_lv[6];      // (e_i, f_i, g_i, c_i)
    float4 cr_d[2];       // d_0 .. d_7
    float4 cr_tpow[5];    // C^(2^j), row-major
    float4 cr_misc;       // e_n, f_n, kappa = max |g_i|, 1 if CR is used for this section
    // read only by sections that run in extended precision (misc.w): the low
    // parts of phi_pow and lane_pow (each power = hi + lo in double-float)
    // and of a1, a2 (alo.x, alo.y; the exact a_i = ab + alo to 48 bits)
    float4 phi_lo[5];
    float4 lane_lo[32];
    float4 alo;
    // read by channels run with double-float samples: the low parts of b0,
    // b1, b2 normalised by a0 (never factored; braw holds the high parts)
    float4 blo;
};

// Extended precision per section (Coef32::misc.w).  Level 2 when the
// largest entry of its powers Phi^(2^j), Phi^l exceeds kDfScanEntry (poles
// close to z = +-1 near the unit circle: the entries grow to about
// min(l N, 1 / sin(theta)) and the FP32 products of the lane scan cancel), or
// when rounding a1, a2 to FP32 moves its poles by more than kDfCoefSens of
// their distance to the circle: the lane scan and fold run in double-float
// and the in-lane recursions add the coefficients' low parts.  Level 1 when
// that displacement exceeds kAloCoefSens only: the low parts alone (two FMAs
// per sample and pass).  The output's relative error from rounding a1, a2
// is about that displacement, so level 1 keeps it below 2^-18.
constexpr float kDfScanEntry = 8.f;
constexpr double kDfCoefSens = 1e-4;
constexpr double kAloCoefSens = 0x1p-18;

// A channel is run with double-float samples throughout (ChanInfo::ext = 3)
// when the relative error that FP32 rounding of the signals handed from one
// section to the next would cause at the output, estimated by the plan for a
// white input from zero state, exceeds kHandOffErrMax (or when the estimate
// cannot be formed and some section needs the double-float scan), or when a
// section's own FP32 rounding is amplified beyond kSectionErrMax: rounding
// its FIR output or its recursion adds white noise of relative size 2^-24,
// which its all-pole part passes with gain ||g|| (g the all-pole impulse
// response) against a signal passed with the whole section's gain ||h|| per
// unit ||b||, so the section's condition number kappa = ||g|| ||b|| / ||h||
// (zeros close to the poles make it large) must stay below
// kSectionErrMax * 2^24.  The measured error of the FP32 path is about 0.4 to
// 30 times the hand-off estimate (the recursions' own roundings add to it);
// kHandOffErrMax keeps the cascades whose estimate says FP32 cannot reach
// about 1e-4 -- a white input from zero state through a random cascade near
// the estimate's bound may still see errors of 1e-5..1e-4
// (SOS_FLAG_DOUBLE_FLOAT removes them).
constexpr float kHandOffErrMax = 0x1p-15f;
constexpr float kSectionErrMax = 0x1p-17f;

// Per (channel, section) double-float powers of the tile transition
// Theta = A^T (T = tile length) for the cross-tile composition, each as
// (a.hi, a.lo, b.hi, b.lo), (c.hi, c.lo, d.hi, d.lo):
// theta_pow[d] = Theta^d, d = 0..32; theta_hi[j] = Theta^(32 j), j = 0..17.
struct __align__(16) CoefDF {
    float4 theta_pow[33][2];
    float4 theta_hi[18][2];
};

// Look-back words, per (section, tile): the tile's inclusive (true outgoing)
// state as four 64-bit words (z1.hi, z1.lo, z2.hi, z2.lo) and its aggregate
// (zero-state outgoing) state as two (z1, z2; the aggregate is an FP32
// quantity).  Every word carries its own tag (epoch << 2 | kind) in the low
// 32 bits, so a reader validates what it read word by word: one L2 round
// trip, no separate flag, no fence.  Stored as structure of arrays, word w of
// tile t in section k at ((k * kWords + w) * cap_tiles + t), so that 32 lanes
// reading 32 consecutive tiles make one coalesced access.
constexpr int kWords = 6;  // inc z1.hi, z1.lo, z2.hi, z2.lo, agg z1, z2

struct WsLayout {
    size_t hdr, chan, tb, tbp, order, porder, rp, c32, cdf, key, slots, total;
    int64_t cap_tiles;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline WsLayout ws_layout(int32_t C, int32_t kmax, int64_t cap_tiles) {
    WsLayout L{};
    size_t o = 0;
    L.hdr = o;   o = align_up(o + sizeof(WsHeader), 256);
    L.chan = o;  o = align_up(o + sizeof(ChanInfo) * (size_t)C, 256);
    L.tb = o;    o = align_up(o + sizeof(int64_t) * ((size_t)C + 1), 256);
    L.tbp = o;   o = align_up(o + sizeof(int64_t) * ((size_t)C + 1), 256);
    L.order = o; o = align_up(o + sizeof(int32_t) * (size_t)C, 256);
    L.porder = o; o = align_up(o + sizeof(int32_t) * (size_t)C, 256);
    // rounds of the interleaved dispatch: at most the longest channel's tile
    // count, which overlapping tiles (stride >= T / 2) at most double
    L.rp = o;    o = align_up(o + sizeof(int64_t) * (2 * (size_t)(cap_tiles > 0 ? cap_tiles : 0) + 2), 256);
    L.c32 = o;   o = align_up(o + sizeof(Coef32) * (size_t)C * kmax, 256);
    L.cdf = o;   o = align_up(o + sizeof(CoefDF) * (size_t)C * kmax, 256);
    L.key = o;   o = align_up(o + chan_key_stride(kmax) * (size_t)C, 256);
    const size_t nt = (size_t)(cap_tiles > 0 ? cap_tiles : 1);
    L.slots = o; o = align_up(o + sizeof(unsigned long long) * kWords * nt * kmax, 256);
    L.total = o;
    L.cap_tiles = cap_tiles;
    return L;
}

// Everything the plan and filter kernels need, by value.
struct Params {
    const float* x;
    float* y;
    const double* sos;
    const int32_t* K;
    const int64_t* lengths;
    const float* zi;
    float* zf;
    WsHeader* hdr;
    ChanInfo* chan;
    int64_t* tb;         // look-back tile prefix over the carried channels [C + 1]
    int64_t* tbp;        // segment prefix over the channels within their horizon, by
                         // dispatch position [C + 1]
    int32_t* porder;     // channel at each dispatch position of those segments [C]
    int32_t* order;      // channels by decreasing tile count (interleaved dispatch)
    int64_t* rp;         // tiles dispatched before round r [nrounds + 1]
    Coef32* c32;
    CoefDF* cdf;
    unsigned char* key;  // plan cache: per channel a ChanKeyHead and kmax raw sos rows
    unsigned long long* words;  // look-back words [kmax][kWords][cap_tiles]
    int64_t cap_tiles;
    int32_t C;
    int32_t kmax;
    int32_t N;           // samples per lane
    int32_t W;           // warps per tile
    int32_t flags_opt;   // SOS_FLAG_*
    int32_t algo;        // recursive-stage solver: 1 PH, 2 CR where well conditioned
    int64_t seg;         // pipeline segment length (samples, a multiple of 32 N)
    float* ck;           // backward: forward-state checkpoints [slots][kmax][2]
    const float* gy;     // backward: dL/dy [total]
    const float* gzf;    // backward: dL/dzf [C][kmax][2], or null
    float* gx;           // backward: dL/dx [total]
    float* gzi;          // backward: dL/dzi [C][kmax][2], or null
    double* gacc;        // backward: [C][kmax][5] sums for b0, b1, b2, a1, a2
    int64_t total;       // samples of all channels
};

// Launch of fn(p); early: programmatic dependent launch, the kernel may be
// scheduled once the previous kernel in the stream has let it (that kernel
// executes griddepcontrol.launch_dependents), and waits for that kernel's
// completion itself (griddepcontrol.wait) before it starts work.
inline cudaError_t launch_params(const void* fn, int64_t grid, int threads, size_t smem,
                                 const Params& p, cudaStream_t stream, bool early) {
    void* args[] = {const_cast<Params*>(&p)};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ld_relaxed_v2u64(const unsigned long long* p, unsigned long long& a,
                                                 unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2u64(unsigned long long* p, unsigned long long a,
                                                 unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ unsigned long long tag_word(float v, uint32_t tag) {
    return ((unsigned long long)__float_as_uint(v) << 32) | tag;
}

__device__ __forceinline__ float word_value(unsigned long long w) {
    return __uint_as_float((uint32_t)(w >> 32));
}

__device__ __forceinline__ bool word_has(unsigned long long w, uint32_t tag) {
    return (uint32_t)w == tag;
}

__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t* p) {
    return *reinterpret_cast<const volatile int32_t*>(p);
}

__device__ __forceinline__ void set_status(WsHeader* h, int32_t s) {
    atomicCAS(&h->status, 0, s);
}

// The bound on a device-side wait: the workspace's spin_limit when set (a
// caller may shorten it to test the time-out path), else the compiled default.
__device__ __forceinline__ uint32_t wait_limit(const WsHeader* h, uint32_t dflt) {
    const uint32_t v = *reinterpret_cast<const volatile uint32_t*>(&h->spin_limit);
    return v ? v : dflt;
}

}  // namespace sosf
