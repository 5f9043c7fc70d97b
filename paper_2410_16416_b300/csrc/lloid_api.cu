// Host runtime and C ABI of the LLOID filter (include/lloid.h).
//
// Per unit (one SVD bank on one detector) the device holds, for every level k
// (rate f0/2^k): the decimated strain with its history (ping-pong buffers),
// the basis filters of the slices at that level, the level's stacked mixing
// matrix, the basis outputs of the current push, the level's SNR block and
// the short SNR history the interpolator needs.  A push runs every stage as
// one launch over all units of the group (task lists, Sec. II.B), then the
// window-max trigger generator, and copies only the triggers back (Sec. II.B).
//
// Streaming bookkeeping (all per level k, in level-k samples, T = top-rate
// samples pushed so far, a multiple of 2^k_max):
//   decimated strain is final for  m <  A_k = T/2^k - e_k,
//       e_0 = 0, e_{k+1} = ceil((e_k + 1 + 2K)/2) - 1   (the halfband look-ahead);
//   SNR at level k is produced for m < Y_k = T/2^k - Lam_k,
//       Lam_k >= e_k - D_s for every slice s at level k (its FIR needs d up to m - D_s),
//       Lam_{k-1} >= 2 Lam_k + 2K + 1                 (interpolation look-ahead).
// Every push therefore produces exactly B/2^k new samples at every level and
// the top-rate SNR x[n] is final for n < T - Lam_0.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include "lloid.h"
#include "lloid_internal.h"

using namespace lloid;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(SB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

// ---------------------------------------------------------------------------
// halfband taps: g[0] = 1/2, odd taps ~ sinc(j/2) * Kaiser_{beta=8.6}(j), |j| <= 2K,
// scaled so that the odd taps sum to 1/2 (unit DC gain, H(w) + H(pi-w) = 1).
// ---------------------------------------------------------------------------
static double i0_series(double x) {
    double sum = 1.0, term = 1.0;
    for (int k = 1; k < 80; ++k) {
        term *= (0.5 * x / k) * (0.5 * x / k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

static Halfband make_halfband() {
    const double beta = 8.6, half_width = 2.0 * kHalfK;
    const double pi = 3.14159265358979323846;
    double taps[kOddTaps], total = 0.0;
    for (int t = 0; t < kOddTaps; ++t) {
        const double j = 2.0 * t + 1.0;
        const double arg = pi * j / 2.0;
        const double r = std::sqrt(std::max(0.0, 1.0 - (j / half_width) * (j / half_width)));
        taps[t] = std::sin(arg) / arg * i0_series(beta * r) / i0_series(beta);
        total += 2.0 * taps[t];                        // taps at +j and -j
    }
    Halfband g;
    for (int t = 0; t < kOddTaps; ++t) g.odd[t] = (float)(taps[t] * 0.5 / total);
    return g;
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
struct SliceDev {
    int level = 0, L = 0, Q = 0;
    int64_t D = 0;
    float *V = nullptr;       // [L x Q] (FP32 mode)
    float *H = nullptr;       // [2M x ldh] reconstructed FP32 slice filters (refinement in the 16/8-bit modes)
    int ldh = 0;
    int o_row = 0;            // first row in the level's basis-output block
    // tensor-core modes: 8-phase expanded weights and their TMA map
    void *W16 = nullptr;      // [phases x L16 x Kpad] 16- or 8-bit expanded weights
    CUtensorMap *mapW = nullptr;   // device address
    int L16 = 0, Kpad = 0, o_col16 = 0;
    int64_t X0 = 0, phi = 0;
};

struct LevelDev {
    int k = 0;
    int Lk = 0;               // basis vectors of all slices at this level
    int64_t e = 0, lam = 0, Hd = 0, Hy = 0, Bk_max = 0;
    float *dbuf[2] = {nullptr, nullptr};
    int dcur = 0;
    int64_t last_Bk = 0;
    float *ynew = nullptr;    // [2M x ldy]
    int64_t ldy = 0;
    float *yhist[2] = {nullptr, nullptr};   // [2M x Hy]
    int ycur = 0;
    float *Mcat = nullptr;    // [2M x Lk]
    float *obuf = nullptr;    // [Lk x Bk_max]
    std::vector<int> slices;
    // tensor-core modes
    int Lk_pad = 0;           // padded width of the level's basis-output block
    float *colscale = nullptr;   // E4M3: per output column, the basis vector's scale
    float *amax = nullptr;       // E4M3: |strain| maximum accumulators [2] (state)
    void *x16 = nullptr;      // 16-bit (E4M3: two 8-bit terms) copy of the decimated strain (+ window slack)
    int64_t x16_len = 0;      // elements per term; E4M3: the second term starts x16_len bytes after x16
    void *O16 = nullptr;      // basis outputs [Bk_max x Lk_pad], time-major
    void *M16 = nullptr;      // stacked mixing [2M x Lk_pad]
    CUtensorMap *mapO = nullptr, *mapM = nullptr;   // device addresses (box 64 x 256 time rows, 64 x 128 filters)
    CUtensorMap *mapY = nullptr;     // yuni as the finer level's interpolation operand (box 64 x 128, 128-byte swizzle)
    // 16-bit modes, levels k >= 1: SNR rows [history (Hy) | new (B_k)] in one buffer, so the
    // next finer level's epilogue can stage a row segment with one TMA load
    float *yuni = nullptr;    // FP32 mode: unused; BF16 mixing: y as FP16 rows [0, 2M); FP16 mode: y as
                              // BF16 hi rows [0, 2M), lo rows [2M, 4M); ld ldu
    int64_t ldu = 0;
    float *ytmp = nullptr;    // history shift staging, same layout with ld Hy
};

struct TriggerSlot {
    DevTrigger *dbuf = nullptr;
    int32_t *dcount = nullptr;
    int64_t cap = 0;
    DevTrigger *hbuf = nullptr;      // pinned, eager part
    int32_t *hcount = nullptr;       // pinned [3]: count, overflow, device-wait timeout code
    int eager = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};

struct TaskArena {
    char *h = nullptr;               // pinned
    char *d = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool used = false;
};

struct sb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t pop_stream = nullptr;
    cudaStream_t alloc_stream = nullptr;
    bool own_stream = false;
    int64_t budget = 0, used = 0;
    Halfband g;
    int64_t next_unit_id = 0;
    std::vector<sb_unit *> units;
    std::vector<TriggerSlot> slots;
    std::deque<int> pending;         // slot indices in push order
    int next_slot = 0;
    std::vector<TaskArena> arenas;
    int next_arena = 0;
    std::deque<sb_trigger> ready;
    int64_t pushes_completed = 0;    // pushes whose trigger slots have been drained
    bool overflow = false;
    int timeout_code = 0;      // first bounded device wait that expired (0: none)
    std::mutex mu;
    sb_ctx_stats stats{};
    // FP32 refinement scratch (allocated on the first refined push, shared by later pushes)
    RefCand *ref_cands = nullptr;
    float *ref_zpart = nullptr;       // per (candidate, FIR work item) FP32 partial sums of the refinement
    int32_t ref_zpart_items = 0;      // work items per candidate ref_zpart holds
    uint32_t *ref_wmax = nullptr;     // per (unit, template, window) 16-bit maxima of one push
    unsigned long long *ref_cum = nullptr;   // running [candidates, pushes with dropped candidates]
    int64_t ref_wmax_cap = 0;
    void *utab = nullptr;      // tensor-core interpolation operand table (16 variants of U as hi / lo terms)
    int *ref_counters = nullptr;
    // CUDA-graph pushes: one executable graph per group shape, updated in place
    bool graphs = false;
    std::map<std::string, cudaGraphExec_t> graph_execs;
    int64_t graph_launches = 0;
    // mixing-kernel pipeline shapes chosen by timing (no effect on results)
    bool autotune = true;
    // test hook (sb_ctx_test_wait): bound of the basis-FIR kernel's waits and a K chunk its first
    // tile does not load (-1: none)
    uint64_t test_wait_ns = 0;
    int test_skip_chunk = -1;
    MixTuner tuner;
    // profiling: event pairs around each launch, summed per stage on query
    bool prof = false;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> ev_pool;
};

// Read-only bank data (basis, mixing, their 16-bit forms and TMA maps, template
// ids), shared by every unit made from the same bank with svdbank_create_like.
struct Weights {
    sb_ctx *ctx = nullptr;
    std::vector<void *> allocs;
    int64_t bytes = 0;
    ~Weights();
};

struct sb_unit {
    sb_ctx *ctx = nullptr;
    std::shared_ptr<Weights> w;
    int64_t state_bytes = 0;
    int64_t id = 0;
    int32_t detector = 0;
    int M = 0, precision = 0, flags = 0;
    bool tc = false, bf16 = false;
    int mode = 0;                 // basis-FIR operand mode (kModeF16 / kModeBF16 / kModeE4M3)
    int mmode = 0;                // mixing + interpolation operand mode (mix_mode(mode))
    int amax_cur = 0;
    bool refine = false;           // 16-bit modes with a refine threshold: FP32 copies kept for a6
    float thr = 0.f, refine_thr = 0.f;
    double f0 = 0.0;
    int64_t win_len = 0;
    int kmax = 0;
    int64_t Bmax = 0;
    int64_t T = 0;
    int64_t last_B = 0;
    std::vector<SliceDev> slices;
    std::vector<LevelDev> levels;
    WinState *wstate[2] = {nullptr, nullptr};
    int wcur = 0;
    WinPart *part = nullptr;       // 16-bit modes: top-level partial window maxima (scratch)
    int64_t part_rec_max = 0;
    int64_t *tids = nullptr;
    float2 *acorr = nullptr;       // [M][kXiLags] template autocorrelation (null: no xi^2)
    std::vector<void *> allocs;
    int64_t bytes = 0;
    int64_t flops_per_s = 0;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

Weights::~Weights() {
    if (!ctx) return;
    for (void *p : allocs) cudaFreeAsync(p, ctx->stream);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->used -= bytes;
}

// Unit memory comes from the device's stream-ordered pool: allocated on the
// context's allocation stream (synchronised at once, so host copies may follow)
// and returned with cudaFreeAsync on the work stream after the unit's last use,
// so that retiring a unit never stalls queued work.
static int dev_alloc(sb_unit *u, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, u->ctx->alloc_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->ctx->alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SB_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    u->allocs.push_back(*p);
    u->state_bytes += (int64_t)bytes;
    return SB_OK;
}

static int dev_alloc_w(sb_unit *u, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, u->ctx->alloc_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->ctx->alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SB_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    u->w->allocs.push_back(*p);
    u->w->bytes += (int64_t)bytes;
    return SB_OK;
}

static void free_unit_memory(sb_unit *u) {
    for (void *p : u->allocs) cudaFreeAsync(p, u->ctx->stream);
    u->allocs.clear();
}

static void release_marks(sb_ctx *c);

static int activate(sb_ctx *ctx) {
    CK(cudaSetDevice(ctx->device));
    return SB_OK;
}

// Layout parameters of one unit, computed before any allocation (admission).
struct Plan {
    int kmax = 0;
    std::vector<int64_t> e, lam, Hd, Hy, Lk;
    // tensor-core layout
    bool tc = false;
    std::vector<int64_t> Lk_pad, x16_len;                 // per level
    std::vector<int64_t> X0, phi, Kpad, L16, o_col16;     // per slice
    int64_t bytes = 0;
};

static bool is_tc(int precision) { return precision == SB_BF16 || precision == SB_FP16 || precision == SB_FP8; }
static int tc_mode(int precision) {
    return precision == SB_FP8 ? kModeE4M3 : precision == SB_BF16 ? kModeBF16 : kModeF16;
}
static int mode_phases(int mode) { return mode == kModeE4M3 ? 16 : 8; }    // 16 bytes of samples
static int mode_bytes(int mode) { return mode == kModeE4M3 ? 1 : 2; }
static int mode_terms(int mode) { return mode == kModeE4M3 ? 2 : 1; }     // terms of the FIR's strain copy

static int plan_unit(const sb_desc *d, std::vector<int> &levels_of_slice, Plan &P) {
    const int S = d->n_slices;
    levels_of_slice.assign(S, 0);
    int kmax = 0;
    for (int s = 0; s < S; ++s) {
        const sb_slice &sl = d->slices[s];
        if (!(sl.rate_hz > 0) || sl.n_basis <= 0 || sl.n_taps <= 0 || !sl.basis || !sl.mixing)
            return fail(SB_EINVAL, "slice " + std::to_string(s) + ": bad rate, shape or null array");
        const double ratio = d->top_rate_hz / sl.rate_hz;
        const int k = (int)std::lround(std::log2(ratio));
        if (k < 0 || k > 16 || std::fabs(std::ldexp(sl.rate_hz, k) - d->top_rate_hz) > 1e-9 * d->top_rate_hz)
            return fail(SB_EINVAL, "slice " + std::to_string(s) + ": rate must be top_rate / 2^k");
        const double dq = (sl.t_end_s - sl.t_start_s) * sl.rate_hz;
        const double dd = sl.t_start_s * sl.rate_hz;
        if (sl.t_start_s < 0 || std::fabs(dq - std::llround(dq)) > 1e-6 || std::fabs(dd - std::llround(dd)) > 1e-6 ||
            std::llround(dq) != sl.n_taps)
            return fail(SB_EINVAL, "slice " + std::to_string(s) + ": span must hold n_taps samples on its rate grid");
        levels_of_slice[s] = k;
        kmax = std::max(kmax, k);
    }
    P.kmax = kmax;
    const int NL = kmax + 1;
    P.e.assign(NL, 0);
    P.lam.assign(NL, 0);
    P.Hd.assign(NL, 0);
    P.Hy.assign(NL, 0);
    P.Lk.assign(NL, 0);
    for (int k = 0; k + 1 < NL; ++k) P.e[k + 1] = (P.e[k] + 1 + 2 * kHalfK + 1) / 2 - 1;   // ceil(x/2) - 1
    std::vector<int64_t> minD(NL, INT64_MAX);
    for (int s = 0; s < S; ++s) {
        const int k = levels_of_slice[s];
        minD[k] = std::min<int64_t>(minD[k], std::llround(d->slices[s].t_start_s * d->slices[s].rate_hz));
        P.Lk[k] += d->slices[s].n_basis;
    }
    for (int k = kmax; k >= 0; --k) {
        int64_t lam = 0;
        if (k < kmax) lam = 2 * P.lam[k + 1] + 2 * kHalfK + 1;
        if (minD[k] != INT64_MAX) lam = std::max(lam, P.e[k] - minD[k]);
        P.lam[k] = std::max<int64_t>(lam, 0);
    }
    for (int k = 0; k < NL; ++k) {
        int64_t hd = 0;
        if (k < kmax) hd = 2 * P.e[k + 1] - P.e[k] + 2 * kHalfK;
        for (int s = 0; s < S; ++s) {
            if (levels_of_slice[s] != k) continue;
            const int64_t D = std::llround(d->slices[s].t_start_s * d->slices[s].rate_hz);
            // 16-bit modes: 128 extra samples for the FP32 refinement's halo below the push
            hd = std::max(hd, P.lam[k] - P.e[k] + D + d->slices[s].n_taps - 1 + (is_tc(d->precision) ? 128 : 0));
        }
        P.Hd[k] = round_up(std::max<int64_t>(hd, 1), 32);
        if (k >= 1) P.Hy[k] = round_up((P.lam[k - 1] + 2 * kHalfK) / 2 + 1 - P.lam[k], 8);   // 16 bytes of BF16
    }
    // tensor-core layout: every slice's 16-bit window start X0 is a multiple of 8
    // samples (16 bytes, the TMA/descriptor alignment); phi zero columns pad W.
    P.tc = is_tc(d->precision);
    P.Lk_pad.assign(NL, 0);
    P.x16_len.assign(NL, 0);
    P.X0.assign(S, 0);
    P.phi.assign(S, 0);
    P.Kpad.assign(S, 0);
    P.L16.assign(S, 0);
    P.o_col16.assign(S, 0);
    std::vector<int64_t> kpad_max(NL, 0);
    const int mode = tc_mode(d->precision), ph = mode_phases(mode), by = mode_bytes(mode);
    const int mmode = mix_mode(mode), mby = mode_bytes(mmode);
    const int lpt = kTcM / ph;                       // basis vectors per 128-row weight tile
    for (int s = 0; s < S; ++s) {
        const int k = levels_of_slice[s];
        const int64_t D = std::llround(d->slices[s].t_start_s * d->slices[s].rate_hz);
        const int64_t Q = d->slices[s].n_taps;
        const int64_t start = P.Hd[k] + P.e[k] - P.lam[k] - D - (Q - 1);    // >= 0 by the choice of Hd
        P.X0[s] = start / ph * ph;                     // window starts on 16 bytes
        P.phi[s] = start - P.X0[s];
        P.Kpad[s] = round_up(Q + ph - 1 + P.phi[s], 128 / by);
        P.L16[s] = round_up(d->slices[s].n_basis, lpt);
        P.o_col16[s] = P.Lk_pad[k];
        P.Lk_pad[k] += P.L16[s];
        kpad_max[k] = std::max(kpad_max[k], P.Kpad[s]);
    }
    for (int k = 0; k < NL; ++k) {
        P.Lk_pad[k] = round_up(P.Lk_pad[k], 16);        // K per 16-bit mixing MMA
        // (a multiple of 256 elements, so the E4M3 second term starts 256-byte aligned)
        P.x16_len[k] = round_up(P.Hd[k] + (d->max_push_samples >> k) + (int64_t)ph * kTcN + kpad_max[k] + 64, 256);
    }
    // bytes
    const int64_t M2 = 2 * (int64_t)d->n_templates;
    int64_t b = 0;
    for (int k = 0; k < NL; ++k) {
        const int64_t Bk = d->max_push_samples >> k;
        const int64_t ldy = round_up(Bk, 4);
        b += 2 * (P.Hd[k] + Bk) * 4;                 // decimated strain ping-pong
        b += M2 * ldy * 4;                           // SNR block
        b += 2 * M2 * P.Hy[k] * 4;                   // SNR history ping-pong
        if (P.tc) {
            b -= M2 * ldy * 4 + 2 * M2 * P.Hy[k] * 4;   // replaced by the unified level buffer
            if (k >= 1) b += (M2 * round_up(P.Hy[k] + Bk, 8) + M2 * P.Hy[k]) * 2 * y_planes(mmode) + 128;
            else if (d->flags & SB_FLAG_KEEP_SNR) b += M2 * ldy * 4;
            b += P.x16_len[k] * by * mode_terms(mode) + ((Bk + 256) * P.Lk_pad[k] + M2 * P.Lk_pad[k]) * mby + 2 * 128;
            if (mode == kModeE4M3) b += (P.Lk_pad[k] + 2) * 4;
        } else {
            b += M2 * P.Lk[k] * 4 + P.Lk[k] * Bk * 4;    // mixing + basis outputs
        }
    }
    for (int s = 0; s < S; ++s)
        b += P.tc ? (int64_t)ph * P.L16[s] * P.Kpad[s] * by + 128
                  : (int64_t)d->slices[s].n_basis * d->slices[s].n_taps * 4;
    b += 2 * (int64_t)d->n_templates * sizeof(WinState) + d->n_templates * 8;
    if (P.tc) b += ((d->max_push_samples + 255) / 256) * 4 * (int64_t)d->n_templates * sizeof(WinPart);
    if (P.tc && d->refine_threshold > 0.0f)            // FP32 reconstructed slice filters for the refinement
        for (int s = 0; s < S; ++s) b += M2 * round_up(d->slices[s].n_taps, 4) * 4;
    P.bytes = b;
    return SB_OK;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" int sb_ctx_create(int32_t device, void *stream, int64_t hbm_budget_bytes, sb_ctx **out) {
    if (!out) return fail(SB_EINVAL, "out is null");
    *out = nullptr;
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(SB_EINVAL, "no such CUDA device");
    sb_ctx *c = new sb_ctx();
    c->device = device;
    if (activate(c) != SB_OK) { delete c; return SB_ECUDA; }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(SB_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->pop_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->alloc_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return fail(SB_ECUDA, "cudaStreamCreate failed");
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete c; return fail(SB_ECUDA, "cudaMemGetInfo failed"); }
    c->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (int64_t)(0.9 * (double)fr);
    c->g = make_halfband();
    c->slots.resize(8);
    for (auto &s : c->slots) {
        if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.hcount, 3 * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&s.dcount, 3 * sizeof(int32_t)) != cudaSuccess) {
            sb_ctx_destroy(c);
            return fail(SB_ENOMEM, "trigger slot allocation failed");
        }
    }
    c->arenas.resize(4);
    for (auto &a : c->arenas) {
        if (cudaEventCreateWithFlags(&a.ev, cudaEventDisableTiming) != cudaSuccess) {
            sb_ctx_destroy(c);
            return fail(SB_ECUDA, "event creation failed");
        }
    }
    {   // interpolation operands of the tensor-core mixing kernel (constant per context)
        std::vector<uint8_t> ut(tc_interp_table_bytes());
        tc_interp_table(c->g, ut.data());
        if (cudaMalloc(&c->utab, ut.size()) != cudaSuccess ||
            cudaMemcpy(c->utab, ut.data(), ut.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            sb_ctx_destroy(c);
            return fail(SB_ENOMEM, "interpolation table allocation failed");
        }
    }
    *out = c;
    return SB_OK;
}

extern "C" int sb_ctx_destroy(sb_ctx *c) {
    if (!c) return SB_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    while (!c->units.empty()) svdbank_destroy(c->units.back());
    for (auto &s : c->slots) {
        if (s.dbuf) cudaFree(s.dbuf);
        if (s.dcount) cudaFree(s.dcount);
        if (s.hbuf) cudaFreeHost(s.hbuf);
        if (s.hcount) cudaFreeHost(s.hcount);
        if (s.ev) cudaEventDestroy(s.ev);
    }
    for (auto &a : c->arenas) {
        if (a.h) cudaFreeHost(a.h);
        if (a.d) cudaFree(a.d);
        if (a.ev) cudaEventDestroy(a.ev);
    }
    release_marks(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto &kv : c->graph_execs) cudaGraphExecDestroy(kv.second);
    c->graph_execs.clear();
    if (c->ref_cands) cudaFree(c->ref_cands);
    if (c->ref_zpart) cudaFree(c->ref_zpart);
    if (c->ref_wmax) cudaFree(c->ref_wmax);
    if (c->ref_cum) cudaFree(c->ref_cum);
    if (c->utab) cudaFree(c->utab);
    if (c->ref_counters) cudaFree(c->ref_counters);
    if (c->stream) cudaStreamSynchronize(c->stream);      // unit memory returned on the work stream
    if (c->pop_stream) cudaStreamDestroy(c->pop_stream);
    if (c->alloc_stream) cudaStreamDestroy(c->alloc_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return SB_OK;
}

// The context's work stream and device, with that device made current (for the conditioner,
// condition.cu, whose work is ordered with the context's pushes).
int lloid_ctx_stream(sb_ctx *c, cudaStream_t *stream, int *device) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    if (activate(c) != SB_OK) return SB_ECUDA;
    *stream = c->stream;
    *device = c->device;
    return SB_OK;
}

extern "C" int sb_ctx_sync(sb_ctx *c) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    if (activate(c) != SB_OK) return SB_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    return SB_OK;
}

// ---------------------------------------------------------------------------
// units
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// tensor-core bank layout
// ---------------------------------------------------------------------------
static uint16_t to16(float v, bool bf16) {
    if (bf16) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        return *reinterpret_cast<uint16_t *>(&h);
    }
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
}

// 2-D K-major tensor map over a row-major [outer x inner] 16-bit matrix with
// 128-byte swizzle and a (64 x box_outer) box; out-of-range elements read as 0.
// The driver's tensor-map encoder, looked up through the runtime so that the
// library does not link libcuda (it loads on machines without a driver).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static void put_elem(std::vector<uint8_t> &buf, size_t i, float v, int mode) {
    if (mode == kModeE4M3) {
        __nv_fp8_e4m3 q(v);
        buf[i] = *reinterpret_cast<uint8_t *>(&q);
    } else {
        const uint16_t h = to16(v, mode == kModeBF16);
        std::memcpy(&buf[2 * i], &h, 2);
    }
}

// Bytes of K per row of a mixing-operand chunk: the padded K when it fits 32 or 64 bytes, else
// 128-byte chunks (the swizzle span matches, so small-K levels move no padding).
static int mix_kbytes(int64_t Lk_pad, int mode) {
    const int64_t b = Lk_pad * mode_bytes(mode);
    return b <= 32 ? 32 : b <= 64 ? 64 : 128;
}

static int encode_map(CUtensorMap *out, void *base, int mode, uint64_t inner, uint64_t outer, uint32_t box_outer,
                      int row_bytes = 128) {
    auto encode = tensor_map_encoder();
    if (!encode) return fail(SB_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int by = mode_bytes(mode);
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * by};
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / by), box_outer};    // row_bytes-byte rows
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(out, mode == kModeE4M3   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                             : mode == kModeBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                        2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        row_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                        : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                          : CU_TENSOR_MAP_SWIZZLE_32B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SB_OK;
}

static int upload_map(sb_unit *u, const CUtensorMap &h, CUtensorMap **dev, bool weights) {
    int rc = weights ? dev_alloc_w(u, (void **)dev, sizeof(CUtensorMap)) : dev_alloc(u, (void **)dev, sizeof(CUtensorMap));
    if (rc) return rc;
    CK(cudaMemcpy(*dev, &h, sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return SB_OK;
}

// The refinement's filters: H_s = M_s V_s, each template's two real FP32
// filters of slice s (step a3's mixing summed over the basis, Sec. II.A), one FP32 GEMM on the device
// at create time; [2M][ldh] rows, ldh = Q rounded up to 4.
static int build_refine_filters(sb_unit *u, SliceDev &sd, const sb_slice &sl) {
    const int64_t M2 = 2 * (int64_t)u->M;
    sd.ldh = (int)round_up(sd.Q, 4);
    int rc = dev_alloc_w(u, (void **)&sd.H, M2 * sd.ldh * 4);
    if (rc) return rc;
    std::vector<float> a((size_t)M2 * sd.L), v((size_t)sd.L * sd.Q);
    for (size_t i = 0; i < a.size(); ++i) a[i] = (float)sl.mixing[i];
    for (size_t i = 0; i < v.size(); ++i) v[i] = (float)sl.basis[i];
    cudaStream_t st = u->ctx->alloc_stream;
    float *dA = nullptr, *dV = nullptr;
    GemmTask *dT = nullptr;
    GemmTask t{};
    t.lda = sd.L;
    t.ldb = sd.Q;
    t.ldc = sd.ldh;
    t.M = (int32_t)M2;
    t.N = sd.Q;
    t.K = sd.L;
    t.tiles_n = (sd.Q + kGemmTN - 1) / kGemmTN;
    const int tiles = (int)((M2 + kGemmTM - 1) / kGemmTM) * t.tiles_n;
    cudaError_t e = cudaMallocAsync(&dA, a.size() * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dV, v.size() * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dT, sizeof(GemmTask), st);
    if (e == cudaSuccess) {
        t.A = dA;
        t.B = dV;
        t.C = sd.H;
        e = cudaMemcpyAsync(dA, a.data(), a.size() * 4, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dV, v.data(), v.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, &t, sizeof(GemmTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_gemm_fp32(dT, 1, tiles, st);
    if (dA) cudaFreeAsync(dA, st);
    if (dV) cudaFreeAsync(dV, st);
    if (dT) cudaFreeAsync(dT, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SB_ECUDA, std::string("refinement filters: ") + cudaGetErrorString(e));
    }
    return SB_OK;
}

// W[(l, r)][j] = v[l][r + Q - 1 + phi - j] (zero outside 0 <= q < Q), rows
// ordered per 128-row tile t as lpt r + l_loc with l = lpt t + l_loc (lpt = 16
// basis vectors x 8 phases in the 16-bit modes, 8 x 16 in E4M3).  E4M3 rows are
// scaled by 448 / max|v_l| (per-basis-vector absmax scaling).
static int upload_expanded_weights(sb_unit *u, SliceDev &sd, const double *basis, std::vector<float> &vscale) {
    const int ph = mode_phases(u->mode), by = mode_bytes(u->mode), lpt = kTcM / ph;
    const int64_t rows = (int64_t)ph * sd.L16, K = sd.Kpad;
    vscale.assign(sd.L, 1.0f);
    if (u->mode == kModeE4M3)
        for (int l = 0; l < sd.L; ++l) {
            double m = 0.0;
            for (int q = 0; q < sd.Q; ++q) m = std::max(m, std::fabs(basis[(int64_t)l * sd.Q + q]));
            vscale[l] = m > 0.0 ? (float)(m / 448.0) : 1.0f;
        }
    std::vector<uint8_t> w((size_t)(rows * K * by), 0);
    for (int64_t t = 0; t < sd.L16 / lpt; ++t)
        for (int r = 0; r < ph; ++r)
            for (int ll = 0; ll < lpt; ++ll) {
                const int64_t l = lpt * t + ll;
                if (l >= sd.L) continue;
                const int64_t row = kTcM * t + lpt * r + ll;
                for (int64_t j = 0; j < K; ++j) {
                    const int64_t q = r + sd.Q - 1 + sd.phi - j;
                    if (q >= 0 && q < sd.Q) put_elem(w, row * K + j, (float)(basis[l * sd.Q + q] / vscale[l]), u->mode);
                }
            }
    int rc = dev_alloc_w(u, &sd.W16, w.size());
    if (rc) return rc;
    CK(cudaMemcpy(sd.W16, w.data(), w.size(), cudaMemcpyHostToDevice));
    CUtensorMap m;
    if ((rc = encode_map(&m, sd.W16, u->mode, K, rows, kTcM))) return rc;
    return upload_map(u, m, &sd.mapW, true);
}

// Stacked mixing matrix of every level in the mixing kernel's operand type
// (BF16 for E4M3 units).  E4M3: colscale holds each basis vector's scale, which
// the basis FIR epilogue applies before writing its BF16 outputs.
static int upload_tc_mixing_and_maps(sb_unit *u, const sb_desc *d, const std::vector<std::vector<float>> &vscale) {
    const int64_t M2 = 2 * (int64_t)u->M;
    const int by = mode_bytes(u->mmode);
    for (auto &L : u->levels) {
        if (L.Lk_pad == 0) continue;
        std::vector<uint8_t> m((size_t)(M2 * L.Lk_pad * by), 0);
        for (int s : L.slices) {
            const SliceDev &sd = u->slices[s];
            const double *mx = d->slices[s].mixing;
            for (int64_t a = 0; a < M2; ++a)
                for (int l = 0; l < sd.L; ++l)
                    put_elem(m, a * L.Lk_pad + sd.o_col16 + l, (float)mx[a * sd.L + l], u->mmode);
        }
        int rc;
        if ((rc = dev_alloc_w(u, &L.M16, m.size()))) return rc;
        CK(cudaMemcpy(L.M16, m.data(), m.size(), cudaMemcpyHostToDevice));
        CUtensorMap hm;
        if ((rc = encode_map(&hm, L.M16, u->mmode, L.Lk_pad, M2, 128, mix_kbytes(L.Lk_pad, u->mmode)))) return rc;
        if ((rc = upload_map(u, hm, &L.mapM, true))) return rc;
        if (u->mode == kModeE4M3) {
            std::vector<float> cs(L.Lk_pad, 0.0f);
            for (int s : L.slices)
                for (int l = 0; l < u->slices[s].L; ++l) cs[u->slices[s].o_col16 + l] = vscale[s][l];
            if ((rc = dev_alloc_w(u, (void **)&L.colscale, L.Lk_pad * 4))) return rc;
            CK(cudaMemcpy(L.colscale, cs.data(), L.Lk_pad * 4, cudaMemcpyHostToDevice));
        }
    }
    return SB_OK;
}

static int validate_desc(const sb_desc *d, std::vector<int> &lvl, Plan &P) {
    if (!d) return fail(SB_EINVAL, "null description");
    if (d->n_templates <= 0 || d->n_slices <= 0 || !d->slices || !(d->top_rate_hz > 0) || !(d->window_s > 0) ||
        d->max_push_samples <= 0 || d->max_push_samples > (int64_t(1) << 30))
        return fail(SB_EINVAL, "bad bank description (templates, slices, rate, window or max_push_samples "
                               "outside (0, 2^30])");
    if (d->precision != SB_FP32 && !is_tc(d->precision))
        return fail(SB_EINVAL, "precision mode not available in this build");
    const double wl = d->window_s * d->top_rate_hz;
    if (std::fabs(wl - std::llround(wl)) > 1e-6 || std::llround(wl) < 1)
        return fail(SB_EINVAL, "window_s * top_rate_hz must be a positive integer");
    int rc = plan_unit(d, lvl, P);
    if (rc) return rc;
    if (P.kmax >= kRefMaxLevels)
        return fail(SB_EINVAL, "slice rates go down to top_rate_hz / 2^" + std::to_string(kRefMaxLevels - 1) +
                                   " at most");
    if (P.tc && std::llround(wl) < 128)
        return fail(SB_EINVAL, "tensor-core modes need window_s * top_rate_hz >= 128");
    if (P.tc && d->refine_threshold > 0.0f && (P.kmax >= kRefMaxLevels || d->n_slices > kRefMaxSlices))
        return fail(SB_EINVAL, "refinement supports at most " + std::to_string(kRefMaxLevels) + " levels and " +
                                   std::to_string(kRefMaxSlices) + " slices");
    if (d->max_push_samples % (1LL << P.kmax))
        return fail(SB_EINVAL, "max_push_samples must be a multiple of 2^k_max");
    if (d->autocorr)                          // xi^2 lag profiles: finite, lag 0 equal to 1
        for (int i = 0; i < d->n_templates; ++i)
            for (int j = 0; j < kXiLags; ++j) {
                const double re = d->autocorr[((size_t)i * kXiLags + j) * 2];
                const double im = d->autocorr[((size_t)i * kXiLags + j) * 2 + 1];
                if (!std::isfinite(re) || !std::isfinite(im) ||
                    (j == kXiJ && std::fabs(re - 1.0) + std::fabs(im) > 1e-6))
                    return fail(SB_EINVAL, "autocorr of template " + std::to_string(i) +
                                               " is not finite or its lag 0 is not 1");
            }
    return SB_OK;
}

static int64_t plan_flops(const sb_desc *d) {
    double f = 0.0;
    for (int s = 0; s < d->n_slices; ++s) {
        const sb_slice &sl = d->slices[s];
        f += 2.0 * sl.n_basis * (sl.n_taps + 2.0 * d->n_templates) * sl.rate_hz;
    }
    return (int64_t)std::llround(f);
}

// Streaming state of a unit (decimated strain, SNR blocks and histories, basis
// outputs, trigger partials and open windows), zero-initialised; every field of
// u->levels except the state pointers must be set.
static int alloc_state(sb_unit *u) {
    const int64_t M2 = 2 * (int64_t)u->M;
    // one allocation carved into 256-byte aligned pieces, zeroed by one memset
    struct Piece { void **dst; int64_t bytes; };
    std::vector<Piece> pieces;
    auto want = [&](void **dst, int64_t bytes) { pieces.push_back({dst, std::max<int64_t>(bytes, 16)}); };
    for (auto &L : u->levels) {
        const int k = L.k;
        for (int b = 0; b < 2; ++b) want((void **)&L.dbuf[b], (L.Hd + L.Bk_max) * 4);
        if (!u->tc) {
            want((void **)&L.ynew, M2 * L.ldy * 4);
            if (L.Hy > 0)
                for (int b = 0; b < 2; ++b) want((void **)&L.yhist[b], M2 * L.Hy * 4);
            if (L.Lk > 0) want((void **)&L.obuf, (int64_t)L.Lk * L.Bk_max * 4);
            continue;
        }
        if (k >= 1) {
            want((void **)&L.yuni, M2 * L.ldu * 2 * y_planes(u->mmode));
            want((void **)&L.ytmp, M2 * L.Hy * 2 * y_planes(u->mmode));
        } else if (u->flags & SB_FLAG_KEEP_SNR) {
            want((void **)&L.ynew, M2 * L.ldy * 4);
        }
        want(&L.x16, L.x16_len * mode_bytes(u->mode) * mode_terms(u->mode));
        if (L.Lk_pad > 0) want(&L.O16, (L.Bk_max + 256) * L.Lk_pad * mode_bytes(u->mmode));
        if (u->mode == kModeE4M3) want((void **)&L.amax, 2 * 4);
    }
    if (u->tc) {
        u->part_rec_max = ((u->Bmax + 255) / 256) * 4;
        want((void **)&u->part, u->part_rec_max * u->M * (int64_t)sizeof(WinPart));
    }
    for (int b = 0; b < 2; ++b) want((void **)&u->wstate[b], u->M * (int64_t)sizeof(WinState));
    int64_t total = 0;
    for (auto &p : pieces) total += round_up(p.bytes, 256);
    char *base = nullptr;
    int rc = dev_alloc(u, (void **)&base, total);
    if (rc) return rc;
    CK(cudaMemsetAsync(base, 0, total, u->ctx->alloc_stream));
    int64_t off = 0;
    for (auto &p : pieces) {
        *p.dst = base + off;
        off += round_up(p.bytes, 256);
    }
    std::vector<WinState> ws(u->M);
    for (auto &w : ws) { w.mag2 = -1.0f; w.re = w.im = w.pk = w.dt = w.xi2 = 0.0f; w.flags = 0; w.n = -1; }
    for (int b = 0; b < 2; ++b)
        CK(cudaMemcpyAsync(u->wstate[b], ws.data(), u->M * sizeof(WinState), cudaMemcpyHostToDevice,
                           u->ctx->alloc_stream));
    for (auto &L : u->levels) {
        if (!u->tc) continue;
        if (L.k >= 1) {                          // y as FP16 rows [2M x ldu], or BF16 hi / lo rows [4M x ldu]
            CUtensorMap hy;                      // level k - 1's interpolation operand (64 samples x 128 filters)
            const int np = y_planes(u->mmode);
            if ((rc = encode_map(&hy, L.yuni, np == 1 ? kModeF16 : kModeBF16, L.ldu, np * M2, 128))) return rc;
            if ((rc = upload_map(u, hy, &L.mapY, false))) return rc;
        }
        if (L.Lk_pad == 0) continue;
        CUtensorMap ho;
        if ((rc = encode_map(&ho, L.O16, u->mmode, L.Lk_pad, L.Bk_max + 256, 256, mix_kbytes(L.Lk_pad, u->mmode))))
            return rc;
        if ((rc = upload_map(u, ho, &L.mapO, false))) return rc;
    }
    CK(cudaStreamSynchronize(u->ctx->alloc_stream));
    return SB_OK;
}

extern "C" int svdbank_plan(const sb_desc *d, sb_unit_info *info) {
    if (!d || !info) return fail(SB_EINVAL, "null argument");
    std::vector<int> lvl;
    Plan P;
    int rc = validate_desc(d, lvl, P);
    if (rc) return rc;
    std::memset(info, 0, sizeof(*info));
    info->n_templates = d->n_templates;
    info->n_slices = d->n_slices;
    info->k_max = P.kmax;
    info->precision = d->precision;
    info->latency_samples = P.lam[0];
    info->device_bytes = P.bytes;
    info->flops_per_second = plan_flops(d);
    return SB_OK;
}

extern "C" int svdbank_create(sb_ctx *c, const sb_desc *d, int32_t detector, sb_unit **out) {
    if (!c || !d || !out) return fail(SB_EINVAL, "null argument");
    *out = nullptr;
    std::vector<int> lvl;
    Plan P;
    int rc = validate_desc(d, lvl, P);
    if (rc) return rc;
    const double wl = d->window_s * d->top_rate_hz;
    if (activate(c) != SB_OK) return SB_ECUDA;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->used + P.bytes > c->budget)
            return fail(SB_EBUSY, "HBM budget exhausted: unit needs " + std::to_string(P.bytes) + " bytes, " +
                                      std::to_string(c->budget - c->used) + " free in budget");
        c->used += P.bytes;
    }
    sb_unit *u = new sb_unit();
    u->ctx = c;
    u->detector = detector;
    u->M = d->n_templates;
    u->precision = d->precision;
    u->tc = is_tc(d->precision);
    u->bf16 = d->precision == SB_BF16;
    u->mode = tc_mode(d->precision);
    u->mmode = mix_mode(u->mode);
    u->refine = u->tc && d->refine_threshold > 0.0f;
    u->flags = d->flags;
    u->thr = d->threshold;
    u->refine_thr = d->refine_threshold;
    u->f0 = d->top_rate_hz;
    u->win_len = std::llround(wl);
    u->kmax = P.kmax;
    u->Bmax = d->max_push_samples;
    u->bytes = P.bytes;
    const int64_t M2 = 2 * (int64_t)u->M;
    auto cleanup = [&](int code) {
        free_unit_memory(u);
        {
            std::lock_guard<std::mutex> lk(c->mu);
            c->used -= P.bytes;
        }
        if (u->w) u->w->bytes = 0;                // nothing of this bank was charged yet
        delete u;
        return code;
    };
    u->w = std::make_shared<Weights>();
    u->w->ctx = c;
    u->levels.resize(P.kmax + 1);
    for (int k = 0; k <= P.kmax; ++k) {
        LevelDev &L = u->levels[k];
        L.k = k;
        L.e = P.e[k];
        L.lam = P.lam[k];
        L.Hd = P.Hd[k];
        L.Hy = P.Hy[k];
        L.Lk = (int)P.Lk[k];
        L.Bk_max = u->Bmax >> k;
        L.ldy = round_up(L.Bk_max, 4);
        if (u->tc) {
            L.Lk_pad = (int)P.Lk_pad[k];
            L.x16_len = P.x16_len[k];
            if (k >= 1) L.ldu = round_up(L.Hy + L.Bk_max, 8);
        }
        if (L.Lk > 0 && !u->tc) {
            if ((rc = dev_alloc_w(u, (void **)&L.Mcat, M2 * L.Lk * 4))) return cleanup(rc);
        }
    }
    // slices: basis filters and the per-level stacked mixing matrices
    std::vector<std::vector<float>> mcat(P.kmax + 1);
    for (int k = 0; k <= P.kmax; ++k) mcat[k].assign(M2 * u->levels[k].Lk, 0.0f);
    std::vector<int> row_of_level(P.kmax + 1, 0);
    std::vector<std::vector<float>> vscale(d->n_slices);
    u->flops_per_s = plan_flops(d);
    for (int s = 0; s < d->n_slices; ++s) {
        const sb_slice &sl = d->slices[s];
        SliceDev sd;
        sd.level = lvl[s];
        sd.L = sl.n_basis;
        sd.Q = sl.n_taps;
        sd.D = std::llround(sl.t_start_s * sl.rate_hz);
        sd.o_row = row_of_level[sd.level];
        row_of_level[sd.level] += sd.L;
        if (!u->tc) {
            std::vector<float> v((size_t)sd.L * sd.Q);
            for (size_t i = 0; i < v.size(); ++i) v[i] = (float)sl.basis[i];
            if ((rc = dev_alloc_w(u, (void **)&sd.V, v.size() * 4))) return cleanup(rc);
            if (cudaMemcpy(sd.V, v.data(), v.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return cleanup(fail(SB_ECUDA, "basis upload"));
            const int Lk = u->levels[sd.level].Lk;
            for (int64_t a = 0; a < M2; ++a)
                for (int l = 0; l < sd.L; ++l) mcat[sd.level][a * Lk + sd.o_row + l] = (float)sl.mixing[a * sd.L + l];
        }
        if (u->tc) {
            sd.L16 = (int)P.L16[s];
            sd.Kpad = (int)P.Kpad[s];
            sd.o_col16 = (int)P.o_col16[s];
            sd.X0 = P.X0[s];
            sd.phi = P.phi[s];
            if ((rc = upload_expanded_weights(u, sd, sl.basis, vscale[s]))) return cleanup(rc);
            if (u->refine && (rc = build_refine_filters(u, sd, sl))) return cleanup(rc);
        }
        u->levels[sd.level].slices.push_back(s);
        u->slices.push_back(sd);
    }
    for (int k = 0; k <= P.kmax && !u->tc; ++k) {
        LevelDev &L = u->levels[k];
        if (L.Lk == 0) continue;
        if (cudaMemcpy(L.Mcat, mcat[k].data(), mcat[k].size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(SB_ECUDA, "mixing upload"));
    }
    if (u->tc && (rc = upload_tc_mixing_and_maps(u, d, vscale))) return cleanup(rc);
    std::vector<int64_t> ids(u->M);
    for (int i = 0; i < u->M; ++i) ids[i] = d->template_ids ? d->template_ids[i] : i;
    if ((rc = dev_alloc_w(u, (void **)&u->tids, u->M * 8))) return cleanup(rc);
    if (cudaMemcpy(u->tids, ids.data(), u->M * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(fail(SB_ECUDA, "template id upload"));
    if (d->autocorr) {                        // xi^2 lag profiles, FP32 on the device
        std::vector<float2> ac((size_t)u->M * kXiLags);          // checked by validate_desc
        for (size_t e = 0; e < ac.size(); ++e)
            ac[e] = make_float2((float)d->autocorr[2 * e], (float)d->autocorr[2 * e + 1]);
        if ((rc = dev_alloc_w(u, (void **)&u->acorr, ac.size() * sizeof(float2)))) return cleanup(rc);
        if (cudaMemcpy(u->acorr, ac.data(), ac.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(SB_ECUDA, "autocorrelation upload"));
    }
    if ((rc = alloc_state(u))) return cleanup(rc);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->used += u->state_bytes + u->w->bytes - P.bytes;     // reservation -> measured
        u->bytes = u->state_bytes;
        u->id = c->next_unit_id++;
        c->units.push_back(u);
    }
    *out = u;
    return SB_OK;
}

extern "C" int svdbank_create_like(sb_ctx *c, sb_unit *src, int32_t detector, sb_unit **out) {
    if (!c || !src || !out) return fail(SB_EINVAL, "null argument");
    if (src->ctx != c) return fail(SB_EINVAL, "source unit belongs to another context");
    *out = nullptr;
    if (activate(c) != SB_OK) return SB_ECUDA;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->used + src->state_bytes > c->budget)
            return fail(SB_EBUSY, "HBM budget exhausted: unit state needs " + std::to_string(src->state_bytes) +
                                      " bytes, " + std::to_string(c->budget - c->used) + " free in budget");
        c->used += src->state_bytes;
    }
    sb_unit *u = new sb_unit();
    u->ctx = c;
    u->w = src->w;
    u->detector = detector;
    u->M = src->M;
    u->precision = src->precision;
    u->tc = src->tc;
    u->bf16 = src->bf16;
    u->mode = src->mode;
    u->mmode = src->mmode;
    u->refine = src->refine;
    u->flags = src->flags;
    u->thr = src->thr;
    u->refine_thr = src->refine_thr;
    u->f0 = src->f0;
    u->win_len = src->win_len;
    u->kmax = src->kmax;
    u->Bmax = src->Bmax;
    u->flops_per_s = src->flops_per_s;
    u->slices = src->slices;
    u->tids = src->tids;
    u->acorr = src->acorr;
    u->levels = src->levels;
    for (auto &L : u->levels) {                  // fresh streaming state, shared weights
        L.amax = nullptr;
        L.dbuf[0] = L.dbuf[1] = nullptr;
        L.dcur = 0;
        L.last_Bk = 0;
        L.ynew = nullptr;
        L.yhist[0] = L.yhist[1] = nullptr;
        L.ycur = 0;
        L.obuf = nullptr;
        L.x16 = nullptr;
        L.O16 = nullptr;
        L.mapO = nullptr;
        L.mapY = nullptr;
        L.yuni = nullptr;
        L.ytmp = nullptr;
    }
    const int64_t reserved = src->state_bytes;
    int rc = alloc_state(u);
    std::lock_guard<std::mutex> lk(c->mu);
    c->used += u->state_bytes - reserved;
    if (rc) {
        free_unit_memory(u);
        c->used -= u->state_bytes;
        delete u;
        return rc;
    }
    u->bytes = u->state_bytes;
    u->id = c->next_unit_id++;
    c->units.push_back(u);
    *out = u;
    return SB_OK;
}

extern "C" int svdbank_destroy(sb_unit *u) {
    if (!u) return SB_OK;
    sb_ctx *c = u->ctx;
    cudaSetDevice(c->device);
    free_unit_memory(u);                  // stream-ordered: after every push already queued
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->used -= u->bytes;
        c->units.erase(std::remove(c->units.begin(), c->units.end(), u), c->units.end());
    }
    delete u;                             // the last unit of a bank releases its weights (~Weights)
    return SB_OK;
}

extern "C" int sb_unit_query(const sb_unit *u, sb_unit_info *info) {
    if (!u || !info) return fail(SB_EINVAL, "null argument");
    info->unit = u->id;
    info->n_templates = u->M;
    info->n_slices = (int32_t)u->slices.size();
    info->k_max = u->kmax;
    info->precision = u->precision;
    info->latency_samples = u->levels[0].lam;
    info->samples_pushed = u->T;
    info->device_bytes = u->bytes;
    info->flops_per_second = u->flops_per_s;
    return SB_OK;
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
static cudaEvent_t pool_event(sb_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs one stage's launches (fn returns a cudaError_t and adds its kernel
// count to *n); with profiling on, brackets them with events.
template <class F>
static int run_stage(sb_ctx *c, int stage, F fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        a = pool_event(c);
        b = pool_event(c);
        CK(cudaEventRecord(a, c->stream));
    }
    int n = 0;
    cudaError_t e = fn(&n);
    if (e != cudaSuccess) return fail(SB_ECUDA, std::string("stage launch: ") + cudaGetErrorString(e));
    c->stats.kernel_launches += n;
    if (c->prof) {
        CK(cudaEventRecord(b, c->stream));
        c->marks.push_back({stage, a, b});
    }
    return SB_OK;
}

extern "C" int sb_ctx_get_stats(sb_ctx *c, sb_ctx_stats *out) {
    if (!c || !out) return fail(SB_EINVAL, "null argument");
    unsigned long long cum[2] = {0, 0};
    if (c->ref_cum) {                          // refinement totals live on the device
        if (activate(c) != SB_OK) return SB_ECUDA;
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaMemcpy(cum, c->ref_cum, sizeof(cum), cudaMemcpyDeviceToHost));
    }
    std::lock_guard<std::mutex> lk(c->mu);
    *out = c->stats;
    out->refine_candidates = (int64_t)cum[0];
    out->refine_dropped = (int64_t)cum[1];
    out->graph_launches = c->graph_launches;
    out->autotune_shapes = (int64_t)c->tuner.best.size();
    out->autotune_launches = c->tuner.timed_launches;
    return SB_OK;
}

static void release_marks(sb_ctx *c) {
    for (auto &m : c->marks) {
        c->ev_pool.push_back(m.a);
        c->ev_pool.push_back(m.b);
    }
    c->marks.clear();
}

extern "C" int sb_ctx_graphs(sb_ctx *c, int32_t enable) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    std::lock_guard<std::mutex> lk(c->mu);
    c->graphs = enable != 0;
    return SB_OK;
}

extern "C" int sb_ctx_test_wait(sb_ctx *c, int64_t wait_limit_ns, int32_t skip_fir_chunk) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    if (wait_limit_ns < 0) return fail(SB_EINVAL, "wait_limit_ns must be >= 0");
    std::lock_guard<std::mutex> lk(c->mu);
    c->test_wait_ns = (uint64_t)wait_limit_ns;
    c->test_skip_chunk = skip_fir_chunk < 0 ? -1 : skip_fir_chunk;
    return SB_OK;
}

extern "C" int sb_ctx_autotune(sb_ctx *c, int32_t enable) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    std::lock_guard<std::mutex> lk(c->mu);
    c->autotune = enable != 0;
    return SB_OK;
}

extern "C" int sb_ctx_autotune_choices(sb_ctx *c, int32_t *out, int32_t cap) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    if (cap < 0 || (cap > 0 && !out)) return fail(SB_EINVAL, "bad output buffer");
    std::lock_guard<std::mutex> lk(c->mu);
    const int n = (int)c->tuner.best.size();
    for (int i = 0; i < n && i < cap; ++i) {
        const auto &kv = c->tuner.best[i];
        out[4 * i] = (int32_t)kv.first;
        out[4 * i + 1] = kv.second.n_st;
        out[4 * i + 2] = kv.second.n_u;
        out[4 * i + 3] = kv.second.n_win;
    }
    return n;
}

extern "C" int sb_ctx_profile(sb_ctx *c, int32_t enable) {
    if (!c) return fail(SB_EINVAL, "ctx is null");
    if (activate(c) != SB_OK) return SB_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaStreamSynchronize(c->stream));
    if (enable) release_marks(c);
    c->prof = enable != 0;
    return SB_OK;
}

extern "C" int sb_ctx_stage_times(sb_ctx *c, double *ms, int64_t *launches, int32_t n_stages) {
    if (!c || !ms || !launches || n_stages < 0 || n_stages > SB_N_STAGES) return fail(SB_EINVAL, "bad argument");
    if (activate(c) != SB_OK) return SB_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n_stages; ++i) { ms[i] = 0.0; launches[i] = 0; }
    for (auto &m : c->marks) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, m.a, m.b));
        if (m.stage < n_stages) { ms[m.stage] += t; launches[m.stage] += 1; }
    }
    return SB_OK;
}

// ---------------------------------------------------------------------------
// triggers
// ---------------------------------------------------------------------------
static int drain_slot(sb_ctx *c, TriggerSlot &s, bool block) {
    if (!s.pending) return SB_OK;
    if (block) {
        CK(cudaEventSynchronize(s.ev));
    } else {
        cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaErrorNotReady) return 1;
        if (q != cudaSuccess) return fail(SB_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(q));
    }
    int64_t n = s.hcount[0];
    if (s.hcount[1]) c->overflow = true;
    if (s.hcount[2]) c->timeout_code = s.hcount[2];
    if (n > s.cap) n = s.cap;
    std::vector<sb_trigger> tr((size_t)n);
    const int64_t ne = std::min<int64_t>(n, s.eager);
    if (ne > 0) std::memcpy(tr.data(), s.hbuf, ne * sizeof(sb_trigger));
    if (n > ne) {
        CK(cudaMemcpyAsync(tr.data() + ne, s.dbuf + ne, (n - ne) * sizeof(sb_trigger), cudaMemcpyDeviceToHost,
                           c->pop_stream));
        CK(cudaStreamSynchronize(c->pop_stream));
        c->stats.d2h_bytes += (n - ne) * (int64_t)sizeof(sb_trigger);
    }
    std::sort(tr.begin(), tr.end(), [](const sb_trigger &a, const sb_trigger &b) {
        if (a.window != b.window) return a.window < b.window;
        if (a.unit != b.unit) return a.unit < b.unit;
        return a.template_id < b.template_id;
    });
    for (auto &t : tr) c->ready.push_back(t);
    s.pending = false;
    return SB_OK;
}

static int drain_ready_slots(sb_ctx *c, bool block_all) {
    while (!c->pending.empty()) {
        const int idx = c->pending.front();
        int rc = drain_slot(c, c->slots[idx], block_all);
        if (rc == 1) break;                      // not finished yet
        if (rc < 0) return rc;
        c->pending.pop_front();
        c->pushes_completed += 1;
    }
    return SB_OK;
}

extern "C" int sb_ctx_progress(sb_ctx *c, int64_t *pushed, int64_t *completed) {
    if (!c || !pushed || !completed) return fail(SB_EINVAL, "null argument");
    if (activate(c) != SB_OK) return SB_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    int rc = drain_ready_slots(c, false);
    if (rc < 0) return rc;
    *pushed = c->stats.pushes;
    *completed = c->pushes_completed;
    return SB_OK;
}

extern "C" int triggers_pop(sb_ctx *c, sb_trigger *out, int64_t cap, int64_t *n_out) {
    if (!c || !n_out || (cap > 0 && !out)) return fail(SB_EINVAL, "null argument");
    *n_out = 0;
    if (activate(c) != SB_OK) return SB_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    int rc = drain_ready_slots(c, false);
    if (rc < 0) return rc;
    int64_t n = 0;
    while (n < cap && !c->ready.empty()) {
        out[n++] = c->ready.front();
        c->ready.pop_front();
    }
    *n_out = n;
    c->stats.triggers += n;
    if (c->timeout_code) {
        const int code = c->timeout_code;
        c->timeout_code = 0;
        return fail(SB_ETIMEOUT, "a tensor-core kernel's bounded wait expired (site " + std::to_string(code) + ")");
    }
    if (c->overflow) {
        c->overflow = false;
        return fail(SB_EOVERFLOW, "a push produced more triggers than its buffer holds; some were dropped");
    }
    return SB_OK;
}

// ---------------------------------------------------------------------------
// push
// ---------------------------------------------------------------------------
struct Packer {
    std::vector<char> buf;
    size_t add(const void *p, size_t bytes) {
        size_t off = round_up((int64_t)buf.size(), 256);
        buf.resize(off + bytes);
        if (bytes) std::memcpy(buf.data() + off, p, bytes);
        return off;
    }
    size_t reserve(size_t bytes) {            // zeroed space, filled in later
        size_t off = round_up((int64_t)buf.size(), 256);
        buf.resize(off + bytes, 0);
        return off;
    }
};

// Graph mode: ends the push's stream capture and launches it, reusing (updating in place)
// the executable graph of the same group shape when CUDA accepts the update.
static int end_capture_and_launch(sb_ctx *c, const std::string &key, cudaStream_t st) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || !g) {
        cudaGetLastError();
        return fail(SB_ECUDA, std::string("push capture: ") + cudaGetErrorString(e));
    }
    auto it = c->graph_execs.find(key);
    if (it != c->graph_execs.end()) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(it->second, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(it->second);
            c->graph_execs.erase(it);
            it = c->graph_execs.end();
        }
    }
    if (it == c->graph_execs.end()) {
        if (c->graph_execs.size() >= 64) {        // many shapes (serving): start over
            for (auto &kv : c->graph_execs) cudaGraphExecDestroy(kv.second);
            c->graph_execs.clear();
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(SB_ECUDA, std::string("push graph instantiation: ") + cudaGetErrorString(e));
        }
        it = c->graph_execs.emplace(key, ex).first;
    }
    cudaGraphDestroy(g);
    e = cudaGraphLaunch(it->second, st);
    if (e != cudaSuccess) return fail(SB_ECUDA, std::string("push graph launch: ") + cudaGetErrorString(e));
    c->graph_launches += 1;
    return SB_OK;
}

// Ends a capture left open by an error inside a captured push.
struct CaptureGuard {
    cudaStream_t st = nullptr;
    bool active = false;
    ~CaptureGuard() {
        if (!active) return;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
};

static int arena_acquire(sb_ctx *c, size_t bytes, TaskArena *&out) {
    TaskArena &a = c->arenas[c->next_arena];
    c->next_arena = (c->next_arena + 1) % (int)c->arenas.size();
    if (a.used) CK(cudaEventSynchronize(a.ev));
    if (a.cap < bytes) {
        if (a.h) cudaFreeHost(a.h);
        if (a.d) cudaFree(a.d);
        a.h = nullptr;
        a.d = nullptr;
        size_t cap = (size_t)round_up((int64_t)bytes * 2, 1 << 16);
        CK(cudaMallocHost(&a.h, cap));
        CK(cudaMalloc(&a.d, cap));
        a.cap = cap;
    }
    out = &a;
    return SB_OK;
}

static int slot_acquire(sb_ctx *c, int64_t need, TriggerSlot *&out, int &idx) {
    idx = c->next_slot;
    c->next_slot = (c->next_slot + 1) % (int)c->slots.size();
    TriggerSlot &s = c->slots[idx];
    if (s.pending) {
        // ring full: finish the oldest pushes first (keeps trigger order)
        while (!c->pending.empty()) {
            const int j = c->pending.front();
            int rc = drain_slot(c, c->slots[j], true);
            if (rc < 0) return rc;
            c->pending.pop_front();
            c->pushes_completed += 1;
            if (j == idx) break;
        }
    }
    if (s.cap < need) {
        if (s.dbuf) cudaFree(s.dbuf);
        if (s.hbuf) cudaFreeHost(s.hbuf);
        s.dbuf = nullptr;
        s.hbuf = nullptr;
        const int64_t cap = round_up(std::max<int64_t>(need, 1024), 1024);
        CK(cudaMalloc(&s.dbuf, cap * sizeof(DevTrigger)));
        s.eager = (int)std::min<int64_t>(cap, 64);
        CK(cudaMallocHost(&s.hbuf, s.eager * sizeof(DevTrigger)));
        s.cap = cap;
    }
    out = &s;
    return SB_OK;
}

// ---------------------------------------------------------------------------
// push: the task lists of one grouped push, one builder per stage
// ---------------------------------------------------------------------------
namespace {

constexpr int kNM = 3;                           // tensor-core operand modes (kModeF16, kModeBF16, kModeE4M3)

// Every task list of one grouped push.  Each builder appends one unit's tasks in level order, so
// every list runs unit by unit; the counters size the launches and the scratch.
struct PushPlan {
    int kall = 0;                                // deepest level over the units
    std::vector<CopyTask> dcopy, ycopy, yshift1, yshift2;
    std::vector<CascadeTask> casc;               // a1 cascade + 16-bit copies, one cluster per unit
    std::vector<GemmTask> fir;                   // SB_FP32 basis FIR
    std::vector<std::vector<UpTask>> ups;        // SB_FP32 interpolation, per level
    std::vector<std::vector<GemmTask>> recon;    // SB_FP32 mixing, per level
    std::vector<WinTask> win;                    // SB_FP32 trigger generator
    std::vector<TcFirTask> tfir[kNM];            // tensor-core basis FIR, per operand mode
    std::vector<std::vector<TcMixUpTask>> tmix[kNM];   // tensor-core mixing, per operand mode and level
    std::vector<WinFinTask> wfin;                // 16/8-bit window finalisation
    std::vector<RefUnit> refu;                   // FP32 refinement of the 16/8-bit candidates
    int64_t ref_max_windows = 0, ref_wmax_total = 0;
    int32_t ref_max_items = 0;                   // largest FIR work-item count of a refined unit
    int kpad_max[kNM] = {0, 0, 0};
    int max_hd = 0, max_hy = 0, max_rows = 0;
    int64_t trig_need = 0;
    // launch sizes (assign_tiles)
    int fir_tiles = 0;
    std::vector<int> recon_tiles;
    int tfir_tiles[kNM] = {0, 0, 0};
    std::vector<int> tmix_tiles[kNM];
    std::vector<MixLaunch> tmix_ml[kNM];
    int wfin_warps = 0, win_warps = 0;

    PushPlan(int n_units, int kall_)
        : kall(kall_), casc(n_units), ups(kall_ + 1), recon(kall_ + 1), recon_tiles(kall_ + 1, 0) {
        for (int h = 0; h < kNM; ++h) {
            tmix[h].resize(kall + 1);
            tmix_tiles[h].assign(kall + 1, 0);
            tmix_ml[h].resize(kall + 1);
        }
    }
};

// This unit's slice of the refinement's window-maxima scratch during one push (an offset; the
// addresses are set at packing).
struct RefineWindows {
    bool on = false;
    int64_t win0 = 0;                            // window of slot 0
    int32_t n_wslot = 0;
    int64_t wmax_off = 0;
};

RefineWindows refine_windows(PushPlan &P, const sb_unit *u, int64_t B) {
    RefineWindows rw;
    const int64_t first_n0 = u->T - u->levels[0].lam;
    const int64_t start0 = std::max<int64_t>(first_n0, 0), end0 = first_n0 + B;
    rw.on = end0 > start0 && u->refine;
    rw.win0 = rw.on ? start0 / u->win_len : 0;
    rw.n_wslot = rw.on ? (int32_t)((end0 - 1) / u->win_len - rw.win0 + 1) : 0;
    rw.wmax_off = P.ref_wmax_total;
    if (rw.on) P.ref_wmax_total += (int64_t)u->M * rw.n_wslot;
    return rw;
}

// History shifts of the decimated strain, the a1 cascade and (tensor-core units) the 16-bit copies.
void plan_streams(PushPlan &P, int i, sb_unit *u, int64_t B) {
    const int64_t Tp = u->T;
    CascadeTask &cs = P.casc[i];
    for (int k = 0; k <= u->kmax; ++k) {
        LevelDev &L = u->levels[k];
        const int nb = 1 - L.dcur;
        CopyTask ct{};
        ct.cur = L.dbuf[L.dcur];
        ct.dst = L.dbuf[nb];
        ct.rows = 1;
        ct.n = (int32_t)L.Hd;
        ct.off = (int32_t)L.last_Bk;
        P.dcopy.push_back(ct);
        P.max_hd = std::max<int>(P.max_hd, (int)L.Hd);
        if (k < u->kmax) {
            LevelDev &N = u->levels[k + 1];
            DecimTask dt{};
            dt.in = L.dbuf[nb];
            dt.out = N.dbuf[1 - N.dcur] + N.Hd;
            dt.in_base = L.Hd + L.e - 2 * N.e;
            dt.first_m = (Tp >> (k + 1)) - N.e;
            dt.n_out = (int32_t)(B >> (k + 1));
            cs.lev[k] = dt;
            cs.n_lev = k + 1;
        }
        if (u->tc) {
            float *am = L.amax ? L.amax + u->amax_cur : nullptr;
            float *am_next = L.amax ? L.amax + (1 - u->amax_cur) : nullptr;
            void *x_lo = mode_terms(u->mode) == 2 ? static_cast<uint8_t *>(L.x16) + L.x16_len : nullptr;
            cs.conv[k] = HalfConvTask{L.dbuf[nb], L.x16, L.Hd + (B >> k), am, am_next, x_lo};
            cs.n_conv = k + 1;
            cs.mode = u->mode;
        }
    }
}

// Tensor-core units: a2 basis FIR per slice, a3 + a4 (+ a5 partials at the top) per level, and the
// interpolation history of every level below the top for the next push.
void plan_tc(PushPlan &P, sb_unit *u, int64_t B, const RefineWindows &rw) {
    const int64_t Tp = u->T;
    const int M2 = 2 * u->M;
    const int h = u->mode;
    for (int k = 0; k <= u->kmax; ++k) {
        LevelDev &L = u->levels[k];
        const int64_t Bk = B >> k;
        const float *am = L.amax ? L.amax + u->amax_cur : nullptr;
        const void *x_lo = mode_terms(u->mode) == 2 ? static_cast<uint8_t *>(L.x16) + L.x16_len : nullptr;
        for (int s : L.slices) {
            const SliceDev &sd = u->slices[s];
            TcFirTask f{};
            f.mapW = sd.mapW;
            f.x = L.x16;
            f.X0 = sd.X0;
            f.O = L.O16;
            f.ldo = L.Lk_pad;
            f.o_col = sd.o_col16;
            f.Kpad = sd.Kpad;
            f.Bk = (int32_t)Bk;
            const int64_t ph = mode_phases(u->mode);       // samples per Hankel block
            f.tiles_n = (int32_t)(((Bk + ph - 1) / ph + kTcN - 1) / kTcN);
            f.tiles_m = sd.L16 / (kTcM / mode_phases(u->mode));
            f.xamax = am;
            f.colscale = L.colscale;
            f.x_lo = x_lo;
            P.tfir[h].push_back(f);
            P.kpad_max[h] = std::max(P.kpad_max[h], sd.Kpad);
        }
        TcMixUpTask mt{};
        mt.mapM = L.mapM;
        mt.mapO = L.mapO;
        if (k < u->kmax) mt.mapY = u->levels[k + 1].mapY;
        mt.Y = k == 0 ? L.ynew : nullptr;             // SB_FLAG_KEEP_SNR
        mt.ldy = L.ldy;
        mt.Yh = k >= 1 ? reinterpret_cast<uint16_t *>(L.yuni) : nullptr;
        mt.ldu = L.ldu;
        mt.yst_col0 = L.Hy;
        mt.kbytes = mix_kbytes(L.Lk_pad, u->mmode);
        mt.part = k == 0 ? u->part : nullptr;
        if (k == 0 && rw.on) {
            mt.wmax = reinterpret_cast<uint32_t *>(rw.wmax_off + 1);   // offset + 1; address at packing
            mt.win0 = rw.win0;
            mt.n_wslot = rw.n_wslot;
            mt.thr2 = u->refine_thr * u->refine_thr;
        }
        mt.first_n = (Tp >> k) - L.lam;
        mt.win_len = u->win_len;
        mt.Lk_pad = L.Lk_pad;
        mt.M2 = M2;
        mt.M = u->M;
        mt.Bk = (int32_t)Bk;
        mt.lam = (int32_t)L.lam;
        mt.in_off = k < u->kmax ? (int32_t)(u->levels[k + 1].lam + u->levels[k + 1].Hy) : 0;
        mt.tiles_t = (int32_t)((Bk + 255) / 256);
        mt.tiles_a = (M2 + 127) / 128;
        mt.n_rec = mt.tiles_t * 4;
        P.tmix[u->mmode][k].push_back(mt);
        if (k >= 1) {           // next push's interpolation history: columns [Bk, Bk + Hy) -> [0, Hy)
            // (in place when the two ranges are disjoint, else through the staging buffer)
            const bool direct = Bk >= L.Hy;
            CopyTask a{};
            a.cur = L.yuni;
            a.ld_cur = L.ldu;
            a.dst = direct ? L.yuni : L.ytmp;
            a.ld_dst = direct ? L.ldu : L.Hy;
            a.rows = M2;
            a.n = (int32_t)L.Hy;
            a.off = (int32_t)Bk;
            a.elem16 = y_planes(u->mmode);
            P.yshift1.push_back(a);
            P.max_hy = std::max<int>(P.max_hy, (int)L.Hy);
            if (!direct) {
                CopyTask bt{};
                bt.cur = L.ytmp;
                bt.ld_cur = L.Hy;
                bt.dst = L.yuni;
                bt.ld_dst = L.ldu;
                bt.rows = M2;
                bt.n = (int32_t)L.Hy;
                bt.off = 0;
                bt.elem16 = y_planes(u->mmode);
                P.yshift2.push_back(bt);
            }
        }
    }
}

// SB_FP32 units: a2 basis FIR per slice (Toeplitz operand), a4 interpolation and a3 mixing per
// level, and the SNR history of every level below the top.
void plan_fp32(PushPlan &P, sb_unit *u, int64_t B) {
    const int64_t Tp = u->T;
    const int M2 = 2 * u->M;
    for (int k = 0; k <= u->kmax; ++k) {
        LevelDev &L = u->levels[k];
        const int nb = 1 - L.dcur;
        const int64_t Bk = B >> k;
        for (int s : L.slices) {
            const SliceDev &sd = u->slices[s];
            GemmTask g{};
            g.A = sd.V;
            g.lda = sd.Q;
            g.B = L.dbuf[nb];
            g.ldb = L.Hd + L.e - L.lam - sd.D;
            g.C = L.obuf + (int64_t)sd.o_row * L.Bk_max;
            g.ldc = L.Bk_max;
            g.M = sd.L;
            g.N = (int32_t)Bk;
            g.K = sd.Q;
            g.beta = 0;
            g.toeplitz = 1;
            P.fir.push_back(g);
        }
        if (k < u->kmax) {
            LevelDev &N = u->levels[k + 1];
            UpTask ut{};
            ut.hist = N.yhist[N.ycur];
            ut.cur = N.ynew;
            ut.out = L.ynew;
            ut.ld_hist = N.Hy;
            ut.ld_cur = N.ldy;
            ut.ld_out = L.ldy;
            ut.n_hist = (int32_t)N.Hy;
            ut.rows = M2;
            ut.n_out = (int32_t)Bk;
            ut.lam_out = (int32_t)L.lam;
            ut.in_off = (int32_t)(N.lam + N.Hy);
            ut.n_cur = (int32_t)(B >> (k + 1));
            ut.first_n = (Tp >> k) - L.lam;
            P.ups[k].push_back(ut);
        }
        if (L.Lk > 0) {
            GemmTask g{};
            g.A = L.Mcat;
            g.lda = L.Lk;
            g.B = L.obuf;
            g.ldb = L.Bk_max;
            g.C = L.ynew;
            g.ldc = L.ldy;
            g.M = M2;
            g.N = (int32_t)Bk;
            g.K = L.Lk;
            g.beta = k < u->kmax ? 1 : 0;
            g.toeplitz = 0;
            P.recon[k].push_back(g);
        }
        if (k >= 1 && L.Hy > 0) {
            CopyTask yt{};
            yt.hist = L.yhist[L.ycur];
            yt.cur = L.ynew;
            yt.dst = L.yhist[1 - L.ycur];
            yt.ld_hist = L.Hy;
            yt.ld_cur = L.ldy;
            yt.ld_dst = L.Hy;
            yt.n_hist = (int32_t)L.Hy;
            yt.rows = M2;
            yt.n = (int32_t)L.Hy;
            yt.off = (int32_t)Bk;
            P.ycopy.push_back(yt);
            P.max_hy = std::max<int>(P.max_hy, (int)L.Hy);
        }
    }
}

// The trigger generator of the top level: window finalisation (16/8-bit units, after the mixing
// kernel's partial maxima) with the FP32 refinement of the candidates, or the window maxima of
// the FP32 SNR block (SB_FP32 units).
void plan_triggers(PushPlan &P, sb_unit *u, int64_t B, const RefineWindows &rw) {
    const int64_t Tp = u->T;
    LevelDev &L0 = u->levels[0];
    const int64_t first_n = Tp - L0.lam;
    const int64_t start = std::max<int64_t>(first_n, 0), end = first_n + B;
    if (end > start && u->refine) {
        RefUnit r{};
        r.part = u->part;
        r.first_n = first_n;
        r.win_len = u->win_len;
        r.thr2 = u->refine_thr * u->refine_thr;
        r.keep2 = u->mode == kModeE4M3 ? kRefKeep8 : kRefKeep16;
        r.win0 = rw.win0;
        r.n_wslot = rw.n_wslot;
        r.wmax = reinterpret_cast<uint32_t *>(rw.wmax_off);         // offset; the base is added before packing
        r.kmax = u->kmax;
        r.M = u->M;
        r.n_rec = (int32_t)((B + kRefTile - 1) / kRefTile) * 4;
        r.B = (int32_t)B;
        r.n_slices = (int32_t)u->slices.size();
        r.acorr = u->acorr;
        for (int k = 0; k <= u->kmax; ++k) {
            LevelDev &L = u->levels[k];
            r.lv_d[k] = L.dbuf[1 - L.dcur];
            r.lv_origin[k] = (Tp >> k) - L.e - L.Hd;
            r.lv_len[k] = L.Hd + (B >> k);
        }
        for (size_t si = 0; si < u->slices.size(); ++si) {
            const SliceDev &sd = u->slices[si];
            r.sl_H[si] = sd.H;
            r.sl_ldh[si] = sd.ldh;
            r.sl_D[si] = sd.D;
            r.sl_Q[si] = sd.Q;
            r.sl_level[si] = sd.level;
            r.sl_item0[si + 1] = r.sl_item0[si] + (sd.Q + kRefQC - 1) / kRefQC;
        }
        P.ref_max_items = std::max(P.ref_max_items, r.sl_item0[u->slices.size()]);
        P.ref_max_windows = std::max<int64_t>(P.ref_max_windows, (int64_t)r.M * r.n_wslot);
        P.refu.push_back(r);
    }
    if (end > start && u->tc) {
        WinFinTask w{};
        w.part = u->part;
        w.state_in = u->wstate[u->wcur];
        w.state_out = u->wstate[1 - u->wcur];
        w.template_ids = u->tids;
        w.unit_id = u->id;
        w.win_len = u->win_len;
        w.first_n = first_n;
        w.start_abs = start;
        w.end_abs = end;
        w.n_rec = (int32_t)(((B + 255) / 256) * 4);
        w.M = u->M;
        w.n_win = (int32_t)((end - 1) / u->win_len - start / u->win_len + 1);
        w.threshold = u->thr;
        // the refinement's window maxima cover every possible trigger when its threshold is lower
        if (rw.on && u->refine_thr < u->thr * (1.0f - 1e-6f)) {
            w.n_wslot = rw.n_wslot;
            w.wmax = reinterpret_cast<const uint32_t *>(rw.wmax_off + 1);   // offset + 1; the base is added at packing
        }
        P.wfin.push_back(w);
        P.trig_need += (int64_t)u->M * w.n_win;
    } else if (end > start) {
        WinTask w{};
        w.x = L0.ynew;
        w.ldx = L0.ldy;
        w.state_in = u->wstate[u->wcur];
        w.state_out = u->wstate[1 - u->wcur];
        w.template_ids = u->tids;
        w.first_n = first_n;
        w.unit_id = u->id;
        w.win_len = u->win_len;
        w.n = (int32_t)B;
        w.M = u->M;
        w.n_seg = (int32_t)((end - 1) / u->win_len - start / u->win_len + 1);
        w.threshold = u->thr;
        w.acorr = u->acorr;
        P.win.push_back(w);
        P.trig_need += (int64_t)u->M * w.n_seg;
    }
}

int assign_gemm_tiles(std::vector<GemmTask> &v) {
    int tot = 0;
    for (auto &g : v) {
        g.tiles_n = (g.N + kGemmTN - 1) / kGemmTN;
        const int tiles_m = (g.M + kGemmTM - 1) / kGemmTM;
        g.tile_begin = tot;
        tot += tiles_m * g.tiles_n;
    }
    return tot;
}

// Tile and warp offsets of every task list (each launch walks its tasks by global tile or warp),
// and the launch description of every mixing launch.
void assign_tiles(PushPlan &P) {
    P.fir_tiles = assign_gemm_tiles(P.fir);
    for (int k = 0; k <= P.kall; ++k) P.recon_tiles[k] = assign_gemm_tiles(P.recon[k]);
    for (int h = 0; h < kNM; ++h) {
        for (auto &f : P.tfir[h]) {
            f.tile_begin = P.tfir_tiles[h];
            P.tfir_tiles[h] += f.tiles_m * f.tiles_n;
        }
        for (int k = 0; k <= P.kall; ++k)
            for (auto &m : P.tmix[h][k]) {
                m.tile_begin = P.tmix_tiles[h][k];
                P.tmix_tiles[h][k] += m.tiles_t * m.tiles_a;
                MixLaunch &ml = P.tmix_ml[h][k];
                if (m.Yh) ml.store_y = true;
                if (m.mapY) ml.interp = true;
                ml.kbytes = std::max(ml.kbytes, (int)m.kbytes);
                const int kc = 128 / mode_bytes(h);                  // K elements per 128-byte chunk
                ml.max_nk = std::max(ml.max_nk, (m.Lk_pad + kc - 1) / kc);
            }
    }
    for (auto &w : P.wfin) {
        w.warp_begin = P.wfin_warps;
        P.wfin_warps += w.M * w.n_win;
    }
    for (auto &w : P.win) {
        w.warp_begin = P.win_warps;
        P.win_warps += w.M * w.n_seg;
    }
}

}  // namespace

namespace {

// Offsets of one push's task lists in its packed task block.
struct PushOffsets {
    size_t dcopy = 0, casc = 0, fir = 0, win = 0, ycopy = 0, wfin = 0, refu = 0, ys1 = 0, ys2 = 0, scopy = 0;
    std::vector<size_t> ups, recon;
    size_t tfir[kNM] = {0, 0, 0};
    std::vector<size_t> tmix[kNM];
};

// The refinement's scratch (window-maxima table, candidate list and counters, FIR partial sums),
// grown on demand; the units' window-maxima offsets become addresses.  Runs before packing.
int prepare_refine_scratch(sb_ctx *c, PushPlan &P, cudaStream_t st) {
    if (P.refu.empty()) return SB_OK;
    if (!c->ref_cands) {                   // candidate list, counters and running totals
        CK(cudaMalloc(&c->ref_cands, kRefCandCap * sizeof(RefCand)));
        CK(cudaMalloc(&c->ref_counters, 4 * sizeof(int)));
        CK(cudaMalloc(&c->ref_cum, 2 * sizeof(unsigned long long)));
        CK(cudaMemsetAsync(c->ref_cum, 0, 2 * sizeof(unsigned long long), st));
    }
    if (c->ref_wmax_cap < P.ref_wmax_total) {
        CK(cudaStreamSynchronize(st));
        if (c->ref_wmax) cudaFree(c->ref_wmax);
        c->ref_wmax = nullptr;
        c->ref_wmax_cap = std::max(P.ref_wmax_total, 2 * c->ref_wmax_cap);
        CK(cudaMalloc(&c->ref_wmax, c->ref_wmax_cap * sizeof(uint32_t)));
    }
    if (c->ref_zpart_items < P.ref_max_items) {       // per (candidate, FIR work item) partial sums
        CK(cudaStreamSynchronize(st));
        if (c->ref_zpart) cudaFree(c->ref_zpart);
        c->ref_zpart = nullptr;
        c->ref_zpart_items = P.ref_max_items;
        CK(cudaMalloc(&c->ref_zpart, (size_t)kRefSplitCap * P.ref_max_items * 2 * kRefSpan * sizeof(float)));
    }
    for (auto &r : P.refu) r.wmax = c->ref_wmax + reinterpret_cast<intptr_t>(r.wmax);   // offset -> address
    for (auto &w : P.wfin)
        if (w.wmax) w.wmax = c->ref_wmax + (reinterpret_cast<intptr_t>(w.wmax) - 1);
    for (int h = 0; h < kNM; ++h)
        for (auto &m : P.tmix[h][0])
            if (m.wmax) m.wmax = c->ref_wmax + (reinterpret_cast<intptr_t>(m.wmax) - 1);
    CK(cudaMemsetAsync(c->ref_wmax, 0, P.ref_wmax_total * sizeof(uint32_t), st));   // before this push's kernels
    return SB_OK;
}

PushOffsets pack_tasks(Packer &pk, const PushPlan &P) {
    PushOffsets o;
    o.ups.resize(P.kall + 1);
    o.recon.resize(P.kall + 1);
    o.dcopy = pk.add(P.dcopy.data(), P.dcopy.size() * sizeof(CopyTask));
    o.casc = pk.add(P.casc.data(), P.casc.size() * sizeof(CascadeTask));
    o.fir = pk.add(P.fir.data(), P.fir.size() * sizeof(GemmTask));
    for (int k = 0; k <= P.kall; ++k) {
        o.ups[k] = pk.add(P.ups[k].data(), P.ups[k].size() * sizeof(UpTask));
        o.recon[k] = pk.add(P.recon[k].data(), P.recon[k].size() * sizeof(GemmTask));
    }
    o.win = pk.add(P.win.data(), P.win.size() * sizeof(WinTask));
    for (int h = 0; h < kNM; ++h) {
        o.tfir[h] = pk.add(P.tfir[h].data(), P.tfir[h].size() * sizeof(TcFirTask));
        o.tmix[h].resize(P.kall + 1);
        for (int k = 0; k <= P.kall; ++k)
            o.tmix[h][k] = pk.add(P.tmix[h][k].data(), P.tmix[h][k].size() * sizeof(TcMixUpTask));
    }
    o.ycopy = pk.add(P.ycopy.data(), P.ycopy.size() * sizeof(CopyTask));
    o.wfin = pk.add(P.wfin.data(), P.wfin.size() * sizeof(WinFinTask));
    o.refu = pk.add(P.refu.data(), P.refu.size() * sizeof(RefUnit));
    o.ys1 = pk.add(P.yshift1.data(), P.yshift1.size() * sizeof(CopyTask));
    o.ys2 = pk.add(P.yshift2.data(), P.yshift2.size() * sizeof(CopyTask));
    return o;
}

// Every stage of one push, in order, on the stream (inside the capture in graph mode).
// derr: the push's device error word; to: its trigger slot.
int launch_stages(sb_ctx *c, const PushPlan &P, const PushOffsets &o, char *D, int *derr, const TrigOut &to,
                  int n_units, int64_t B, bool tune_now, cudaStream_t st) {
    int rc;
    // 1. history shifts of the decimated strain
    if ((rc = run_stage(c, SB_STAGE_HISTORY, [&](int *n) {
             *n = P.dcopy.empty() ? 0 : 1;
             return launch_copy((CopyTask *)(D + o.dcopy), (int)P.dcopy.size(), 1, P.max_hd, st);
         })))
        return rc;
    // 2. new top-rate strain
    if ((rc = run_stage(c, SB_STAGE_STRAIN, [&](int *n) {
             *n = 1;
             return launch_copy((CopyTask *)(D + o.scopy), n_units, 1, (int)B, st);
         })))
        return rc;
    // 3. a1 decimation cascade of every unit and the 16-bit copies for the tensor-core FIR (one launch)
    if ((rc = run_stage(c, SB_STAGE_DECIMATE, [&](int *n) {
             *n = 1;
             return launch_cascade((CascadeTask *)(D + o.casc), n_units, c->g, st);
         })))
        return rc;
    // 4. a2 basis FIR, all slices of all units at once
    if (!P.fir.empty() && (rc = run_stage(c, SB_STAGE_FIR, [&](int *n) {
                             *n = 1;
                             return launch_gemm_fp32((GemmTask *)(D + o.fir), (int)P.fir.size(), P.fir_tiles, st);
                         })))
        return rc;
    for (int h = 0; h < kNM; ++h)
        if (!P.tfir[h].empty() && (rc = run_stage(c, SB_STAGE_FIR, [&](int *n) {
                                     *n = 1;
                                     return launch_tc_fir((TcFirTask *)(D + o.tfir[h]), (int)P.tfir[h].size(),
                                                          P.tfir_tiles[h], P.kpad_max[h], h, derr, st, c->test_wait_ns,
                                                          c->test_skip_chunk);
                                 })))
            return rc;
    // 5. a4 + a3 from the lowest rate up
    for (int k = P.kall; k >= 0; --k) {
        if (!P.ups[k].empty() &&
            (rc = run_stage(c, SB_STAGE_UPSAMPLE, [&](int *n) {
                 *n = 1;
                 return launch_upsample((UpTask *)(D + o.ups[k]), (int)P.ups[k].size(), P.max_rows, (int)(B >> k),
                                        c->g, st);
             })))
            return rc;
        if (!P.recon[k].empty() &&
            (rc = run_stage(c, SB_STAGE_MIX, [&](int *n) {
                 *n = 1;
                 return launch_gemm_fp32((GemmTask *)(D + o.recon[k]), (int)P.recon[k].size(), P.recon_tiles[k], st);
             })))
            return rc;
        for (int h = 0; h < kNM; ++h)
            if (!P.tmix[h][k].empty() &&
                (rc = run_stage(c, SB_STAGE_MIX, [&](int *n) {
                     const int64_t timed0 = c->tuner.timed_launches;
                     cudaError_t e = launch_tc_mixup((TcMixUpTask *)(D + o.tmix[h][k]), (int)P.tmix[h][k].size(),
                                                     P.tmix_tiles[h][k], P.tmix_ml[h][k],
                                                     c->utab, h, derr, c->autotune ? &c->tuner : nullptr, tune_now,
                                                     st);
                     *n = (int)std::max<int64_t>(1, c->tuner.timed_launches - timed0);
                     return e;
                 })))
                return rc;
    }
    // a6: FP32 refinement of the top level's candidate maxima (16-bit modes)
    if (!P.refu.empty()) {
        CK(cudaMemsetAsync(c->ref_counters, 0, 4 * sizeof(int), st));
        if ((rc = run_stage(c, SB_STAGE_REFINE, [&](int *n) {
                 *n = 3;
                 return launch_refine((RefUnit *)(D + o.refu), (int)P.refu.size(), P.ref_max_windows, c->ref_cands,
                                      c->ref_counters, c->ref_cum, c->ref_zpart, P.ref_max_items, c->g, st);
             })))
            return rc;
    }
    // 6. a5 trigger generator
    if ((rc = run_stage(c, SB_STAGE_TRIGGER, [&](int *n) {
             *n = (P.win.empty() ? 0 : 1) + (P.wfin.empty() ? 0 : 1);
             cudaError_t e = launch_window_max((WinTask *)(D + o.win), (int)P.win.size(), P.win_warps, to, st);
             if (e != cudaSuccess) return e;
             return launch_win_finalize((WinFinTask *)(D + o.wfin), (int)P.wfin.size(), P.wfin_warps, to, st);
         })))
        return rc;
    // 7. SNR history for the interpolators of the next push
    if ((rc = run_stage(c, SB_STAGE_SNRHIST, [&](int *n) {
             *n = (P.ycopy.empty() ? 0 : 1) + (P.yshift1.empty() ? 0 : 1) + (P.yshift2.empty() ? 0 : 1);
             cudaError_t e = launch_copy((CopyTask *)(D + o.ycopy), (int)P.ycopy.size(), P.max_rows, P.max_hy, st);
             if (e != cudaSuccess) return e;
             e = launch_copy16((CopyTask *)(D + o.ys1), (int)P.yshift1.size(), P.max_rows, st);
             if (e != cudaSuccess) return e;
             return launch_copy16((CopyTask *)(D + o.ys2), (int)P.yshift2.size(), P.max_rows, st);
         })))
        return rc;
    return SB_OK;
}

}  // namespace

extern "C" int filter_push_group(sb_ctx *c, int32_t n_units, sb_unit *const *units, const float *const *strains,
                                 int64_t B, const int64_t *t0, int32_t on_device) {
    if (!c || n_units <= 0 || !units || !strains || !t0) return fail(SB_EINVAL, "null or empty argument");
    if (B <= 0) return fail(SB_EINVAL, "n_samples must be positive");
    for (int i = 0; i < n_units; ++i) {
        sb_unit *u = units[i];
        if (!u || u->ctx != c) return fail(SB_EINVAL, "unit does not belong to this context");
        if (!strains[i]) return fail(SB_EINVAL, "null strain pointer");
        if (t0[i] != u->T)
            return fail(SB_EGAP, "unit " + std::to_string(u->id) + ": t0 " + std::to_string(t0[i]) +
                                     " is not contiguous with samples pushed so far (" + std::to_string(u->T) + ")");
        if (B % (1LL << u->kmax)) return fail(SB_EINVAL, "n_samples must be a multiple of 2^k_max");
        if (B > u->Bmax) return fail(SB_EINVAL, "n_samples exceeds max_push_samples");
        for (int j = 0; j < i; ++j)
            if (units[j] == u) return fail(SB_EINVAL, "a unit appears twice in one group");
    }
    if (activate(c) != SB_OK) return SB_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = c->stream;
    int kall = 0;
    for (int i = 0; i < n_units; ++i) kall = std::max(kall, units[i]->kmax);

    PushPlan P(n_units, kall);
    for (int i = 0; i < n_units; ++i) {
        sb_unit *u = units[i];
        P.max_rows = std::max(P.max_rows, 2 * u->M);
        const RefineWindows rw = refine_windows(P, u, B);
        plan_streams(P, i, u, B);
        if (u->tc) plan_tc(P, u, B, rw);
        else plan_fp32(P, u, B);
        plan_triggers(P, u, B, rw);
    }
    assign_tiles(P);
    int rc = prepare_refine_scratch(c, P, st);
    if (rc) return rc;

    // pack task lists (and host strain) into one pinned block
    Packer pk;
    PushOffsets o = pack_tasks(pk, P);
    std::vector<size_t> o_strain(n_units, 0);
    if (!on_device)
        for (int i = 0; i < n_units; ++i) o_strain[i] = pk.add(strains[i], B * sizeof(float));
    // the new top-rate strain of every unit is copied by one task-driven kernel (its source
    // pointers are data in the task block, not launch arguments)
    o.scopy = pk.reserve(n_units * sizeof(CopyTask));


    TaskArena *ar = nullptr;
    rc = arena_acquire(c, pk.buf.size(), ar);
    if (rc) return rc;
    char *D = ar->d;
    {
        CopyTask *sc = reinterpret_cast<CopyTask *>(pk.buf.data() + o.scopy);
        for (int i = 0; i < n_units; ++i) {
            LevelDev &L0 = units[i]->levels[0];
            CopyTask t{};
            t.cur = on_device ? strains[i] : reinterpret_cast<const float *>(D + o_strain[i]);
            t.dst = L0.dbuf[1 - L0.dcur] + L0.Hd;
            t.rows = 1;
            t.n = (int32_t)B;
            sc[i] = t;
        }
    }
    TriggerSlot *slot = nullptr;
    int slot_idx = 0;
    if ((rc = slot_acquire(c, P.trig_need, slot, slot_idx))) return rc;
    std::memcpy(ar->h, pk.buf.data(), pk.buf.size());

    // graph mode: everything from the task upload to the trigger read-back is one captured graph
    // a push that times a new mixing launch shape runs uncaptured (the tuner synchronises)
    bool tune_now = false;
    if (c->autotune)
        for (int h = 0; h < kNM; ++h)
            for (int k = 0; k <= P.kall; ++k)
                if (!P.tmix[h][k].empty() &&
                    !c->tuner.find(tc_mixup_shape_key(h, P.tmix_ml[h][k], P.tmix_tiles[h][k])))
                    tune_now = true;
    const bool capture = c->graphs && !c->prof && !tune_now;
    std::string gkey;
    CaptureGuard guard;
    if (capture) {
        gkey = std::to_string(B) + (on_device ? "d" : "h") + std::to_string(slot_idx) + ":" +
               std::to_string(c->next_arena);
        for (int i = 0; i < n_units; ++i) gkey += "," + std::to_string(units[i]->id);
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        guard.st = st;
        guard.active = true;
    }
    CK(cudaMemcpyAsync(ar->d, ar->h, pk.buf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(slot->dcount, 0, 3 * sizeof(int32_t), st));
    int *derr = slot->dcount + 2;
    const TrigOut to{slot->dbuf, slot->dcount, (int32_t)slot->cap};
    if ((rc = launch_stages(c, P, o, D, derr, to, n_units, B, tune_now, st))) return rc;
    // 8. triggers to the host (count plus an eager prefix; the rest on demand)
    CK(cudaMemcpyAsync(slot->hcount, slot->dcount, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(slot->hbuf, slot->dbuf, slot->eager * sizeof(DevTrigger), cudaMemcpyDeviceToHost, st));
    if (capture) {
        guard.active = false;
        if ((rc = end_capture_and_launch(c, gkey, st))) return rc;
    }
    CK(cudaEventRecord(slot->ev, st));
    slot->pending = true;
    c->pending.push_back(slot_idx);
    CK(cudaEventRecord(ar->ev, st));
    ar->used = true;
    c->stats.pushes += 1;
    c->stats.h2d_bytes += (int64_t)pk.buf.size();
    c->stats.d2h_bytes += 3 * sizeof(int32_t) + slot->eager * (int64_t)sizeof(DevTrigger);

    // 9. advance host bookkeeping
    for (int i = 0; i < n_units; ++i) {
        sb_unit *u = units[i];
        for (int k = 0; k <= u->kmax; ++k) {
            LevelDev &L = u->levels[k];
            L.dcur = 1 - L.dcur;
            L.last_Bk = B >> k;
            if (k >= 1 && L.Hy > 0 && !u->tc) L.ycur = 1 - L.ycur;
        }
        const int64_t first_n = u->T - u->levels[0].lam;
        if (first_n + B > std::max<int64_t>(first_n, 0)) u->wcur = 1 - u->wcur;
        u->T += B;
        u->last_B = B;
        u->amax_cur = 1 - u->amax_cur;
    }
    return SB_OK;
}

extern "C" int filter_push(sb_unit *u, const float *strain, int64_t n, int64_t t0, int32_t on_device) {
    if (!u) return fail(SB_EINVAL, "unit is null");
    sb_unit *const us[1] = {u};
    const float *const ss[1] = {strain};
    const int64_t ts[1] = {t0};
    return filter_push_group(u->ctx, 1, us, ss, n, ts, on_device);
}

extern "C" int sb_unit_snr(sb_unit *u, float *host_out, int64_t cap, int64_t *first_sample, int64_t *n) {
    if (!u || !first_sample || !n) return fail(SB_EINVAL, "null argument");
    if (!(u->flags & SB_FLAG_KEEP_SNR)) return fail(SB_EINVAL, "unit was created without SB_FLAG_KEEP_SNR");
    sb_ctx *c = u->ctx;
    if (activate(c) != SB_OK) return SB_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    const int64_t B = u->last_B;
    const int64_t first = u->T - B - u->levels[0].lam;
    const int64_t p0 = first < 0 ? std::min<int64_t>(-first, B) : 0;
    const int64_t nv = B - p0;
    *first_sample = first + p0;
    *n = nv;
    const int64_t M2 = 2 * (int64_t)u->M;
    if (nv <= 0) return SB_OK;
    if (!host_out || cap < M2 * nv) return fail(SB_EINVAL, "host buffer too small");
    LevelDev &L0 = u->levels[0];
    CK(cudaMemcpy2D(host_out, nv * sizeof(float), L0.ynew + p0, L0.ldy * sizeof(float), nv * sizeof(float), M2,
                    cudaMemcpyDeviceToHost));
    return SB_OK;
}

extern "C" const char *sb_last_error(void) { return g_err.c_str(); }

void set_last_error(const std::string &msg) { g_err = msg; }
