// Internal structures shared by the host runtime (lloid_api.cu) and the kernels.
// Every kernel consumes a device-resident list of tasks, so one launch covers
// every unit (SVD bank x detector) of a grouped push (Sec. II.B: same-rate
// slices of several banks are filtered together).
#pragma once
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

namespace lloid {

// Programmatic dependent launch: every kernel of a push is launched with
// programmatic stream serialization, so its CTAs may start (and run their
// prologue) while the previous kernel's last CTAs finish; each kernel calls
// griddep_wait() before it touches memory that earlier work in the stream
// produces or still reads.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int kHalfK = 16;              // halfband kernel spans |j| <= 2K (65 taps)
constexpr int kOddTaps = kHalfK;        // g[2t+1], t = 0..K-1 (even taps are 0, g[0] = 1/2)

// Odd halfband taps g[1], g[3], ..., g[2K-1] (the kernel is symmetric).
struct Halfband {
    float odd[kOddTaps];
};

// ---- resampling -----------------------------------------------------------
// Decimation by two (step a1): out[p] = 0.5*in[b + 2p] + sum_t g[2t+1] (in[b+2p-2t-1] + in[b+2p+2t+1]).
// Outputs whose absolute index (first_m + p) is negative are written as 0.
struct DecimTask {
    const float *in;
    float *out;
    int64_t in_base;     // b: input position of output p = 0's centre tap
    int64_t first_m;     // absolute index of output p = 0
    int32_t n_out;
    int32_t pad;
};

// Interpolation by two plus history (step a4, the up-sampling half):
// out[a][p] = sum_m 2 g[n - 2m] y[a][m] with n = first_n + p, reading y through
// the virtual row [hist (Hy columns) | cur (n_in columns)].
// y position of absolute index m is  (nrel - j)/2 + in_off  with nrel = p - lam_out.
struct UpTask {
    const float *hist;   // [rows x ld_hist]
    const float *cur;    // [rows x ld_cur]
    float *out;          // [rows x ld_out]
    int64_t ld_hist, ld_cur, ld_out;
    int32_t n_hist;      // Hy of the input level
    int32_t rows;
    int32_t n_out;       // new samples at the output level
    int32_t lam_out;     // Lambda of the output level
    int32_t in_off;      // Lambda_in + Hy_in
    int32_t n_cur;       // valid columns of cur
    int64_t first_n;     // absolute index of output p = 0 (negative -> write 0)
};
constexpr int kUpChunk = 2048;   // outputs per shared-memory pass of the interpolation kernel
constexpr int kUpGroup = 4;      // passes per CTA

// Generic strided copy (history shifts): dst[r][i] = src_virtual[r][off + i],
// src_virtual = [hist (n_hist cols) | cur].
struct CopyTask {
    const float *hist;
    const float *cur;
    float *dst;
    int64_t ld_hist, ld_cur, ld_dst;
    int32_t n_hist;
    int32_t rows;
    int32_t n;           // columns to copy
    int32_t off;         // first virtual column
    int32_t elem16;      // 0: FP32 elements; p > 0: 16-bit elements in p planes (rows r + i rows, i < p)
    int32_t pad;
};

// ---- GEMM-shaped steps (a2 basis FIR as a Toeplitz GEMM, a3 mixing GEMM) --
// C[M x N] (+)= A[M x K] * B[K x N];  A row-major (lda);
// dense B:    B[k][n] = B[k*ldb + n]
// Toeplitz B: B[k][n] = x[ldb + n - k]   (x = decimated strain, ldb = base position)
struct GemmTask {
    const float *A;
    const float *B;
    float *C;
    int64_t lda, ldb, ldc;
    int32_t M, N, K;
    int32_t beta;        // 1: accumulate into C, 0: overwrite
    int32_t toeplitz;
    int32_t tiles_n;
    int32_t tile_begin;  // first global tile index of this task
    int32_t pad;
};

// ---- trigger generator (step a5) -------------------------------------------
struct WinState {        // running maximum of one template in its open window
    float mag2;          // |rho|^2 (-1: empty)
    float re, im;
    float pk, dt;        // sub-sample peak |rho| and offset (valid with SB_TRIG_SUBSAMPLE_BIT)
    float xi2;           // signal consistency (valid with SB_TRIG_XI2_BIT)
    int32_t flags;       // SB_TRIG_* bits of the maximum
    int64_t n;
};
constexpr int32_t SB_TRIG_REFINED_BIT = 1;
constexpr int32_t SB_TRIG_SUBSAMPLE_BIT = 2;
constexpr int32_t SB_TRIG_XI2_BIT = 4;
constexpr int kXiJ = 16;                 // xi^2 lags -kXiJ .. kXiJ (SB_XI2_HALF)
constexpr int kXiLags = 2 * kXiJ + 1;

// Sub-sample peak: vertex of the parabola through |rho|^2 = ym, y0, yp at
// n - 1, n, n + 1 when n is a local maximum: offset dt in [-1/2, 1/2] and |rho|.
__host__ __device__ __forceinline__ bool subsample_peak(float ym, float y0, float yp, float &pk, float &dt) {
    const float den = ym - 2.0f * y0 + yp;
    if (!(y0 >= ym && y0 >= yp && den < 0.0f)) return false;
    dt = 0.5f * (ym - yp) / den;
    pk = sqrtf(y0 - 0.25f * (ym - yp) * dt);
    return true;
}

struct DevTrigger {      // layout-identical to sb_trigger
    int64_t unit, template_id, sample, window;
    float snr, phase, snr_peak, dt_peak;
    int32_t flags;
    float xi2;
};

struct WinTask {
    const float *x;      // [2M x ldx], column p = absolute sample first_n + p
    int64_t ldx;
    const WinState *state_in;
    WinState *state_out;
    const int64_t *template_ids;
    int64_t first_n;     // absolute sample of column 0 (may be negative)
    int64_t unit_id;
    int64_t win_len;     // W f0
    int32_t n;           // columns
    int32_t M;
    int32_t n_seg;       // window segments covered by [max(0, first_n), first_n + n)
    int32_t warp_begin;  // first global warp of this task
    float threshold;
    int32_t pad;
    const float2 *acorr; // [M][kXiLags] template autocorrelation R_i[j] at j + kXiJ; null: no xi^2
};

struct TrigOut {
    DevTrigger *buf;
    int32_t *count;      // [0] = triggers written, [1] = overflow flag
    int32_t cap;
};

// ---- tensor-core path (kernels_tc.cu) ---------------------------------------
constexpr int kTcM = 128;   // MMA M (rows of the A operand per tile)
constexpr int kModeF16 = 0, kModeBF16 = 1, kModeE4M3 = 2;   // tensor-core operand modes
constexpr int kTcN = 256;   // MMA N (columns of the accumulator per tile)
// Planes of the stored per-level SNR y_k (levels k >= 1) in the tensor-core modes, by the mixing
// kernel's operand mode: BF16 keeps y as one FP16 plane (11-bit significand; |y| is an SNR partial,
// far inside FP16's range); FP16 keeps BF16 hi + lo planes (about 16 significant bits) for its
// smaller error.  (The E4M3 precision runs its mixing in BF16: see mix_mode.)
__host__ __device__ constexpr int y_planes(int mode) { return mode == kModeF16 ? 2 : 1; }
// Operand mode of the mixing + interpolation kernel for a unit whose basis FIR runs in `mode`.
// SB_FP8 takes E4M3 for the basis FIR only (weights one E4M3 term with a per-basis-vector scale,
// strain two E4M3 terms with a per-buffer scale) and writes its basis outputs in BF16: one
// single-term E4M3 operand adds about 0.027 of |SNR| (rms) in white noise, and a second one
// (the mixing weights) would put the largest window-maximum errors above 0.15.
__host__ __device__ constexpr int mix_mode(int mode) { return mode == kModeE4M3 ? kModeBF16 : mode; }

struct HalfConvTask {       // dst[i] = narrow(src[i]), i < n (E4M3: scaled by 448 / absmax)
    const float *src;
    void *dst;
    int64_t n;
    float *amax;               // E4M3: this push's |src| maximum (accumulated by the cascade kernel)
    float *amax_next;          // E4M3: the next push's accumulator, zeroed here
    void *dst_lo;              // E4M3: second term, dst_lo[i] = narrow(s src[i] - dst[i]); null otherwise
};

// a2 on tensor cores.  Tile (mt, nt): W rows [128 mt, 128 mt + 128) (16 basis
// vectors x 8 phases, row 16 r + l_loc), blocks b in [256 nt, 256 nt + 256).
struct TcFirTask {
    const CUtensorMap *mapW;   // W [8 L16 rows x Kpad] 16-bit, K-major, 128-byte swizzle
    const void *x;             // decimated strain, 16-bit
    int64_t X0;                // x index of (b = 0, j = 0); multiple of 8
    void *O;                   // basis outputs, 16-bit, [m][ldo]
    int64_t ldo;
    int32_t o_col;             // column of this slice's first basis vector in O
    int32_t Kpad;              // multiple of 64
    int32_t Bk;                // outputs m' < Bk are written
    int32_t tiles_m;           // padded basis vectors / basis vectors per tile
    int32_t tiles_n;
    int32_t tile_begin;
    const float *xamax;        // E4M3: |strain| maximum of this push at this level
    const float *colscale;     // E4M3: per output column, the basis vector's scale
    const void *x_lo;          // E4M3: second term of the strain (same layout as x); O is BF16
};

// Partial window maximum of one template over one column run of one tile.
struct __align__(16) WinPart {
    float mag2;                // |rho|^2 (-1: no valid sample)
    float re, im;
    float pk, dt;              // sub-sample peak (refined records with SB_TRIG_SUBSAMPLE_BIT)
    float xi2;                 // signal consistency (refined records with SB_TRIG_XI2_BIT)
    int32_t flags;             // SB_TRIG_* bits (refined, sub-sample, xi^2)
    int32_t nr;                // top-rate sample relative to column 0 of the record set (records live
                               // for one push; the carried window state keeps absolute samples)
};
static_assert(sizeof(WinPart) == 32 && alignof(WinPart) == 16, "window records: two 16-byte accesses each");

// a3 + a4 on tensor cores (+ a5 partial maxima at the top level).
// Tile (tt, at): time columns [256 tt, +256) of this level, filters [128 at, +128).
struct TcMixUpTask {
    const CUtensorMap *mapM;   // A: mixing [2M x Lk_pad] 16-bit, box 64 x 128 (unused when Lk_pad = 0)
    const CUtensorMap *mapO;   // B: basis outputs [rows x Lk_pad] 16-bit, box 64 x 256
    const CUtensorMap *mapY;   // coarser level y_{k+1}: FP16 rows [0, 2M) (BF16 / E4M3 modes) or BF16 hi
                               // rows [0, 2M) and lo rows [2M, 4M) (FP16 mode); box 64 x 128, 128-byte
                               // swizzle; null at the deepest level
    float *Y;                  // top level with SB_FLAG_KEEP_SNR: FP32 SNR (row a at Y + a ldy); else null
    int64_t ldy;
    uint16_t *Yh;              // this level's y in the layout of mapY (ld ldu); null at the top
    int64_t ldu;
    int64_t yst_col0;          // column of this push's first sample in Yh
    WinPart *part;             // top level: partials [i][n_rec], record (tt*2 + half)*2 + seg; null below
    int64_t first_n;           // absolute index (this level's rate) of column 0
    int64_t win_len;           // top level: window length in samples (>= 128)
    int32_t Lk_pad, M2, M, Bk;
    int32_t kbytes;            // bytes of K per mixing-operand row in one chunk: 32, 64 or 128 (the swizzle span)
    int32_t lam;               // Lambda of this level
    int32_t in_off;            // Lambda_{k+1} + Hy_{k+1}: coarser position of (relative index 0) / 2
    int32_t tiles_t, tiles_a, tile_begin, n_rec;
    uint32_t *wmax;            // top level with refinement: [M][n_wslot] 16-bit window maxima above thr2
    int64_t win0;              //   (mag2 bits, atomicMax), window of slot 0
    int32_t n_wslot;
    float thr2;                //   refine threshold squared
};

// Window bookkeeping after the top-level partial maxima: one warp per
// (unit, template, window touched by the push) reduces that window's records,
// merges the open window's state (first window), emits the trigger of a
// completed window and stores the state of the one left open (last window).
struct WinFinTask {
    const WinPart *part;       // [M][n_rec]; record r covers push columns [128 (r/2), +128), seg r%2
    const WinState *state_in;
    WinState *state_out;
    const int64_t *template_ids;
    int64_t unit_id;
    int64_t win_len;
    int64_t first_n;           // absolute sample of push column 0
    int64_t start_abs, end_abs; // valid absolute samples of this push: [start_abs, end_abs)
    int32_t n_rec, M, n_win;
    int32_t warp_begin;
    float threshold;
    int32_t n_wslot;           // with wmax: window slots of this push (window start_abs / win_len + s)
    const uint32_t *wmax;      // null, or [M][n_wslot] maxima of the records above a threshold below
                               // `threshold` (16-bit |rho|^2 bits): a completed window in the middle of
                               // the push with a zero maximum cannot trigger and is skipped
};

size_t tc_fir_smem_bytes(int kpad_max, int mode);
// Launch description of one tc_mixup launch, from its tasks: the most K chunks of a tile, whether
// any task stores its y (levels below the top) or interpolates a coarser level, and the widest
// mixing-operand row (bytes of K per chunk: 32, 64 or 128), which sets the stage size.
struct MixLaunch {
    int max_nk = 0;
    bool store_y = false;
    bool interp = false;
    int kbytes = 32;
};
size_t tc_mixup_stage_bytes(int kbytes);
size_t tc_mixup_smem_bytes(int n_st, int n_win, int n_u, int n_stbuf, int ublk, int np, int kbytes);
// wait_ns: bound of the kernel's waits (0: the default, 2 s); skip_chunk >= 0: test hook (the first
// tile's producer skips that K chunk's load, so its consumer's wait runs out).
cudaError_t launch_tc_fir(const TcFirTask *d_tasks, int n_tasks, int total_tiles, int kpad_max, int mode, int *err,
                          cudaStream_t s, uint64_t wait_ns = 0, int skip_chunk = -1);
// Pipeline shape of one tc_mixup launch: mixing stages, interpolation-operand buffers and the
// depth of the window ring.  None of them changes the arithmetic, so results do not depend on
// the choice; the autotuner times the candidates that fit in shared memory once per launch
// shape (mode, MixLaunch, tile count) and keeps the fastest.
struct MixCfg {
    int n_st, n_u, n_win;
};
struct MixTuner {
    std::vector<std::pair<uint32_t, MixCfg>> best;    // launch shape -> fastest pipeline shape
    int64_t timed_launches = 0;
    const MixCfg *find(uint32_t key) const {
        for (auto &kv : best)
            if (kv.first == key) return &kv.second;
        return nullptr;
    }
};
uint32_t tc_mixup_shape_key(int mode, const MixLaunch &ml, int total_tiles);
// utab: the interpolation operand table (tc_interp_table_bytes(), built by tc_interp_table).
// tuner: null, or the context's tuner; may_tune: the shape may be timed now (no capture running).
cudaError_t launch_tc_mixup(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, const MixLaunch &ml,
                            const void *utab, int mode, int *err, MixTuner *tuner, bool may_tune, cudaStream_t s);
size_t tc_interp_table_bytes();
void tc_interp_table(const Halfband &g, void *host_out);
cudaError_t launch_win_finalize(const WinFinTask *d_tasks, int n_tasks, int total_warps, TrigOut out,
                                cudaStream_t s);

// ---- FP32 refinement of candidate maxima (kernels_refine.cu) ----------------
constexpr int kRefTile = 256;            // top-level samples per record tile (= mixing tile)
constexpr int kRefR = 8;                 // refined samples on either side of a candidate maximum
constexpr int kRefMaxLevels = 8;
constexpr int kRefMaxSlices = 12;
constexpr int kRefSpan = 64;             // level-k samples one candidate needs (<= 62 for R = 8 and 16 xi^2 lags)
constexpr int kRefCandCap = 1 << 16;     // candidates one push refines at most
constexpr int kRefSplitCap = 4096;       // candidates whose FIR chunks run as separate blocks (the rest inline)
constexpr int kRefQC = 2048;             // filter taps of one FIR work item

struct RefUnit {                         // one unit of a push with refinement on
    WinPart *part;                       // [M][n_rec] top-level partial maxima (refined in place)
    int64_t first_n;                     // absolute top-level index of push column 0
    int64_t win_len;
    float thr2;                          // refine threshold squared
    float keep2;                         // a record is refined when mag2 >= keep2 x its window's 16-bit maximum
    uint32_t *wmax;                      // [M][n_wslot] 16-bit window maxima of this push (mag2 bits)
    int64_t win0;                        // window of slot 0
    int32_t n_wslot;
    int32_t kmax, M, n_rec, B, n_slices;
    const float *lv_d[kRefMaxLevels];    // FP32 decimated strain of this push, position 0 = absolute lv_origin
    int64_t lv_origin[kRefMaxLevels], lv_len[kRefMaxLevels];
    const float *sl_H[kRefMaxSlices];    // FP32 reconstructed slice filters [2M][ldh] (mixing x basis)
    int64_t sl_D[kRefMaxSlices];
    int32_t sl_Q[kRefMaxSlices], sl_ldh[kRefMaxSlices], sl_level[kRefMaxSlices];
    int32_t sl_item0[kRefMaxSlices + 1];  // FIR work items (kRefQC-tap chunks) of slice s: [sl_item0[s], sl_item0[s + 1])
    const float2 *acorr;                 // [M][kXiLags] template autocorrelation; null: no xi^2
};
struct RefCand {                         // one partial record to refine
    int32_t unit;
    int64_t idx;                         // i * n_rec + record
};
// cands: kRefCandCap entries; counters[1] = candidates found, counters[2] = 1 when some were dropped
// cum: running totals [candidates, pushes with dropped candidates] (device, never reset)
// max_windows: the largest M x n_wslot of the units (one candidate-scan thread per template and window)
// zpart: kRefSplitCap x max_items x 2 x kRefSpan floats of FIR scratch; max_items: the largest
// sl_item0[n_slices] of the units
cudaError_t launch_refine(const RefUnit *d_units, int n_units, int64_t max_windows, RefCand *cands, int *counters,
                          unsigned long long *cum, float *zpart, int max_items, const Halfband &g, cudaStream_t s);
// Margin of the candidate rule per operand mode: records within (1 - margin) of their window's
// 16-bit maximum are refined (the 16-bit error stays well inside it).
constexpr float kRefKeep16 = 0.81f;      // (1 - 0.1)^2, BF16 / FP16
constexpr float kRefKeep8 = 0.64f;       // (1 - 0.2)^2, E4M3 (errors <= 0.15 near |rho| = 5.5)

// ---- a1 cascade and 16-bit copies in one launch (kernels_cascade.cu) --------
// One unit per cluster of kCascadeCtas CTAs.  Levels run in order: the 16-bit copy of level k
// (tensor-core units) and the decimation k -> k + 1 both read level k, then a cluster barrier makes
// level k + 1 visible to every CTA of the cluster before the next step.
constexpr int kCascadeCtas = 8;
struct CascadeTask {
    DecimTask lev[kRefMaxLevels];        // level k -> k + 1, k < n_lev
    HalfConvTask conv[kRefMaxLevels];    // 16-bit operand copy of level k, k < n_conv
    int32_t n_lev, n_conv;
    int32_t mode;                        // operand mode of the copies (kModeF16, kModeBF16, kModeE4M3)
    int32_t pad;
};
cudaError_t launch_cascade(const CascadeTask *d_tasks, int n_tasks, const Halfband &g, cudaStream_t s);

// ---- launchers (kernels_simt.cu) -------------------------------------------
cudaError_t launch_upsample(const UpTask *d_tasks, int n_tasks, int max_rows, int max_out,
                            const Halfband &g, cudaStream_t s);
cudaError_t launch_copy(const CopyTask *d_tasks, int n_tasks, int max_rows, int max_n, cudaStream_t s);
// 16-bit tasks only (elem16 > 0): one warp per row
cudaError_t launch_copy16(const CopyTask *d_tasks, int n_tasks, int max_rows, cudaStream_t s);
cudaError_t launch_gemm_fp32(const GemmTask *d_tasks, int n_tasks, int total_tiles, cudaStream_t s);
cudaError_t launch_window_max(const WinTask *d_tasks, int n_tasks, int total_warps, TrigOut out,
                              cudaStream_t s);

constexpr int kGemmTM = 128, kGemmTN = 128, kGemmTK = 8;

}  // namespace lloid
