// Internal structures shared by the host runtime (lloid_api.cu) and the kernels.
// Every kernel consumes a device-resident list of tasks, so one launch covers
// every unit (SVD bank x detector) of a grouped push (Sec. II.B: same-rate
// slices of several banks are filtered together).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lloid {

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
    int32_t pad;
    int64_t first_n;     // absolute index of output p = 0 (negative -> write 0)
};

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
    int64_t n;
};

struct DevTrigger {      // layout-identical to sb_trigger
    int64_t unit, template_id, sample, window;
    float snr, phase;
    int32_t flags, reserved;
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
};

struct TrigOut {
    DevTrigger *buf;
    int32_t *count;      // [0] = triggers written, [1] = overflow flag
    int32_t cap;
};

// ---- launchers (kernels_simt.cu) -------------------------------------------
cudaError_t launch_decimate(const DecimTask *d_tasks, int n_tasks, int max_out, const Halfband &g,
                            cudaStream_t s);
cudaError_t launch_upsample(const UpTask *d_tasks, int n_tasks, int max_rows, int max_out,
                            const Halfband &g, cudaStream_t s);
cudaError_t launch_copy(const CopyTask *d_tasks, int n_tasks, int max_rows, int max_n, cudaStream_t s);
cudaError_t launch_gemm_fp32(const GemmTask *d_tasks, int n_tasks, int total_tiles, cudaStream_t s);
cudaError_t launch_window_max(const WinTask *d_tasks, int n_tasks, int total_warps, TrigOut out,
                              cudaStream_t s);

constexpr int kGemmTM = 64, kGemmTN = 128, kGemmTK = 16;

}  // namespace lloid
