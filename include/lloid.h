/*
 * lloid.h - C ABI of the B300 multirate SVD matched filter (LLOID) and its
 * device-side trigger generator.
 *
 * The operation is the filtering stage of Sec. II.A of "Scalable
 * matched-filtering pipeline for gravitational-wave searches of compact binary
 * mergers" (arXiv:2410.16416): whitened strain is down-sampled to each time
 * slice's rate, cross-correlated with the slice's orthonormal SVD basis
 * filters, the orthogonal SNR series are multiplied by the SVD coefficients,
 * the per-slice SNR segments are up-sampled and summed, and per-window |SNR|
 * maxima above a threshold become triggers with their phase (Sec. II.A and the
 * Fig. 1 caption); the trigger generator runs on the device so that only the
 * reduced trigger set crosses to the host (Sec. II.B).  Several SVD banks are
 * filtered in one grouped launch per stage (Sec. II.B).
 *
 * Notation: f0 = top rate; n = absolute top-rate sample index (n >= 0, the
 * strain is zero before n = 0); M templates per bank, real filter a = 2i + p
 * (p = 0 cosine phase, p = 1 sine phase); slice s at rate f_s = f0 / 2^k_s
 * covers tau in [t_s, t_{s+1}) seconds before coalescence, has Q_s taps,
 * delay D_s = t_s f_s and L_s basis vectors.
 *
 * Conventions: status 0 = OK, negative = error (SB_E*); sb_last_error() gives
 * a message for the calling thread's last failure.  The caller owns every host
 * array it passes; the library copies what it needs before returning.  The
 * library owns all device memory it allocates.  Nothing here blocks on the GPU
 * except where stated.
 */
#ifndef LLOID_H
#define LLOID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SB_OK        0
#define SB_EINVAL   (-1)  /* bad argument or bank shape                       */
#define SB_ENOMEM   (-2)  /* a device or pinned allocation failed             */
#define SB_EBUSY    (-3)  /* admission refused: HBM budget of the context full */
#define SB_EGAP     (-4)  /* t0 not contiguous with the unit's previous push   */
#define SB_ETIMEOUT (-5)  /* a bounded device wait expired                    */
#define SB_ECUDA    (-6)  /* a CUDA runtime call failed (message has details)  */
#define SB_EOVERFLOW (-7) /* trigger buffer overflow (triggers were dropped)   */

/* ---- arithmetic of the two GEMM-shaped steps (basis FIR, reconstruction) */
#define SB_FP32 0   /* FP32 operands, FP32 accumulate (SIMT)                  */
#define SB_BF16 1   /* BF16 operands, FP32 accumulate (tensor cores)          */
#define SB_FP16 2   /* FP16 operands, FP32 accumulate (tensor cores)          */
#define SB_FP8  3   /* E4M3 operands with per-vector scales, FP32 accumulate  */

/* ---- sb_desc.flags --------------------------------------------------- */
#define SB_FLAG_KEEP_SNR 1  /* keep the last push's top-rate SNR readable (sb_unit_snr) */

/* ---- trigger flags --------------------------------------------------- */
#define SB_TRIG_REFINED 1   /* SNR recomputed in FP32 around the peak.  With
                             * refinement on (16/8-bit units, refine_threshold
                             * below threshold) every trigger carries it, except
                             * in a push whose candidates overflowed the 65,536
                             * list: its remaining triggers keep their 16-bit
                             * value and phase (sb_ctx_stats.refine_dropped
                             * counts such pushes).                              */
#define SB_TRIG_SUBSAMPLE 2 /* snr_peak / dt_peak hold the sub-sample peak       */
#define SB_TRIG_XI2 4       /* xi2 holds the signal-consistency value           */
#define SB_XI2_HALF 16      /* xi^2 lags j = -16 .. 16 top-rate samples         */

/* One time slice of an SVD bank (Sec. II.A "time slices ... SVD").
 * basis : [n_basis * n_taps] row-major; row l is v_l[q], q = 0 is the tap
 *         t_start_s seconds before coalescence, q grows back in time.
 * mixing: [2M * n_basis] row-major; row a = 2i + p holds the coefficients
 *         of real filter a on the basis vectors (h_{a,s} ~= sum_l M[a,l] v_l).
 * rate_hz must be top_rate_hz / 2^k (0 <= k <= 7); (t_end_s - t_start_s) * rate_hz
 * and t_start_s * rate_hz must be integers.                                   */
typedef struct sb_slice {
    double rate_hz;
    double t_start_s;
    double t_end_s;
    int32_t n_basis;
    int32_t n_taps;
    const double *basis;
    const double *mixing;
} sb_slice;

/* One SVD bank (one template group for one detector, Sec. IV: "one SVD bank
 * for each instrument").
 * template_ids: [n_templates] ids copied into triggers (NULL: 0..M-1).
 * threshold: a window maximum triggers when |rho| > threshold.
 * refine_threshold: in SB_BF16/SB_FP16/SB_FP8 modes, window maxima above this
 *   are recomputed in FP32 (0 disables refinement).
 * window_s: trigger window length (windows start at multiples of window_s*f0).
 * max_push_samples: the largest n_samples a filter_push will pass (top rate),
 *   at most 2^30.
 * autocorr: NULL, or [n_templates][2 SB_XI2_HALF + 1][2] (re, im) doubles, the
 *   normalised complex autocorrelation of each template at f0, lag j at index
 *   j + SB_XI2_HALF: R_i[j] = sum_q h_i[q] conj(h_i[q - j]) / sum_q |h_i[q]|^2
 *   with h_i = h_{2i} + i h_{2i+1}.  Given, every trigger whose lags n* - 16 ..
 *   n* + 16 are computed in FP32 in one pass carries the signal-consistency
 *   value of Sec. II.A (GstLAL's xi^2, a reading):
 *     xi2 = sum_j |rho[n* + j] - rho[n*] R_i[j]|^2 / sum_j (2 - 2 |R_i[j]|^2).
 *   Copied before return; |R_i[0] - 1| must be <= 1e-6 (SB_EINVAL otherwise). */
typedef struct sb_desc {
    int32_t n_templates;
    int32_t n_slices;
    double top_rate_hz;
    const sb_slice *slices;
    const int64_t *template_ids;
    int32_t precision;
    int32_t flags;
    float threshold;
    float refine_threshold;
    double window_s;
    int64_t max_push_samples;
    const double *autocorr;
} sb_desc;

/* One trigger: the |SNR| maximum of one template in one window (Sec. II.A: a
 * template, a time, an SNR and a phase).  sample = absolute top-rate index n*
 * of the maximum (first one on ties), window = n* / (window_s * f0),
 * snr = |rho(n*)|, phase = atan2(x_{2i+1}(n*), x_{2i}(n*)) in radians.
 * With SB_TRIG_SUBSAMPLE set, the
 * peak between samples (the future feature named in Sec. III for the SNR gap
 * to GstLAL) is the vertex of the parabola through |rho|^2 at sample - 1,
 * sample, sample + 1: |SNR| snr_peak at time sample + dt_peak (in samples,
 * |dt_peak| <= 1/2).  It is set where both neighbours are computed in FP32 in
 * the same pass (FP32 mode: inside one push; 16/8-bit modes: refined maxima)
 * and the sample is a local maximum; otherwise snr_peak = snr, dt_peak = 0.
 * With SB_TRIG_XI2 set (the bank carries sb_desc.autocorr and the lags
 * sample - 16 .. sample + 16 were computed in FP32 in the same pass), xi2 is
 * the signal-consistency value defined at sb_desc.autocorr.                   */
typedef struct sb_trigger {
    int64_t unit;
    int64_t template_id;
    int64_t sample;
    int64_t window;
    float snr;
    float phase;
    float snr_peak;
    float dt_peak;
    int32_t flags;
    float xi2;      /* signal consistency (SB_TRIG_XI2 set; 0 otherwise)        */
} sb_trigger;

/* Read-only facts about a unit (for tests, benchmarks and admission). */
typedef struct sb_unit_info {
    int64_t unit;             /* id used in triggers                           */
    int32_t n_templates;
    int32_t n_slices;
    int32_t k_max;            /* deepest level: lowest rate = f0 / 2^k_max      */
    int32_t precision;
    int64_t latency_samples;  /* top-rate look-ahead: after pushing T samples,  */
                              /* SNR is final for n < T - latency_samples       */
    int64_t samples_pushed;   /* T                                              */
    int64_t device_bytes;     /* device memory of this unit's own state (bank   */
                              /* data shared by several units is not included)  */
    int64_t flops_per_second; /* algorithmic FLOPs per second of data (FIR+mix) */
} sb_unit_info;

typedef struct sb_ctx sb_ctx;
typedef struct sb_unit sb_unit;

/* Context: one CUDA device, one stream, one HBM budget, one trigger queue.
 * device: CUDA ordinal; stream: a cudaStream_t to launch on (NULL: the
 * library creates its own); hbm_budget_bytes: device bytes the context may
 * hold for units (<= 0: 90% of free memory at creation). */
int sb_ctx_create(int32_t device, void *stream, int64_t hbm_budget_bytes, sb_ctx **out);
int sb_ctx_destroy(sb_ctx *ctx);
/* Block until all work queued on the context's stream has finished. */
int sb_ctx_sync(sb_ctx *ctx);

/* Create one (bank, detector) unit: validates the bank, copies the host
 * arrays, converts them to the working precision, allocates the unit's
 * device state (zeroed histories) and admits it against the budget.
 * Returns SB_EBUSY (nothing allocated) when the budget cannot hold it. */
int svdbank_create(sb_ctx *ctx, const sb_desc *desc, int32_t detector, sb_unit **out);
/* Release one unit (Sec. IV: one SVD bank per instrument, so one unit per
 * (bank, detector) pair).  The unit's device state is freed in stream order,
 * after every push already queued on the context's stream (the call does not
 * block), and its bytes return to the context's budget; bank data shared
 * through svdbank_create_like is freed with the last unit that uses it.
 * Triggers the unit already produced stay in the queue.  NULL is a no-op
 * (SB_OK); the pointer is invalid after the call. */
int svdbank_destroy(sb_unit *unit);

/* A new unit that filters with the same SVD bank as src (same precision,
 * thresholds, window and push size) but has its own streaming state: the
 * read-only bank data on the device (basis, mixing, their converted forms and
 * template ids) is shared and freed with the last unit that uses it.  This is
 * "the same SVD bank provided multiple times" of the paper's GPU benchmark
 * (Sec. IV), and the two detectors of one bin when their banks coincide.
 * Admission charges only the new unit's state (SB_EBUSY when it does not fit). */
int svdbank_create_like(sb_ctx *ctx, sb_unit *src, int32_t detector, sb_unit **out);
int sb_unit_query(const sb_unit *unit, sb_unit_info *info);

/* Validate a bank description and report the unit it would create (k_max,
 * latency, device bytes, FLOPs) without touching any device.  Fields of
 * *info that need a live unit (unit, samples_pushed) are set to 0. */
int svdbank_plan(const sb_desc *desc, sb_unit_info *info);

/* Push the next n_samples top-rate samples of whitened strain to one unit:
 * the filtering stage of Sec. II.A (down-sample, cross-correlate with the
 * orthogonal basis, multiply by the SVD coefficients, up-sample and sum), run
 * with the device-side trigger generator of Sec. II.B on its output.
 * strain: host pointer (on_device = 0) or device pointer (on_device = 1),
 * FP32, contiguous.  t0_sample must equal the unit's samples pushed so far
 * (SB_EGAP otherwise); n_samples must be a multiple of 2^k_max and at most
 * max_push_samples.  The host buffer may be reused when the call returns.
 * Work is queued on the context's stream; triggers of every window the push
 * completes become available to triggers_pop once that work has finished. */
int filter_push(sb_unit *unit, const float *strain, int64_t n_samples, int64_t t0_sample,
                int32_t on_device);

/* Push one buffer to each of n units at once: every stage runs as one grouped
 * launch over all units (Sec. II.B: same-rate slices of several banks are
 * stacked and filtered together).  All units must belong to ctx; strains[u],
 * t0_samples[u] as in filter_push; n_samples is common to all units. */
int filter_push_group(sb_ctx *ctx, int32_t n_units, sb_unit *const *units,
                      const float *const *strains, int64_t n_samples,
                      const int64_t *t0_samples, int32_t on_device);

/* Progress of the context's pushes (never blocks): *pushed = filter_push /
 * filter_push_group calls so far, *completed = how many of them (the oldest
 * ones) have finished on the device with their triggers moved to the host
 * queue that triggers_pop reads.  Push i (0-based, in call order) is complete
 * when *completed > i. */
int sb_ctx_progress(sb_ctx *ctx, int64_t *pushed, int64_t *completed);

/* Move up to cap finished triggers into out (never blocks on queued work):
 * the hand-off of the trigger generator that runs on the device (Sec. II.B),
 * so that only triggers, never SNR series, cross to the host.
 * *n_out = number written.  Triggers come out push by push, and within a push
 * sorted by (window, unit, template).  Returns SB_EOVERFLOW once if triggers
 * were dropped because a push produced more than its buffer holds. */
int triggers_pop(sb_ctx *ctx, sb_trigger *out, int64_t cap, int64_t *n_out);

/* Debug read-back (blocks): the top-rate SNR series x_a[n] of the unit's last
 * push, written row-major [2M][*n] into host_out (capacity cap floats), for
 * n in [*first_sample, *first_sample + *n).  Needs SB_FLAG_KEEP_SNR. */
int sb_unit_snr(sb_unit *unit, float *host_out, int64_t cap, int64_t *first_sample, int64_t *n);

/* ---- data conditioning: PSD estimate, whitening, gating ------------------ */
/* The conditioning stage that precedes the filter (Sec. II.A: the PSD is
 * estimated, its running average whitens the strain, large deviations of the
 * whitened data are gated and removed; Fig. 1: "whitening and gating").  The
 * paper names the steps only; this library's readings:
 *   whitening: segments of fft_len = N samples every H = N/2 samples
 *     (segment j covers input samples [jH, jH + N); the strain is 0 before
 *     sample 0), periodic Hann window w[n] = sin^2(pi n / N);
 *     X_j = DFT(w d_j), S_j = |X_j|^2 / sum w^2 per frequency bin;
 *     running average P_j = P_{j-1} + (S_j - P_{j-1}) / min(j + 1, n_avg);
 *     segment j is divided by sqrt(P_{j-1}) (segment 0 by sqrt(P_0)), inverse
 *     DFT, overlap-add.  White noise of variance s^2 comes out as d / s.
 *   gating: every whitened sample with |x| > gate_threshold is a glitch
 *     sample; samples within gate_half of one are set to 0 and the weight
 *     returns to 1 as sin^2(pi (r - gate_half) / (2 gate_taper)) for distances
 *     gate_half < r < gate_half + gate_taper.
 * FP32 on the device (FFT in shared memory).  One sb_cond per detector stream;
 * its work is queued on the context's stream, ordered with filter_push. */
typedef struct sb_cond_desc {
    double rate_hz;            /* sample rate of the strain (> 0; informational)   */
    int32_t fft_len;           /* N: a power of two in [64, 16384]                  */
    int32_t n_avg;             /* running-average length, >= 1                      */
    float gate_threshold;      /* glitch level of the whitened data; <= 0: no gate   */
    int32_t gate_half;         /* samples zeroed on each side of a glitch sample     */
    int32_t gate_taper;        /* samples of the ramp back to full weight, >= 1      */
    int64_t max_push_samples;  /* largest push, a multiple of N / 2, at most 2^30    */
} sb_cond_desc;
typedef struct sb_cond sb_cond;
/* Allocates the conditioner's device state (zeroed: the strain is 0 before
 * the first push) on the context's device.  SB_EINVAL for a bad description,
 * SB_ENOMEM when an allocation fails.  Destroy conditioners before their
 * context. */
int sb_cond_create(sb_ctx *ctx, const sb_cond_desc *desc, sb_cond **out);
/* Waits for the context's queued work and frees the device state (NULL: no-op). */
int sb_cond_destroy(sb_cond *cond);
/* latency = N/2 + gate_half + gate_taper: the look-ahead of the overlap-add
 * and the gate.  Output sample i of the conditioned stream is the conditioned
 * strain at input sample i - latency (0 for i < latency). */
int sb_cond_latency(const sb_cond *cond, int64_t *latency_samples);
/* Push the next n_samples input samples (a positive multiple of N/2, at most
 * max_push_samples; t0_sample must equal the samples pushed so far, SB_EGAP
 * otherwise).  strain: FP32, host (on_device = 0, copied before the call
 * returns) or device (on_device = 1).  out: device FP32 [n_samples], written by
 * the queued work with output samples [t0_sample, t0_sample + n_samples) of
 * the conditioned stream, so that a filter_push of out with the same t0 on the
 * same context follows it in stream order.  Non-blocking. */
int sb_cond_push(sb_cond *cond, const float *strain, int64_t n_samples, int64_t t0_sample, int32_t on_device,
                 float *out);
/* The running PSD average after the segments processed so far (blocks):
 * *n_bins = N/2 + 1 values P[f] (per-bin variance, bin f at f rate_hz / N Hz;
 * the one-sided PSD is 2 P[f] / rate_hz) into host_out (cap >= *n_bins, or
 * cap = 0 to query the sizes only), *segments = segments averaged. */
int sb_cond_psd(sb_cond *cond, float *host_out, int64_t cap, int64_t *n_bins, int64_t *segments);

/* ---- coincidence generator (host only) ----------------------------------- */
/* One coincidence: triggers index_a of detector A and index_b of detector B
 * (indices into the arrays passed in), same template, |sample_a - sample_b|
 * <= max_dt_samples; network_snr = sqrt(snr_a^2 + snr_b^2).                 */
typedef struct sb_coinc {
    int64_t template_id;
    int64_t index_a, index_b;
    int64_t sample_a, sample_b;
    float snr_a, snr_b, network_snr;
    int32_t reserved;
} sb_coinc;
/* The coincidence generator that follows the filter (Sec. II.A): every pair of
 * a trigger of detector A and one of detector B with the same template_id and
 * |sample_a - sample_b| <= max_dt_samples (top-rate samples: the light-travel
 * time between the two sites, about 10 ms for the LIGO pair, plus any timing
 * margin, times f0).  Inputs in any order (as triggers_pop returns them); the
 * pairs are written to out ordered by (template_id, sample_a, sample_b,
 * index_a, index_b).  *n_out = the number of coincidences.  Host memory only,
 * no device.  Returns SB_OK, SB_EINVAL (null pointers with nonzero counts,
 * negative max_dt_samples or cap), or SB_EOVERFLOW when more than cap pairs
 * exist (the first cap are written). */
int sb_coincidences(const sb_trigger *a, int64_t n_a, const sb_trigger *b, int64_t n_b, int64_t max_dt_samples,
                    sb_coinc *out, int64_t cap, int64_t *n_out);

/* ---- instrumentation ------------------------------------------------- */
/* Stages of a push, in launch order (indices of sb_ctx_stage_times). */
#define SB_STAGE_HISTORY   0  /* history shifts of the decimated strain          */
#define SB_STAGE_STRAIN    1  /* new strain into the top-rate buffer             */
#define SB_STAGE_DECIMATE  2  /* a1: halfband decimation cascade                 */
#define SB_STAGE_FIR       3  /* a2: basis FIR (Toeplitz GEMM)                   */
#define SB_STAGE_UPSAMPLE  4  /* a4: interpolation by two                        */
#define SB_STAGE_MIX       5  /* a3: reconstruction (mixing) GEMM                */
#define SB_STAGE_TRIGGER   6  /* a5: window maxima, threshold, phase             */
#define SB_STAGE_SNRHIST   7  /* SNR history for the next push's interpolators   */
#define SB_STAGE_REFINE    8  /* a6: FP32 recomputation of candidate maxima       */
#define SB_N_STAGES        9

/* Cumulative counters of a context since creation. */
typedef struct sb_ctx_stats {
    int64_t pushes;          /* filter_push / filter_push_group calls          */
    int64_t kernel_launches; /* this library's kernels launched                */
    int64_t h2d_bytes;       /* host -> device bytes copied by pushes          */
    int64_t d2h_bytes;       /* device -> host bytes copied for triggers       */
    int64_t triggers;        /* triggers delivered by triggers_pop             */
    int64_t refine_candidates;  /* partial window maxima recomputed in FP32 (a6)  */
    int64_t refine_dropped;     /* pushes whose candidates exceeded the list (65536); the rest kept 16-bit values */
    int64_t graph_launches;     /* pushes launched as one CUDA graph (sb_ctx_graphs)  */
    int64_t autotune_shapes;    /* mixing-kernel launch shapes timed by the autotuner  */
    int64_t autotune_launches;  /* mixing-kernel launches spent timing candidates        */
} sb_ctx_stats;
int sb_ctx_get_stats(sb_ctx *ctx, sb_ctx_stats *out);

/* enable != 0: bracket every kernel launch with CUDA events on the context's
 * stream; enable == 0: stop.  Enabling clears previously collected times. */
int sb_ctx_profile(sb_ctx *ctx, int32_t enable);
/* enable != 0: every push (filter_push / filter_push_group) is stream-captured
 * into a CUDA graph and launched as one graph; pushes with the same group
 * (same units in the same order, same n_samples, host or device strain) reuse
 * one executable graph, updated in place with the push's arguments
 * (cudaGraphExecUpdate).  Pushes made while profiling is enabled are not
 * captured.  enable == 0 (the default): kernels are launched one by one.
 * Results are identical either way. */
int sb_ctx_graphs(sb_ctx *ctx, int32_t enable);
/* enable != 0 (the default): the first push that launches the mixing kernel
 * (a3 + a4) with a new launch shape (operand type, whether the level's SNR is
 * stored, whether it interpolates a coarser level, K chunks per tile, bytes of
 * K per chunk, tile count rounded down to a power of four) times every
 * pipeline shape that fits in shared memory (mixing stages 1-4,
 * interpolation buffers 1-2, window-ring depth 2-4) on that push's
 * own data, three times in interleaved rounds, and keeps the one with the
 * smallest time for later pushes; that push is not graph-captured.  The
 * pipeline shape changes no arithmetic: results are bitwise the same for every
 * choice.  enable == 0: later launches use the built-in shape for new launch
 * shapes (tuned shapes are kept). */
int sb_ctx_autotune(sb_ctx *ctx, int32_t enable);
/* The tuned launch shapes: writes min(cap, number tuned) records of four int32
 * {shape key, mixing stages, interpolation buffers, window-ring depth} into out
 * (4 * cap entries) and returns the number of tuned shapes (>= 0), or a
 * negative SB_E* code.  Shape key bits: 0-1 operand type of the mixing (0 FP16,
 * 1 BF16; SB_FP8 units mix in BF16), 2 SNR stored, 3 interpolates a coarser
 * level, 4-5 K chunks per tile (capped at 3), 6-7 bytes of K per chunk (0: 32,
 * 1: 64, 2: 128), 8+ log4 tiles. */
int sb_ctx_autotune_choices(sb_ctx *ctx, int32_t *out, int32_t cap);
/* Test hook of the bounded device waits (the paper has no counterpart): every
 * later push's basis-FIR kernel (SB_BF16 / SB_FP16 / SB_FP8) bounds its waits
 * by wait_limit_ns (0: the default, 2 s), and when skip_fir_chunk >= 0 the
 * producer of the launch's first tile does not issue the load of that K chunk,
 * so that the chunk's consumer waits until the bound expires; the kernel then
 * lets every copy it issued land, lets its issued MMAs finish, frees its TMEM
 * and returns, and triggers_pop reports SB_ETIMEOUT for that push (whose
 * results are void).  Nothing faults and nothing stays in flight.  Make the
 * test pushes with sb_ctx_graphs off; a negative skip_fir_chunk restores normal
 * operation. */
int sb_ctx_test_wait(sb_ctx *ctx, int64_t wait_limit_ns, int32_t skip_fir_chunk);
/* Blocks until queued work is done, then writes per stage the summed kernel
 * time (ms) and the number of launches since profiling was enabled
 * (arrays of n_stages entries; n_stages <= SB_N_STAGES). */
int sb_ctx_stage_times(sb_ctx *ctx, double *ms, int64_t *launches, int32_t n_stages);

/* Window maxima and triggers of a caller's top-rate SNR block without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc/cudaFree while they run (a serving
 * loop replaying CUDA graphs, or a process whose device memory belongs to a
 * pool it does not own), where allocating would synchronise the device or
 * fail.
 * x: device FP32 [2M][ldx], row a = 2i + p (p = 0 cosine, 1 sine phase);
 * column c is absolute top-rate sample first_sample + c.  Every window
 * [w window_len, (w+1) window_len) lying entirely inside
 * [max(0, first_sample), first_sample + n_samples) gives its |rho| maximum
 * (first sample on ties); a trigger (unit = -1, template_id from the device
 * array template_ids or i when NULL) is written to the device array out when
 * |rho| > threshold.  out_count: device int32[2] = {triggers stored, overflow
 * flag}, zeroed by the call; at most cap triggers are stored, out_count[0]
 * never exceeds cap, and out_count[1] = 1 when more windows qualified than
 * cap (which ones were kept is then unspecified).  Work is queued on stream
 * (a cudaStream_t; NULL = legacy default stream) and nothing blocks.
 * Scratch: a fixed device array of 2^18 partial records (8 MiB) that every
 * GPU loading this library holds until the process exits; a call needs
 * 2 * M * ceil(n_samples / 256) records and returns SB_EINVAL (see
 * sb_last_error) beyond that, or when window_len < 256.  The first call on a
 * device looks up the array's device address; with CUDA's lazy module loading
 * (the default) that lookup may load the library's device module, which can
 * allocate device memory, so make the first call on each device before the
 * phase in which nothing may allocate, and before any stream capture.  The
 * looked-up address is cached per device ordinal and is no longer valid after
 * cudaDeviceReset on that device.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race; serialise them. */
int sb_window_triggers_noalloc(const float *x, int64_t ldx, int32_t n_templates, int64_t n_samples,
                               int64_t first_sample, int64_t window_len, float threshold,
                               const int64_t *template_ids, sb_trigger *out, int32_t *out_count, int32_t cap,
                               void *stream);

/* Message describing the calling thread's last error ("" if none). */
const char *sb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LLOID_H */
