// SIMT kernels of the LLOID hot path: interpolation (a4), history copies, the
// FP32 GEMM used for the basis FIR (a2, Toeplitz B operand) and the mixing step
// (a3) in SB_FP32 mode, and the window-maximum trigger generator (a5).  The
// decimation cascade (a1) is in kernels_cascade.cu.  Every kernel walks a device task list so that one
// launch serves all units of a grouped push.
#include "gemm_fp32_tile.cuh"
#include "lloid_internal.h"

namespace lloid {

// ---------------------------------------------------------------------------
// a4 (up-sampling half): y'[n] = sum_m 2 g[n - 2m] y[m]; even n copy y[n/2].
// ---------------------------------------------------------------------------
// One CTA per (task, row, group of kUpGroup chunks of kUpChunk outputs).  Each
// chunk's input segment (half the chunk plus the 2K-1 tap halo on each side) is
// staged in shared memory with coalesced loads; the next chunk's segment is
// fetched into registers while the current one is filtered (two shared-memory
// buffers), so the loads' latency hides behind the arithmetic.  Each thread
// forms whole output pairs (the even output of coarser sample a and the odd one
// after it), so no lane idles while its neighbour filters, consecutive lanes
// read consecutive shared-memory words, and the 2K-tap sum runs in four
// independent partial sums.
constexpr int kUpSeg = kUpChunk / 2 + 2 * kHalfK + 2;
constexpr int kUpThreads = 256;
constexpr int kUpLoads = (kUpSeg + kUpThreads - 1) / kUpThreads;   // segment samples per thread

__global__ void __launch_bounds__(kUpThreads) upsample_kernel(const UpTask *__restrict__ tasks, Halfband g) {
    griddep_wait();
    __shared__ float seg[2][kUpSeg];
    const UpTask &t = tasks[blockIdx.z];
    const int row = blockIdx.y;
    if (row >= t.rows) return;
    const int64_t n_valid = (int64_t)t.n_hist + t.n_cur;
    const float *hist = t.hist + row * t.ld_hist;
    const float *cur = t.cur + row * t.ld_cur;
    float *out = t.out + row * t.ld_out;
    float c[kOddTaps];
#pragma unroll
    for (int k = 0; k < kOddTaps; ++k) c[k] = 2.0f * g.odd[k];
    // first input position touched by the chunk at p0: output nrel = p0 - lam_out, tap j = 2K - 1
    auto pos_lo_of = [&](int64_t p0) { return (((p0 - t.lam_out) - (2 * kHalfK - 1)) >> 1) + t.in_off; };
    float rv[kUpLoads];
    auto fetch = [&](int64_t p0) {
        const int64_t pos_lo = pos_lo_of(p0);
#pragma unroll
        for (int r = 0; r < kUpLoads; ++r) {
            const int i = threadIdx.x + kUpThreads * r;
            const int64_t pos = pos_lo + i;
            float v = 0.0f;
            if (i < kUpSeg && pos >= 0 && pos < n_valid) v = pos < t.n_hist ? hist[pos] : cur[pos - t.n_hist];
            rv[r] = v;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int r = 0; r < kUpLoads; ++r) {
            const int i = threadIdx.x + kUpThreads * r;
            if (i < kUpSeg) seg[buf][i] = rv[r];
        }
    };
    const int64_t g0 = (int64_t)blockIdx.x * kUpGroup * kUpChunk;
    if (g0 >= t.n_out) return;                               // block-uniform
    fetch(g0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int ch = 0; ch < kUpGroup; ++ch) {
        const int64_t p0 = g0 + (int64_t)ch * kUpChunk;
        if (p0 >= t.n_out) break;                            // block-uniform
        const bool more = ch + 1 < kUpGroup && p0 + kUpChunk < t.n_out;
        if (more) fetch(p0 + kUpChunk);                      // in flight while this chunk is filtered
        const float *sg = seg[buf];
        const int64_t nrel0 = p0 - t.lam_out;
        const int64_t pos_lo = pos_lo_of(p0);
        const int64_t p_end = min((int64_t)t.n_out, p0 + kUpChunk);
        // coarser samples a whose outputs 2a, 2a + 1 (relative to lam_out) fall in [p0, p_end)
        const int64_t a_first = nrel0 >> 1;
        const int64_t a_last = (p_end - 1 - t.lam_out) >> 1;
        const int64_t off = t.in_off - pos_lo;              // seg index of coarser sample a: a + off
        for (int64_t a = a_first + threadIdx.x; a <= a_last; a += kUpThreads) {
            const int lo = (int)(a + off);
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
            for (int k = 0; k < kOddTaps; k += 4) {
                s0 = fmaf(c[k], sg[lo - k] + sg[lo + 1 + k], s0);
                s1 = fmaf(c[k + 1], sg[lo - k - 1] + sg[lo + 2 + k], s1);
                s2 = fmaf(c[k + 2], sg[lo - k - 2] + sg[lo + 3 + k], s2);
                s3 = fmaf(c[k + 3], sg[lo - k - 3] + sg[lo + 4 + k], s3);
            }
            const int64_t pe = 2 * a + t.lam_out;           // output index of the even sample
            if (pe >= p0 && pe < p_end) out[pe] = t.first_n + pe >= 0 ? sg[lo] : 0.0f;
            if (pe + 1 >= p0 && pe + 1 < p_end)
                out[pe + 1] = t.first_n + pe + 1 >= 0 ? (s0 + s1) + (s2 + s3) : 0.0f;
        }
        if (more) {
            stash(buf ^ 1);                                  // the other buffer: last read one chunk ago
            __syncthreads();
            buf ^= 1;
        }
    }
}

// ---------------------------------------------------------------------------
// history shifts: dst[r][i] = [hist | cur][r][off + i]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) copy_kernel(const CopyTask *__restrict__ tasks) {
    griddep_wait();
    const CopyTask t = tasks[blockIdx.z];
    const int row = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= t.rows || i >= t.n) return;
    const int64_t pos = (int64_t)t.off + i;
    if (t.elem16) {
        const uint16_t *hist = reinterpret_cast<const uint16_t *>(t.hist);
        const uint16_t *cur = reinterpret_cast<const uint16_t *>(t.cur);
        uint16_t *dst = reinterpret_cast<uint16_t *>(t.dst);
        for (int part = 0; part < t.elem16; ++part) {
            const int64_t r = row + (int64_t)part * t.rows;
            dst[r * t.ld_dst + i] = pos < t.n_hist ? hist[r * t.ld_hist + pos] : cur[r * t.ld_cur + (pos - t.n_hist)];
        }
        return;
    }
    const float v = pos < t.n_hist ? t.hist[row * t.ld_hist + pos] : t.cur[row * t.ld_cur + (pos - t.n_hist)];
    t.dst[row * t.ld_dst + i] = v;
}

// 16-bit history shifts (the stored y_k of the tensor-core modes): one warp per row, each
// instruction moving 32 consecutive columns (rows are a few dozen to a few hundred columns long).
__global__ void __launch_bounds__(256) copy16_kernel(const CopyTask *__restrict__ tasks) {
    griddep_wait();
    const CopyTask t = tasks[blockIdx.y];
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= t.rows) return;
    const uint16_t *hist = reinterpret_cast<const uint16_t *>(t.hist);
    const uint16_t *cur = reinterpret_cast<const uint16_t *>(t.cur);
    uint16_t *dst = reinterpret_cast<uint16_t *>(t.dst);
    for (int part = 0; part < t.elem16; ++part) {
        const int64_t r = row + (int64_t)part * t.rows;
        for (int i = lane; i < t.n; i += 32) {
            const int64_t pos = (int64_t)t.off + i;
            dst[r * t.ld_dst + i] = pos < t.n_hist ? hist[r * t.ld_hist + pos] : cur[r * t.ld_cur + (pos - t.n_hist)];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 tiled GEMM over a task list (64 x 128 tile, 256 threads, 4x8 per thread).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_task_by_tile(const GemmTask *tasks, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256, 2) gemm_fp32_kernel(const GemmTask *__restrict__ tasks, int n_tasks) {
    griddep_wait();
    const int ti = find_task_by_tile(tasks, n_tasks, blockIdx.x);
    const GemmTask t = tasks[ti];
    const int local = blockIdx.x - t.tile_begin;
    gemm_fp32_tile(t, (local / t.tiles_n) * kGemmTM, (local % t.tiles_n) * kGemmTN);
}

// ---------------------------------------------------------------------------
// a5: per (template, window) maximum of |rho|^2 (first index on ties), strict
// threshold, phase; one warp per (unit, template, window segment).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool better(float m_a, int64_t n_a, float m_b, int64_t n_b) {
    return m_a > m_b || (m_a == m_b && n_a < n_b);
}

__device__ __forceinline__ int find_task_by_warp(const WinTask *tasks, int n, int w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].warp_begin <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) window_max_kernel(const WinTask *__restrict__ tasks, int n_tasks,
                                                         int total_warps, TrigOut out) {
    griddep_wait();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= total_warps) return;
    const WinTask &t = tasks[find_task_by_warp(tasks, n_tasks, gw)];
    const int local = gw - t.warp_begin;
    const int i = local / t.n_seg;
    const int s = local % t.n_seg;
    const int64_t start_abs = t.first_n > 0 ? t.first_n : 0;
    const int64_t end_abs = t.first_n + t.n;
    const int64_t w = start_abs / t.win_len + s;
    const int64_t seg_lo = max(w * t.win_len, start_abs);
    const int64_t seg_hi = min((w + 1) * t.win_len, end_abs);
    const float *xc = t.x + (int64_t)(2 * i) * t.ldx;    // column p <-> absolute n = first_n + p
    const float *xs = xc + t.ldx;

    float best = -1.0f;
    int64_t bn = INT64_MAX;
    for (int64_t n = seg_lo + lane; n < seg_hi; n += 32) {
        const float c = xc[n - t.first_n], q = xs[n - t.first_n];
        const float m2 = fmaf(q, q, c * c);
        if (m2 > best) { best = m2; bn = n; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t on = __shfl_xor_sync(0xffffffffu, bn, off);
        if (better(ob, on, best, bn)) { best = ob; bn = on; }
    }
    // xi^2 over lags -kXiJ .. kXiJ when they all lie in this push (every lane holds bn)
    float xi = 0.0f;
    bool has_xi = false;
    if (t.acorr && bn != INT64_MAX && bn - kXiJ >= 0 && bn - t.first_n - kXiJ >= 0 && bn - t.first_n + kXiJ < t.n) {
        const int64_t p = bn - t.first_n;
        const float z0c = xc[p], z0s = xs[p];
        const float2 *Ri = t.acorr + (int64_t)i * kXiLags;
        float num = 0.0f, den = 0.0f;
        for (int j = lane; j < kXiLags; j += 32) {
            const float2 r = Ri[j];
            const float ec = xc[p - kXiJ + j] - (z0c * r.x - z0s * r.y);
            const float es = xs[p - kXiJ + j] - (z0c * r.y + z0s * r.x);
            num += fmaf(es, es, ec * ec);
            den += 2.0f - 2.0f * fmaf(r.y, r.y, r.x * r.x);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, off);
            den += __shfl_xor_sync(0xffffffffu, den, off);
        }
        xi = num / den;
        has_xi = true;
    }
    if (lane != 0) return;
    float re = 0.0f, im = 0.0f, pk = 0.0f, dt = 0.0f;
    int fl = 0;
    if (bn != INT64_MAX) {
        const int64_t p = bn - t.first_n;
        re = xc[p];
        im = xs[p];
        if (bn >= 1 && p >= 1 && p + 1 < t.n) {   // both neighbours in this push: sub-sample peak
            const float ym = fmaf(xs[p - 1], xs[p - 1], xc[p - 1] * xc[p - 1]);
            const float yp = fmaf(xs[p + 1], xs[p + 1], xc[p + 1] * xc[p + 1]);
            if (subsample_peak(ym, best, yp, pk, dt)) fl = SB_TRIG_SUBSAMPLE_BIT;
        }
        if (has_xi) fl |= SB_TRIG_XI2_BIT;
    }
    if (s == 0) {                          // the open window carried over from the last push
        const WinState st = t.state_in[i];
        if (st.mag2 >= 0.0f && !(best > st.mag2)) {
            best = st.mag2; bn = st.n; re = st.re; im = st.im; pk = st.pk; dt = st.dt; xi = st.xi2; fl = st.flags;
        }
    }
    const bool complete = (w + 1) * t.win_len <= end_abs;
    if (complete) {
        if (bn != INT64_MAX && sqrtf(best) > t.threshold) {
            const int slot = atomicAdd(out.count, 1);
            if (slot < out.cap) {
                DevTrigger r;
                r.unit = t.unit_id;
                r.template_id = t.template_ids[i];
                r.sample = bn;
                r.window = w;
                r.snr = sqrtf(best);
                r.phase = atan2f(im, re);
                r.snr_peak = (fl & SB_TRIG_SUBSAMPLE_BIT) ? pk : r.snr;
                r.dt_peak = (fl & SB_TRIG_SUBSAMPLE_BIT) ? dt : 0.0f;
                r.flags = fl;
                r.xi2 = (fl & SB_TRIG_XI2_BIT) ? xi : 0.0f;
                out.buf[slot] = r;
            } else {
                atomicExch(out.count + 1, 1);
            }
        }
    }
    if (s == t.n_seg - 1) {
        WinState ns;
        if (complete) { ns.mag2 = -1.0f; ns.re = ns.im = ns.pk = ns.dt = ns.xi2 = 0.0f; ns.n = -1; ns.flags = 0; }
        else { ns.mag2 = best; ns.re = re; ns.im = im; ns.pk = pk; ns.dt = dt; ns.xi2 = xi; ns.n = bn; ns.flags = fl; }
        t.state_out[i] = ns;
    }
}

// ---------------------------------------------------------------------------
// a5 after partial maxima: one thread per (unit, template) walks the unit's
// partial records in time order, closes every window the push completes
// (threshold, phase, trigger) and keeps the open window's running maximum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_task_by_warp(const WinFinTask *tasks, int n, int w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].warp_begin <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) win_finalize_kernel(const WinFinTask *__restrict__ tasks, int n_tasks,
                                                           int total_warps, TrigOut out) {
    griddep_wait();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= total_warps) return;
    const WinFinTask &t = tasks[find_task_by_warp(tasks, n_tasks, gw)];
    const int local = gw - t.warp_begin;
    const int i = local / t.n_win, s = local % t.n_win;
    // a completed window that neither takes over nor hands on an open state, with no record above the
    // (lower) refinement threshold, has no trigger
    if (t.wmax && s > 0 && s < t.n_win - 1 && t.wmax[(int64_t)i * t.n_wslot + s] == 0u) return;
    const int64_t w = t.start_abs / t.win_len + s;
    const int64_t lo = max(w * t.win_len, t.start_abs) - t.first_n;        // push columns of window w
    const int64_t hi = min((w + 1) * t.win_len, t.end_abs) - t.first_n;
    const int r0 = (int)(lo / 128) * 2, r1 = (int)((hi - 1) / 128) * 2 + 2;
    const WinPart *rec = t.part + (int64_t)i * t.n_rec;
    float best = -1.0f, re = 0.0f, im = 0.0f, pk = 0.0f, dt = 0.0f, xi = 0.0f;
    int64_t bn = INT64_MAX;
    int fl = 0;
    for (int r = r0 + lane; r < r1; r += 32) {
        const WinPart p = rec[r];
        const int64_t pn = t.first_n + p.nr;
        if (p.mag2 < 0.0f || pn / t.win_len != w) continue;
        if (p.mag2 > best || (p.mag2 == best && pn < bn)) {
            best = p.mag2; bn = pn; re = p.re; im = p.im; pk = p.pk; dt = p.dt; xi = p.xi2; fl = p.flags;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t on = __shfl_xor_sync(0xffffffffu, bn, off);
        const float ore = __shfl_xor_sync(0xffffffffu, re, off);
        const float oim = __shfl_xor_sync(0xffffffffu, im, off);
        const float opk = __shfl_xor_sync(0xffffffffu, pk, off);
        const float odt = __shfl_xor_sync(0xffffffffu, dt, off);
        const float oxi = __shfl_xor_sync(0xffffffffu, xi, off);
        const int ofl = __shfl_xor_sync(0xffffffffu, fl, off);
        if (ob > best || (ob == best && on < bn)) {
            best = ob; bn = on; re = ore; im = oim; pk = opk; dt = odt; xi = oxi; fl = ofl;
        }
    }
    if (lane != 0) return;
    if (s == 0) {                          // the window left open by the previous push (earlier samples)
        const WinState st = t.state_in[i];
        if (st.mag2 >= 0.0f && !(best > st.mag2)) {
            best = st.mag2; bn = st.n; re = st.re; im = st.im; pk = st.pk; dt = st.dt; xi = st.xi2; fl = st.flags;
        }
    }
    const bool complete = (w + 1) * t.win_len <= t.end_abs;
    if (complete && bn != INT64_MAX && sqrtf(best) > t.threshold) {
        const int slot = atomicAdd(out.count, 1);
        if (slot < out.cap) {
            DevTrigger r;
            r.unit = t.unit_id;
            r.template_id = t.template_ids[i];
            r.sample = bn;
            r.window = w;
            r.snr = sqrtf(best);
            r.phase = atan2f(im, re);
            r.snr_peak = (fl & SB_TRIG_SUBSAMPLE_BIT) ? pk : r.snr;
            r.dt_peak = (fl & SB_TRIG_SUBSAMPLE_BIT) ? dt : 0.0f;
            r.flags = fl;
            r.xi2 = (fl & SB_TRIG_XI2_BIT) ? xi : 0.0f;
            out.buf[slot] = r;
        } else {
            atomicExch(out.count + 1, 1);
        }
    }
    if (s == t.n_win - 1) {
        WinState ns;
        if (complete || bn == INT64_MAX) {
            ns.mag2 = -1.0f; ns.re = ns.im = ns.pk = ns.dt = ns.xi2 = 0.0f; ns.n = -1; ns.flags = 0;
        } else {
            ns.mag2 = best; ns.re = re; ns.im = im; ns.pk = pk; ns.dt = dt; ns.xi2 = xi; ns.n = bn; ns.flags = fl;
        }
        t.state_out[i] = ns;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_win_finalize(const WinFinTask *d_tasks, int n_tasks, int total_warps, TrigOut out,
                                cudaStream_t s) {
    if (n_tasks == 0 || total_warps == 0) return cudaSuccess;
    return launch_pdl(win_finalize_kernel, dim3((total_warps * 32 + 255) / 256), dim3(256), 0, s, d_tasks, n_tasks,
                      total_warps, out);
}

cudaError_t launch_upsample(const UpTask *d_tasks, int n_tasks, int max_rows, int max_out,
                            const Halfband &g, cudaStream_t s) {
    if (n_tasks == 0 || max_out <= 0 || max_rows <= 0) return cudaSuccess;
    dim3 grid((max_out + kUpGroup * kUpChunk - 1) / (kUpGroup * kUpChunk), max_rows, n_tasks);
    return launch_pdl(upsample_kernel, grid, dim3(kUpThreads), 0, s, d_tasks, g);
}

cudaError_t launch_copy16(const CopyTask *d_tasks, int n_tasks, int max_rows, cudaStream_t s) {
    if (n_tasks == 0 || max_rows <= 0) return cudaSuccess;
    return launch_pdl(copy16_kernel, dim3((max_rows + 7) / 8, n_tasks), dim3(256), 0, s, d_tasks);
}

cudaError_t launch_copy(const CopyTask *d_tasks, int n_tasks, int max_rows, int max_n, cudaStream_t s) {
    if (n_tasks == 0 || max_n <= 0 || max_rows <= 0) return cudaSuccess;
    dim3 grid((max_n + 255) / 256, max_rows, n_tasks);
    return launch_pdl(copy_kernel, grid, dim3(256), 0, s, d_tasks);
}

cudaError_t launch_gemm_fp32(const GemmTask *d_tasks, int n_tasks, int total_tiles, cudaStream_t s) {
    if (n_tasks == 0 || total_tiles == 0) return cudaSuccess;
    return launch_pdl(gemm_fp32_kernel, dim3(total_tiles), dim3(256), 0, s, d_tasks, n_tasks);
}

cudaError_t launch_window_max(const WinTask *d_tasks, int n_tasks, int total_warps, TrigOut out,
                              cudaStream_t s) {
    if (n_tasks == 0 || total_warps == 0) return cudaSuccess;
    const int blocks = (total_warps * 32 + 255) / 256;
    return launch_pdl(window_max_kernel, dim3(blocks), dim3(256), 0, s, d_tasks, n_tasks, total_warps, out);
}

}  // namespace lloid
