// sb_window_triggers_noalloc: the window-maximum trigger pick (partial maxima
// per window segment, then one merge per template) on a caller's top-rate SNR
// block, with its scratch in a fixed device array instead of library-allocated
// memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree at run time — for
// example a caller running inside a CUDA-graph-driven serving loop or under a
// memory pool it does not control, where an allocation would synchronise the
// device or fail.  It passes its own input and output buffers; the scratch
// lives in the static array below, which every GPU that loads this library
// holds until the process exits.
#include <cstddef>
#include <mutex>
#include <string>

#include "lloid.h"
#include "lloid_internal.h"

namespace lloid {

// Maximum partial-maximum records one call may need: 2 per (template, 256-sample chunk).
constexpr int64_t kNoAllocRecords = int64_t(1) << 18;      // 262144 records x 32 B = 8 MiB
constexpr int kNoAllocChunk = 256;

static __device__ __align__(256) WinPart g_noalloc_scratch[kNoAllocRecords];

// The merge kernel writes sb_trigger records through DevTrigger.
static_assert(sizeof(DevTrigger) == sizeof(sb_trigger), "DevTrigger and sb_trigger differ in size");
static_assert(offsetof(DevTrigger, template_id) == offsetof(sb_trigger, template_id) &&
                  offsetof(DevTrigger, sample) == offsetof(sb_trigger, sample) &&
                  offsetof(DevTrigger, window) == offsetof(sb_trigger, window) &&
                  offsetof(DevTrigger, snr) == offsetof(sb_trigger, snr) &&
                  offsetof(DevTrigger, phase) == offsetof(sb_trigger, phase) &&
                  offsetof(DevTrigger, snr_peak) == offsetof(sb_trigger, snr_peak) &&
                  offsetof(DevTrigger, dt_peak) == offsetof(sb_trigger, dt_peak) &&
                  offsetof(DevTrigger, flags) == offsetof(sb_trigger, flags) &&
                  offsetof(DevTrigger, xi2) == offsetof(sb_trigger, xi2),
              "DevTrigger and sb_trigger differ in layout");

// One warp per (template, chunk): the |rho|^2 maximum (first sample on ties) of
// each of the (at most two) windows the chunk touches.  Records of samples
// outside [start_abs, end_abs) are left empty (mag2 = -1).
__global__ void __launch_bounds__(256) noalloc_partials_kernel(const float *__restrict__ x, int64_t ldx, int M,
                                                               int64_t n, int64_t first, int64_t start_abs,
                                                               int64_t end_abs, int64_t win_len, int n_chunks,
                                                               WinPart *__restrict__ scratch) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= M * n_chunks) return;
    const int i = gw / n_chunks, c = gw % n_chunks;
    const int64_t p0 = (int64_t)c * kNoAllocChunk;
    const int64_t chunk_first = first + p0;
    const int64_t w0 = (chunk_first > start_abs ? chunk_first : start_abs) / win_len;
    const float *xc = x + (int64_t)(2 * i) * ldx;
    const float *xs = xc + ldx;
    float best[2] = {-1.0f, -1.0f};
    int64_t bn[2] = {INT64_MAX, INT64_MAX};
    for (int64_t p = p0 + lane; p < p0 + kNoAllocChunk && p < n; p += 32) {
        const int64_t na = first + p;
        if (na < start_abs || na >= end_abs) continue;
        const float cval = xc[p], sval = xs[p];
        const float m2 = fmaf(sval, sval, cval * cval);
        const int s = (na / win_len == w0) ? 0 : 1;
        if (m2 > best[s]) { best[s] = m2; bn[s] = na; }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best[s], off);
            const int64_t on = __shfl_xor_sync(0xffffffffu, bn[s], off);
            if (ob > best[s] || (ob == best[s] && on < bn[s])) { best[s] = ob; bn[s] = on; }
        }
    }
    if (lane == 0) {
        for (int s = 0; s < 2; ++s) {
            WinPart r{-1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, -1};
            if (bn[s] != INT64_MAX) {
                const int64_t p = bn[s] - first;
                r = WinPart{best[s], xc[p], xs[p], 0.0f, 0.0f, 0.0f, 0, (int32_t)p};
            }
            scratch[((int64_t)c * 2 + s) * M + i] = r;
        }
    }
}

// One thread per template: merge the records in time order; every window that
// lies entirely inside [start_abs, end_abs) yields its maximum, a trigger when
// |rho| > threshold.
__global__ void __launch_bounds__(256) noalloc_merge_kernel(const WinPart *__restrict__ scratch, int M, int n_rec,
                                                            const int64_t *__restrict__ template_ids, int64_t first,
                                                            int64_t start_abs, int64_t end_abs, int64_t win_len,
                                                            float threshold, DevTrigger *out, int32_t *count,
                                                            int32_t cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    float bm = -1.0f, bre = 0.0f, bim = 0.0f;
    int64_t bnn = -1, w_cur = -1;
    auto close = [&](int64_t w) {
        const bool whole = w * win_len >= start_abs && (w + 1) * win_len <= end_abs;
        if (!whole || bm < 0.0f || !(sqrtf(bm) > threshold)) return;
        // claim a slot only while fewer than cap are taken, so count[0] never exceeds cap
        int slot = *reinterpret_cast<volatile int32_t *>(count);
        while (slot < cap) {
            const int prev = atomicCAS(count, slot, slot + 1);
            if (prev == slot) break;
            slot = prev;
        }
        if (slot >= cap) {
            atomicExch(count + 1, 1);
            return;
        }
        DevTrigger r;
        r.unit = -1;
        r.template_id = template_ids ? template_ids[i] : i;
        r.sample = bnn;
        r.window = w;
        r.snr = sqrtf(bm);
        r.phase = atan2f(bim, bre);
        r.snr_peak = r.snr;
        r.dt_peak = 0.0f;
        r.flags = 0;
        r.xi2 = 0.0f;
        out[slot] = r;
    };
    for (int r = 0; r < n_rec; ++r) {
        const WinPart p = scratch[(int64_t)r * M + i];
        if (p.mag2 < 0.0f) continue;
        const int64_t pn = first + p.nr;
        const int64_t w = pn / win_len;
        if (w != w_cur) {
            if (w_cur >= 0) close(w_cur);
            bm = -1.0f;
            w_cur = w;
        }
        if (p.mag2 > bm) { bm = p.mag2; bre = p.re; bim = p.im; bnn = pn; }
    }
    if (w_cur >= 0) close(w_cur);
}

}  // namespace lloid

using namespace lloid;

// Reported through sb_last_error (lloid_api.cu).
void set_last_error(const std::string &msg);

// Device address of the static scratch, looked up once per device with that
// device current (a host-side use of the array's name would not be a device address).
static int scratch_address(int device, WinPart **out) {
    static std::mutex mu;
    static WinPart *addr[64] = {nullptr};
    if (device < 0 || device >= 64) return SB_EINVAL;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SB_ECUDA;
        }
        addr[device] = static_cast<WinPart *>(p);
    }
    *out = addr[device];
    return SB_OK;
}

extern "C" int sb_window_triggers_noalloc(const float *x, int64_t ldx, int32_t n_templates, int64_t n_samples,
                                          int64_t first_sample, int64_t window_len, float threshold,
                                          const int64_t *template_ids, sb_trigger *out, int32_t *out_count,
                                          int32_t cap, void *stream) {
    if (!x || !out || !out_count || n_templates <= 0 || n_samples <= 0 || ldx < n_samples || window_len <= 0 ||
        cap < 0) {
        set_last_error("sb_window_triggers_noalloc: null pointer or bad size");
        return SB_EINVAL;
    }
    const int64_t n_chunks = (n_samples + kNoAllocChunk - 1) / kNoAllocChunk;
    if (window_len < kNoAllocChunk) {
        set_last_error("sb_window_triggers_noalloc: window_len must be >= 256 samples");
        return SB_EINVAL;
    }
    if ((int64_t)n_templates * n_chunks * 2 > kNoAllocRecords) {
        set_last_error("sb_window_triggers_noalloc: n_templates * ceil(n_samples / 256) * 2 = " +
                        std::to_string((int64_t)n_templates * n_chunks * 2) + " exceeds the fixed scratch of " +
                        std::to_string(kNoAllocRecords) + " records");
        return SB_EINVAL;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return SB_ECUDA;
    }
    WinPart *scratch = nullptr;
    int rc = scratch_address(device, &scratch);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t start_abs = first_sample > 0 ? first_sample : 0;
    const int64_t end_abs = first_sample + n_samples;
    e = cudaMemsetAsync(out_count, 0, 2 * sizeof(int32_t), st);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return SB_ECUDA;
    }
    const int64_t warps = (int64_t)n_templates * n_chunks;
    noalloc_partials_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        x, ldx, n_templates, n_samples, first_sample, start_abs, end_abs, window_len, (int)n_chunks, scratch);
    noalloc_merge_kernel<<<(n_templates + 255) / 256, 256, 0, st>>>(
        scratch, n_templates, (int)(n_chunks * 2), template_ids, first_sample, start_abs, end_abs, window_len,
        threshold,
        reinterpret_cast<DevTrigger *>(out), out_count, cap);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return SB_ECUDA;
    }
    return SB_OK;
}
