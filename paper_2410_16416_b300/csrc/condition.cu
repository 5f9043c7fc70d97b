// Data conditioning ahead of the filter (Sec. II.A, Fig. 1 caption): a running
// average of the noise PSD whitens the strain, and large deviations of the
// whitened data are gated out.  The paper names the steps only; the library
// follows these readings:
//
//  whitening  N-sample segments every H = N/2 samples, periodic Hann window
//             w[n] = sin^2(pi n / N) (its copies H apart sum to one);
//             X_j = DFT(w d_j), S_j = |X_j|^2 / sum w^2 (per-bin variance);
//             running average P_j = P_{j-1} + (S_j - P_{j-1}) / min(j+1, n_avg);
//             segment j is divided by the average of the segments before it,
//             Y_j = X_j / sqrt(P_{j-1}) (segment 0 by its own P_0), inverse DFT,
//             overlap-add.
//  gating     every whitened sample above the threshold is a glitch sample;
//             samples within `half` of one are zeroed and the weight returns to
//             one over a sin^2 ramp of `taper` samples.
//
// One push of n samples (a multiple of H) runs five kernels on the context's
// stream: the forward FFT of every segment the push completes (one CTA per
// segment, radix-2 Stockham FFT of N/2 complex points in shared memory with
// the real-input split), the running average and the division (one thread per
// frequency bin, segments in order), the inverse FFT, the overlap-add into a
// ring of whitened samples (plus the list of glitch samples in it), and the
// gate.  The output is delayed by latency = H + half + taper samples, the
// look-ahead the overlap-add and the gate need.
#include <cmath>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "lloid.h"
#include "lloid_internal.h"

namespace lloid {

constexpr int kCondThreads = 512;
constexpr int kCondMinN = 64, kCondMaxN = 16384;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Radix-2 Stockham FFT of M = 2^logM points held in shared memory (a), ping-pong with b; stage s
// (span Ns = 2^s) takes a[j], a[j + M/2] to b[2 Ns (j / Ns) + j % Ns] and the same + Ns with the
// twiddle e^{-+2 pi i (j % Ns) / (2 Ns)} = tw[(j % Ns) M / (2 Ns)] (conjugated for the inverse).
// Returns the buffer holding the result, in natural order.
template <bool INV>
__device__ float2 *fft_stockham(float2 *a, float2 *b, int M, int logM, const float2 *__restrict__ tw) {
    for (int s = 0; s < logM; ++s) {
        const int Ns = 1 << s;
        for (int j = threadIdx.x; j < M / 2; j += blockDim.x) {
            const int k = j & (Ns - 1);
            float2 w = __ldg(&tw[k << (logM - 1 - s)]);
            if (INV) w.y = -w.y;
            const float2 v0 = a[j], t = cmul(a[j + M / 2], w);
            const int o = ((j - k) << 1) + k;
            b[o] = cadd(v0, t);
            b[o + Ns] = csub(v0, t);
        }
        __syncthreads();
        float2 *x = a;
        a = b;
        b = x;
    }
    return a;
}

struct CondGeom {
    int N, M, logM, H;
    float inv_sumw2;          // 1 / sum w^2 = 8 / (3 N)
};

// Forward: segment s of this push starts at raw[seg0_off + s H]; X[s][f], f = 0 .. M.
__global__ void __launch_bounds__(kCondThreads) cond_forward_kernel(const float *__restrict__ raw, int64_t seg0_off,
                                                                     CondGeom g, const float2 *__restrict__ tw,
                                                                     const float2 *__restrict__ rtw,
                                                                     float2 *__restrict__ X) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + g.M;
    const float *x = raw + seg0_off + (int64_t)blockIdx.x * g.H;
    const float inv_n = 1.0f / (float)g.N;
    for (int m = threadIdx.x; m < g.M; m += blockDim.x) {
        const float s0 = sinpif((float)(2 * m) * inv_n), s1 = sinpif((float)(2 * m + 1) * inv_n);
        a[m] = make_float2(x[2 * m] * s0 * s0, x[2 * m + 1] * s1 * s1);
    }
    __syncthreads();
    const float2 *Z = fft_stockham<false>(a, b, g.M, g.logM, tw);
    float2 *out = X + (int64_t)blockIdx.x * (g.M + 1);
    // real split: X[f] = (Z[f] + conj Z[M-f]) / 2 - i/2 W^f (Z[f] - conj Z[M-f]), W = e^{-2 pi i / N}
    for (int f = threadIdx.x; f <= g.M; f += blockDim.x) {
        const float2 zf = Z[f == g.M ? 0 : f], zc = conjf2(Z[f == 0 ? 0 : g.M - f]);
        const float2 e = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y + zc.y));
        const float2 d = make_float2(0.5f * (zf.x - zc.x), 0.5f * (zf.y - zc.y));
        const float2 od = cmul(make_float2(d.y, -d.x), __ldg(&rtw[f]));     // -i d W^f
        out[f] = cadd(e, od);
    }
}

// Running average and division, one thread per bin: for this push's segments in order,
// Y = X / sqrt(P_before) (segment 0 of the stream: its own average), then P += (S - P) / min(j+1, n_avg).
__global__ void __launch_bounds__(256) cond_psd_kernel(float2 *__restrict__ X, float *__restrict__ psd, int n_seg,
                                                       int64_t seg_first, int n_avg, CondGeom g) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f > g.M) return;
    float P = psd[f];
    for (int s = 0; s < n_seg; ++s) {
        float2 *x = X + (int64_t)s * (g.M + 1) + f;
        const float2 v = *x;
        const float S = (v.x * v.x + v.y * v.y) * g.inv_sumw2;
        const int64_t j = seg_first + s;
        const float Pn = P + (S - P) / (float)(j + 1 < n_avg ? j + 1 : n_avg);
        const float Pw = j == 0 ? Pn : P;
        const float r = Pw > 0.0f ? rsqrtf(Pw) : 0.0f;
        *x = make_float2(v.x * r, v.y * r);
        P = Pn;
    }
    psd[f] = P;
}

// Inverse: Y[s] (M + 1 bins) -> z[s][0 .. N).
__global__ void __launch_bounds__(kCondThreads) cond_inverse_kernel(const float2 *__restrict__ Y, CondGeom g,
                                                                     const float2 *__restrict__ tw,
                                                                     const float2 *__restrict__ rtw,
                                                                     float *__restrict__ z) {
    extern __shared__ float2 sm[];
    float2 *a = sm, *b = sm + g.M;
    const float2 *y = Y + (int64_t)blockIdx.x * (g.M + 1);
    // Ze = (X[f] + conj X[M-f]) / 2, Zo = (X[f] - conj X[M-f]) W^{-f} / 2, Z = Ze + i Zo
    for (int f = threadIdx.x; f < g.M; f += blockDim.x) {
        const float2 xf = y[f], xc = conjf2(y[g.M - f]);
        const float2 e = make_float2(0.5f * (xf.x + xc.x), 0.5f * (xf.y + xc.y));
        const float2 o = cmul(make_float2(0.5f * (xf.x - xc.x), 0.5f * (xf.y - xc.y)), conjf2(__ldg(&rtw[f])));
        a[f] = make_float2(e.x - o.y, e.y + o.x);
    }
    __syncthreads();
    const float2 *Z = fft_stockham<true>(a, b, g.M, g.logM, tw);
    float *out = z + (int64_t)blockIdx.x * g.N;
    const float inv_m = 1.0f / (float)g.M;
    for (int m = threadIdx.x; m < g.M; m += blockDim.x) {
        out[2 * m] = Z[m].x * inv_m;
        out[2 * m + 1] = Z[m].y * inv_m;
    }
}

// Overlap-add into the whitened ring and the glitch list.
// ring_new[k], k < 2G: ring_old[k + n_prev] (the previous push's last 2G whitened samples);
// ring_new[2G + i], i < n: whitened sample s = T - H + i: z of segment a = floor(s / H) (first half)
// plus z of segment a - 1 (second half; from carry when it is the previous push's last segment).
// Every ring sample with |x| > thr is appended (absolute index) to cent.
struct CombineArgs {
    const float *ring_old;
    float *ring_new;
    const float *z;             // this push's segments [seg_first, seg_first + n_seg), N floats each
    const float *carry_old;     // second half of segment seg_first - 1 (H floats)
    float *carry_new;           // second half of this push's last segment
    int64_t T;                  // samples pushed before this push
    int64_t seg_first;
    int n_seg, n, n_prev, G;
    float thr;
    int64_t *cent;
    int *n_cent;
};
__global__ void __launch_bounds__(256) cond_combine_kernel(CombineArgs c, CondGeom g) {
    const int64_t ring_len = 2 * (int64_t)c.G + c.n;
    const int64_t ring0 = c.T - g.H - 2 * (int64_t)c.G;           // absolute sample of ring index 0
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ring_len;
         k += (int64_t)gridDim.x * blockDim.x) {
        float v;
        if (k < 2 * c.G) {
            v = c.ring_old[k + c.n_prev];
        } else {
            const int64_t s = ring0 + k;
            v = 0.0f;
            if (s >= 0) {
                const int64_t a = s / g.H;
                const int64_t r = s - a * g.H;
                v = c.z[(a - c.seg_first) * g.N + r];
                if (a - 1 >= c.seg_first) v += c.z[(a - 1 - c.seg_first) * g.N + g.H + r];
                else if (a - 1 >= 0) v += c.carry_old[r];
            }
        }
        c.ring_new[k] = v;
        if (c.thr > 0.0f && fabsf(v) > c.thr) {
            const int slot = atomicAdd(c.n_cent, 1);
            c.cent[slot] = ring0 + k;                              // slots <= ring length: no overflow
        }
    }
    if (c.n_seg > 0)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < g.H; r += (int64_t)gridDim.x * blockDim.x)
            c.carry_new[r] = c.z[(int64_t)(c.n_seg - 1) * g.N + g.H + r];
}

// Gate: out[i] = x(m) g(r(m)), m = T - latency + i, r = distance to the nearest glitch sample.
__global__ void __launch_bounds__(256) cond_gate_kernel(const float *__restrict__ ring, int64_t ring0, int64_t m0,
                                                        int n, const int64_t *__restrict__ cent,
                                                        const int *__restrict__ n_cent, int half, int taper,
                                                        float *__restrict__ out) {
    const int nc = *n_cent;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = m0 + i;
        float v = ring[m - ring0];
        if (nc > 0) {
            int64_t r = INT64_MAX;
            for (int q = 0; q < nc; ++q) {
                const int64_t d = cent[q] > m ? cent[q] - m : m - cent[q];
                r = d < r ? d : r;
            }
            if (r <= half) {
                v = 0.0f;
            } else if (r < (int64_t)half + taper) {
                const float sr = sinpif(0.5f * (float)(r - half) / (float)taper);
                v *= sr * sr;
            }
        }
        out[i] = v;
    }
}

}  // namespace lloid

using namespace lloid;

void set_last_error(const std::string &msg);
int lloid_ctx_stream(sb_ctx *c, cudaStream_t *stream, int *device);

struct sb_cond {
    sb_ctx *ctx = nullptr;
    CondGeom g{};
    int n_avg = 1, half = 0, taper = 1, G = 0;
    float thr = 0.0f;
    int64_t Bmax = 0, T = 0, seg_done = 0, n_prev = 0;
    int cur = 0;                       // ping-pong index of the raw / ring / carry buffers
    float *raw[2] = {nullptr, nullptr};        // [H + Bmax]: samples [T - H, T + n)
    float *ring[2] = {nullptr, nullptr};       // [2G + Bmax]: whitened samples [T - H - 2G, T + n - H)
    float *carry[2] = {nullptr, nullptr};      // [H]
    float *psd = nullptr;                      // [M + 1]
    float2 *X = nullptr;                       // [Bmax / H][M + 1]
    float *Z = nullptr;                        // [Bmax / H][N]
    float2 *tw = nullptr, *rtw = nullptr;      // [M / 2], [M + 1]
    int64_t *cent = nullptr;                   // [2G + Bmax]
    int *n_cent = nullptr;
    std::vector<void *> allocs;
};

static int cond_fail(int code, const std::string &msg) {
    set_last_error(msg);
    return code;
}

template <class K>
static cudaError_t cond_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const std::pair<const void *, int> id(reinterpret_cast<const void *>(kernel), dev);
    if (done.count(id)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * (kCondMaxN / 2) * sizeof(float2)));
    if (e == cudaSuccess) done.insert(id);
    return e;
}

extern "C" int sb_cond_create(sb_ctx *ctx, const sb_cond_desc *d, sb_cond **out) {
    if (!ctx || !d || !out) return cond_fail(SB_EINVAL, "sb_cond_create: null argument");
    *out = nullptr;
    const int N = d->fft_len;
    if (N < kCondMinN || N > kCondMaxN || (N & (N - 1)))
        return cond_fail(SB_EINVAL, "sb_cond_create: fft_len must be a power of two in [64, 16384]");
    if (!(d->rate_hz > 0) || d->n_avg < 1 || d->gate_half < 0 || d->gate_taper < 1 || d->max_push_samples <= 0 ||
        d->max_push_samples % (N / 2) || d->max_push_samples > (int64_t(1) << 30))
        return cond_fail(SB_EINVAL, "sb_cond_create: bad rate, n_avg, gate lengths or max_push_samples (a positive "
                                    "multiple of fft_len / 2, at most 2^30)");
    cudaStream_t st = nullptr;
    int device = 0;
    int rc = lloid_ctx_stream(ctx, &st, &device);
    if (rc) return rc;
    sb_cond *c = new sb_cond();
    c->ctx = ctx;
    c->g.N = N;
    c->g.M = N / 2;
    c->g.H = N / 2;
    int logM = 0;
    while ((1 << logM) < c->g.M) ++logM;
    c->g.logM = logM;
    c->g.inv_sumw2 = (float)(8.0 / (3.0 * N));
    c->n_avg = d->n_avg;
    c->thr = d->gate_threshold;
    c->half = d->gate_half;
    c->taper = d->gate_taper;
    c->G = d->gate_half + d->gate_taper;
    c->Bmax = d->max_push_samples;
    const int64_t H = c->g.H, M = c->g.M, max_seg = c->Bmax / H;
    auto alloc = [&](void **p, size_t bytes) {
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) return false;
        c->allocs.push_back(*p);
        return cudaMemsetAsync(*p, 0, bytes, st) == cudaSuccess;
    };
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = alloc((void **)&c->raw[b], (H + c->Bmax) * 4) && alloc((void **)&c->ring[b], (2 * c->G + c->Bmax) * 4) &&
             alloc((void **)&c->carry[b], H * 4);
    }
    ok = ok && alloc((void **)&c->psd, (M + 1) * 4) && alloc((void **)&c->X, max_seg * (M + 1) * sizeof(float2)) &&
         alloc((void **)&c->Z, max_seg * (int64_t)N * 4) && alloc((void **)&c->tw, (M / 2) * sizeof(float2)) &&
         alloc((void **)&c->rtw, (M + 1) * sizeof(float2)) && alloc((void **)&c->cent, (2 * c->G + c->Bmax) * 8) &&
         alloc((void **)&c->n_cent, 4);
    if (ok) {                                      // twiddles e^{-2 pi i t / M} and e^{-2 pi i f / N}, in FP64
        std::vector<float2> tw(M / 2), rtw(M + 1);
        for (int64_t t = 0; t < M / 2; ++t)
            tw[t] = make_float2((float)std::cos(2.0 * M_PI * t / M), (float)-std::sin(2.0 * M_PI * t / M));
        for (int64_t f = 0; f <= M; ++f)
            rtw[f] = make_float2((float)std::cos(2.0 * M_PI * f / N), (float)-std::sin(2.0 * M_PI * f / N));
        ok = cudaMemcpyAsync(c->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st) ==
                 cudaSuccess &&
             cudaMemcpyAsync(c->rtw, rtw.data(), rtw.size() * sizeof(float2), cudaMemcpyHostToDevice, st) ==
                 cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
    }
    if (!ok) {
        for (void *p : c->allocs) cudaFree(p);
        delete c;
        cudaGetLastError();
        return cond_fail(SB_ENOMEM, "sb_cond_create: device allocation failed");
    }
    *out = c;
    return SB_OK;
}

extern "C" int sb_cond_destroy(sb_cond *c) {
    if (!c) return SB_OK;
    cudaStream_t st = nullptr;
    int device = 0;
    if (lloid_ctx_stream(c->ctx, &st, &device) == SB_OK) cudaStreamSynchronize(st);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
    return SB_OK;
}

extern "C" int sb_cond_latency(const sb_cond *c, int64_t *latency) {
    if (!c || !latency) return cond_fail(SB_EINVAL, "sb_cond_latency: null argument");
    *latency = c->g.H + c->G;
    return SB_OK;
}

extern "C" int sb_cond_push(sb_cond *c, const float *strain, int64_t n, int64_t t0, int32_t on_device, float *out) {
    if (!c || !strain || !out) return cond_fail(SB_EINVAL, "sb_cond_push: null argument");
    if (t0 != c->T) return cond_fail(SB_EGAP, "sb_cond_push: t0 is not contiguous with the samples pushed so far");
    if (n <= 0 || n > c->Bmax || n % c->g.H)
        return cond_fail(SB_EINVAL, "sb_cond_push: n_samples must be a positive multiple of fft_len / 2, at most "
                                    "max_push_samples");
    cudaStream_t st = nullptr;
    int device = 0;
    int rc = lloid_ctx_stream(c->ctx, &st, &device);
    if (rc) return rc;
    const int H = c->g.H, M = c->g.M;
    const int o = c->cur, nb = 1 - c->cur;
    cudaError_t e = cudaSuccess;
    auto launch_ok = [&]() {
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess;
    };
    // raw ring: [T - H, T) from the previous ring's tail, then this push's samples
    e = cudaMemcpyAsync(c->raw[nb], c->raw[o] + c->n_prev, (size_t)H * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->raw[nb] + H, strain, (size_t)n * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    // segments j with j H + N <= T + n that are not done yet: j in [seg_done, (T + n) / H - 2]
    const int64_t seg_last = (c->T + n) / H - 2;
    const int n_seg = (int)std::max<int64_t>(0, seg_last - c->seg_done + 1);
    const size_t smem = 2 * (size_t)M * sizeof(float2);
    if (e == cudaSuccess && n_seg > 0) {
        if ((e = cond_smem(cond_forward_kernel, smem)) == cudaSuccess &&
            (e = cond_smem(cond_inverse_kernel, smem)) == cudaSuccess) {
            const int64_t seg0_off = c->seg_done * H - (c->T - H);         // raw index of the first segment
            cond_forward_kernel<<<n_seg, kCondThreads, smem, st>>>(c->raw[nb], seg0_off, c->g, c->tw, c->rtw, c->X);
            if (launch_ok())
                cond_psd_kernel<<<(M + 1 + 255) / 256, 256, 0, st>>>(c->X, c->psd, n_seg, c->seg_done, c->n_avg, c->g);
            if (launch_ok())
                cond_inverse_kernel<<<n_seg, kCondThreads, smem, st>>>(c->X, c->g, c->tw, c->rtw, c->Z);
            launch_ok();
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->n_cent, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        CombineArgs a{};
        a.ring_old = c->ring[o];
        a.ring_new = c->ring[nb];
        a.z = c->Z;
        a.carry_old = c->carry[o];
        a.carry_new = c->carry[nb];
        a.T = c->T;
        a.seg_first = c->seg_done;
        a.n_seg = n_seg;
        a.n = (int)n;
        a.n_prev = (int)c->n_prev;
        a.G = c->G;
        a.thr = c->thr;
        a.cent = c->cent;
        a.n_cent = c->n_cent;
        const int64_t work = 2 * (int64_t)c->G + n;
        const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 8);
        cond_combine_kernel<<<blocks, 256, 0, st>>>(a, c->g);
        if (launch_ok()) {
            const int64_t ring0 = c->T - H - 2 * (int64_t)c->G;
            const int64_t m0 = c->T - (H + c->G);
            cond_gate_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 148 * 8), 256, 0, st>>>(
                c->ring[nb], ring0, m0, (int)n, c->cent, c->n_cent, c->half, c->taper, out);
            launch_ok();
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cond_fail(SB_ECUDA, std::string("sb_cond_push: ") + cudaGetErrorString(e));
    }
    c->T += n;
    c->seg_done += n_seg;
    c->n_prev = n;
    if (n_seg == 0) {
        // no segment completed (the first push of H samples): the carry stays zero, keep it in place
        cudaMemcpyAsync(c->carry[nb], c->carry[o], (size_t)H * 4, cudaMemcpyDeviceToDevice, st);
    }
    c->cur = nb;
    return SB_OK;
}

extern "C" int sb_cond_psd(sb_cond *c, float *host_out, int64_t cap, int64_t *n_bins, int64_t *segments) {
    if (!c || !n_bins || !segments) return cond_fail(SB_EINVAL, "sb_cond_psd: null argument");
    *n_bins = c->g.M + 1;
    *segments = c->seg_done;
    if (cap <= 0) return SB_OK;
    if (!host_out || cap < c->g.M + 1) return cond_fail(SB_EINVAL, "sb_cond_psd: output holds fewer than fft_len/2+1");
    cudaStream_t st = nullptr;
    int device = 0;
    int rc = lloid_ctx_stream(c->ctx, &st, &device);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(host_out, c->psd, (size_t)(c->g.M + 1) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cond_fail(SB_ECUDA, std::string("sb_cond_psd: ") + cudaGetErrorString(e));
    return SB_OK;
}
