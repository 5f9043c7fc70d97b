// a6: FP32 refinement of candidate window maxima in the 16-bit and 8-bit modes.
//
// After the top level's partial maxima are known, every partial record whose
// |rho| exceeds the refine threshold and comes within a margin of its window's
// 16-bit maximum (so that it may be that window's maximum once refined) is
// recomputed in FP32 over the top-level samples within R = 8 of its maximum
// (clipped to the record's half tile and window).  The SVD factorisation pays
// off when all M templates are filtered; for a handful of candidates it does
// not, so the refinement filters the
// strain directly with each template's reconstructed slice filters
// H_s = M_s V_s (step a3's mixing summed over the basis, FP32, built once per bank):
//   z_k[row][m] = sum_{slices s at level k} sum_q H_s[2i+row][q] d_k[m - D_s - q]
// plus the x2 interpolation of z_{k+1} (step a4), level by level from the coarsest.
// That is the same sum as the basis path in exact arithmetic; per candidate it
// costs 2 x sum_s Q_s x (<= 64) multiply-adds instead of a full basis output.
//
// Level ranges (absolute indices): the top level covers [lo_0, hi_0]; level
// k+1 needs [ceil((lo_k - 31)/2), floor((hi_k + 31)/2)] for the interpolation,
// at most kRefSpan = 64 samples for 2R + 1 = 17.
#include <algorithm>

#include "lloid_internal.h"

namespace lloid {

__device__ __forceinline__ int64_t floor_div2(int64_t v) { return v >> 1; }
__device__ __forceinline__ int64_t ceil_div2(int64_t v) { return -((-v) >> 1); }

// R1: records above the threshold and within the margin of their window's maximum become
// candidates.  The maxima (|rho|^2 bits, which order like the non-negative floats) are
// gathered per (template, window) by the top level's mixing epilogue.
__global__ void __launch_bounds__(256) refine_flag_kernel(const RefUnit *__restrict__ units,
                                                          RefCand *__restrict__ cands, int *__restrict__ counters,
                                                          int cand_cap) {
    griddep_wait();
    const RefUnit &u = units[blockIdx.y];
    // one thread per (template, window of this push) reads the window's maximum; a window without a
    // record above the refine threshold has a zero maximum and no candidate.  The warp then scans
    // the records of its few windows with a maximum together, one window after the other.
    const int64_t nw = (int64_t)u.M * u.n_wslot;
    const int64_t gw0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31;
    const int lane = threadIdx.x & 31;
    if (gw0 >= nw) return;                         // warp-uniform
    const uint32_t mine = gw0 + lane < nw ? u.wmax[gw0 + lane] : 0u;
    uint32_t todo = __ballot_sync(0xffffffffu, mine != 0u);
    const int64_t start = max(u.first_n, (int64_t)0), end = u.first_n + u.B;
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float wm = __uint_as_float(__shfl_sync(0xffffffffu, mine, src));
        const int64_t gw = gw0 + src;
        const int i = (int)(gw / u.n_wslot), sl = (int)(gw % u.n_wslot);
        const int64_t w = u.win0 + sl;
        const int64_t lo = max(w * u.win_len, start) - u.first_n, hi = min((w + 1) * u.win_len, end) - u.first_n;
        const int r0 = (int)(lo / 128) * 2, r1 = min((int)((hi - 1) / 128) * 2 + 2, u.n_rec);
        for (int r = r0 + lane; r < r1; r += 32) {
            const int64_t idx = (int64_t)i * u.n_rec + r;
            const WinPart p = u.part[idx];
            if (!(p.mag2 > u.thr2) || (u.first_n + p.nr) / u.win_len != w) continue;
            if (p.mag2 < u.keep2 * wm) continue;
            const int slot = atomicAdd(&counters[1], 1);
            if (slot < cand_cap) cands[slot] = RefCand{(int)blockIdx.y, idx};
            else atomicExch(&counters[2], 1);      // not every candidate could be refined
        }
    }
}

// R2: the FP32 FIR of the candidates, split into work items of kRefQC filter taps of one slice,
// one block (8 warps) per (candidate, work item), so that a candidate's slices and the chunks of
// its long slices run in parallel.  A work item's two filter rows and the strain they meet are
// staged in shared memory by coalesced loads of the whole block (one candidate's taps are a few
// hundred kB spread over HBM; staging turns them into streaming reads).  Every warp takes a
// contiguous share of the item's taps; lane l accumulates both rows for m = lo + 2l and
// m = lo + 2l + 1 (as q steps by one, the second output's strain sample is the first's previous
// one, so one read per tap); the warps' partial sums are added in a fixed order, and the work
// items of a level in item order.
constexpr int kRefWarps = 8;

struct RefShared {
    float z[2][2][kRefSpan];                             // ping-pong levels [buf][row][m - lo_k]
    float part[kRefWarps][2][kRefSpan];                  // per-warp partial FIR sums
    __align__(16) float hs[2 * kRefQC];                  // staged filter rows, interleaved: (cos, sin) of tap q
    __align__(16) float xs[kRefQC + kRefSpan + 8];       // staged strain
};

// Level ranges (absolute indices) of one candidate: the top level covers [lo_0, hi_0] (the search
// range widened by kXiJ for the sub-sample peak's neighbours and the xi^2 lags, inside the samples
// this push produces and n >= 0; the strain history reaches 128 samples below the push at every
// level, which covers it), level k + 1 the interpolation's inputs.  Returns false when the record's
// search range is empty.
struct RefRange {
    int64_t slo, shi, lo[kRefMaxLevels], hi[kRefMaxLevels];
    int i;
};
__device__ __forceinline__ bool ref_range(const RefUnit &u, int64_t idx, RefRange &r) {
    const WinPart rec = u.part[idx];
    r.i = (int)(idx / u.n_rec);
    const int rr = (int)(idx % u.n_rec);
    const int tt = rr / 4, h = (rr / 2) % 2;
    const int64_t rn = u.first_n + rec.nr;              // absolute sample of the 16-bit maximum
    const int64_t w = rn / u.win_len;
    const int64_t half0 = u.first_n + (int64_t)kRefTile * tt + 128 * h;
    r.slo = max(rn - kRefR, max(half0, w * u.win_len));
    r.shi = min(min(rn + kRefR, half0 + 127), min((w + 1) * u.win_len, u.first_n + u.B) - 1);
    if (r.shi < r.slo) return false;
    r.lo[0] = max(r.slo - kXiJ, (int64_t)0);
    r.hi[0] = min(r.shi + kXiJ, u.first_n + u.B - 1);
    for (int k = 0; k < u.kmax; ++k) {
        r.lo[k + 1] = ceil_div2(r.lo[k] - (2 * kHalfK - 1));
        r.hi[k + 1] = floor_div2(r.hi[k] + (2 * kHalfK - 1));
    }
    return true;
}

// FP32 FIR of taps [qb, qb + kRefQC) of slice s for template row pair i over [lo, lo + kRefSpan) of its
// level: returns this thread's sums a0 / a1 (output lo + 2 lane, rows 0 / 1) and b0 / b1 (output
// lo + 2 lane + 1).
__device__ __forceinline__ void ref_chunk_fir(const RefUnit &u, int s, int i, int64_t lo, int qb, RefShared &sh,
                                              float &a0, float &a1, float &b0, float &b1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = u.sl_level[s];
    const float *d = u.lv_d[k];
    const int64_t dlen = u.lv_len[k];
    const float *H0 = u.sl_H[s] + (int64_t)(2 * i) * u.sl_ldh[s];
    const float *H1 = H0 + u.sl_ldh[s];
    const int64_t p0 = lo - u.sl_D[s] - u.lv_origin[k];     // d position of output lo + mi at tap q: p0 + mi - q
    const int qn = min(kRefQC, u.sl_Q[s] - qb);
    a0 = a1 = b0 = b1 = 0.0f;
    // strain positions the item reads: [p0 - (qb + qn - 1), p0 + 63 - qb], from a 16-byte boundary
    const int64_t plo = p0 - (qb + qn - 1);
    const int64_t base = plo - (((plo % 4) + 4) % 4);
    const int nx = (int)(p0 + kRefSpan - qb - base);
    const int nx4 = (nx + 3) & ~3;
    __syncthreads();                                           // the previous item's readers are done
    for (int v = threadIdx.x; v < (qn + 3) / 4; v += blockDim.x) {   // rows padded to 4 floats
        const float4 c = __ldg(reinterpret_cast<const float4 *>(H0 + qb) + v);
        const float4 t = __ldg(reinterpret_cast<const float4 *>(H1 + qb) + v);
        reinterpret_cast<float4 *>(sh.hs)[2 * v] = make_float4(c.x, t.x, c.y, t.y);
        reinterpret_cast<float4 *>(sh.hs)[2 * v + 1] = make_float4(c.z, t.z, c.w, t.w);
    }
    if (base >= 0 && base + nx4 <= dlen) {
        for (int v = threadIdx.x; v < nx4 / 4; v += blockDim.x)
            reinterpret_cast<float4 *>(sh.xs)[v] = __ldg(reinterpret_cast<const float4 *>(d + base) + v);
    } else {                                                   // buffer edge: zero outside
        for (int v = threadIdx.x; v < nx4; v += blockDim.x) {
            const int64_t pp = base + v;
            sh.xs[v] = (pp >= 0 && pp < dlen) ? d[pp] : 0.0f;
        }
    }
    __syncthreads();
    const int qcw = ((qn + kRefWarps - 1) / kRefWarps + 3) & ~3;   // taps per warp
    const int q0 = warp * qcw, q1 = min(qn, q0 + qcw);
    if (q0 < q1) {
        const int xa0 = (int)(p0 - base - qb) + 2 * lane;        // x index of output 2 lane at tap 0
        float xb = sh.xs[xa0 + 1 - q0];
        int q = q0;                                              // even: both taps' rows in one float4
        for (; q + 1 < q1; q += 2) {
            const float4 h = reinterpret_cast<const float4 *>(sh.hs)[q >> 1];
            const float xa = sh.xs[xa0 - q], xc = sh.xs[xa0 - q - 1];
            a0 = fmaf(h.x, xa, a0);
            a1 = fmaf(h.y, xa, a1);
            b0 = fmaf(h.x, xb, b0);
            b1 = fmaf(h.y, xb, b1);
            a0 = fmaf(h.z, xc, a0);
            a1 = fmaf(h.w, xc, a1);
            b0 = fmaf(h.z, xa, b0);
            b1 = fmaf(h.w, xa, b1);
            xb = xc;
        }
        if (q < q1) {
            const float xa = sh.xs[xa0 - q];
            a0 = fmaf(sh.hs[2 * q], xa, a0);
            a1 = fmaf(sh.hs[2 * q + 1], xa, a1);
            b0 = fmaf(sh.hs[2 * q], xb, b0);
            b1 = fmaf(sh.hs[2 * q + 1], xb, b1);
        }
    }
}

// The warps' partial sums of one thread block, added in warp order: out[row][mi] for mi < kRefSpan.
__device__ __forceinline__ void ref_block_sum(RefShared &sh, float a0, float a1, float b0, float b1, float *out0,
                                              float *out1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    sh.part[warp][0][2 * lane] = a0;
    sh.part[warp][1][2 * lane] = a1;
    sh.part[warp][0][2 * lane + 1] = b0;
    sh.part[warp][1][2 * lane + 1] = b1;
    __syncthreads();
    if (threadIdx.x < 2 * kRefSpan) {
        const int row = threadIdx.x / kRefSpan, mi = threadIdx.x % kRefSpan;
        float v = 0.0f;
        for (int wp = 0; wp < kRefWarps; ++wp) v += sh.part[wp][row][mi];
        (row == 0 ? out0 : out1)[mi] = v;
    }
}

// R2a: FIR work items of the first kRefSplitCap candidates, block (x, j) takes item j of candidates
// x, x + gridDim.x, ...; out: zpart[cand][item][row][kRefSpan] (zstride items per candidate).
__global__ void __launch_bounds__(kRefWarps * 32) refine_fir_kernel(const RefUnit *__restrict__ units,
                                                                    const int *__restrict__ counters,
                                                                    const RefCand *__restrict__ cands,
                                                                    int cand_cap, float *__restrict__ zpart,
                                                                    int zstride) {
    __shared__ RefShared sh;
    griddep_wait();
    const int n_cand = min(min(counters[1], cand_cap), kRefSplitCap);
    const int j = blockIdx.y;
    for (int ci = blockIdx.x; ci < n_cand; ci += gridDim.x) {
        const RefCand cand = cands[ci];
        const RefUnit &u = units[cand.unit];
        if (j >= u.sl_item0[u.n_slices]) continue;      // block-uniform
        int s = 0;
        while (u.sl_item0[s + 1] <= j) ++s;
        RefRange r;
        if (!ref_range(u, cand.idx, r)) continue;
        float a0, a1, b0, b1;
        ref_chunk_fir(u, s, r.i, r.lo[u.sl_level[s]], (j - u.sl_item0[s]) * kRefQC, sh, a0, a1, b0, b1);
        float *zp = zpart + ((int64_t)ci * zstride + j) * 2 * kRefSpan;
        ref_block_sum(sh, a0, a1, b0, b1, zp, zp + kRefSpan);
    }
}

// R2b: one block per candidate, level by level from the coarsest: the level's FIR work items (from
// zpart for the first kRefSplitCap candidates, computed here for any beyond) plus the x2
// interpolation of the coarser level; then the search, the sub-sample peak and xi^2.
__global__ void __launch_bounds__(kRefWarps * 32) refine_candidate_kernel(const RefUnit *__restrict__ units,
                                                                          const int *__restrict__ counters,
                                                                          const RefCand *__restrict__ cands,
                                                                          int cand_cap, unsigned long long *cum,
                                                                          const float *__restrict__ zpart,
                                                                          int zstride, Halfband g) {
    __shared__ RefShared sh;
    __shared__ float fir[2][kRefSpan];                  // the level's summed slice FIRs
    __shared__ float tmp[2][kRefSpan];                  // one work item's FIR (candidates past kRefSplitCap)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    griddep_wait();
    const int n_cand = min(counters[1], cand_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&cum[0], (unsigned long long)n_cand);
        if (counters[2]) atomicAdd(&cum[1], 1ull);
    }
    for (int ci = blockIdx.x; ci < n_cand; ci += gridDim.x) {
        const RefCand cand = cands[ci];
        const RefUnit &u = units[cand.unit];
        const int64_t idx = cand.idx;
        WinPart rec = u.part[idx];
        RefRange r;
        if (!ref_range(u, idx, r)) continue;            // block-uniform
        const int i = r.i;
        const int64_t slo = r.slo, shi = r.shi;
        const int64_t *lo = r.lo, *hi = r.hi;
        // this candidate's work-item sums, staged in shared memory at once (one latency, not one per item)
        const int n_items = u.sl_item0[u.n_slices];
        const bool staged = ci < kRefSplitCap && n_items * 2 * kRefSpan <= 2 * kRefQC;
        const float *zc_ = zpart + (int64_t)ci * zstride * 2 * kRefSpan;
        if (staged) {
            __syncthreads();                            // the previous candidate's readers are done
            for (int v = threadIdx.x; v < n_items * 2 * kRefSpan / 4; v += blockDim.x)
                reinterpret_cast<float4 *>(sh.hs)[v] = reinterpret_cast<const float4 *>(zc_)[v];
        }
        int cur = 0;                                    // sh.z[cur]: level k + 1
        for (int k = u.kmax; k >= 0; --k) {
            // the level's work items added in item order: read from refine_fir_kernel's output for the
            // first kRefSplitCap candidates, computed here the same way for any beyond, so that a
            // record's value does not depend on its place in the candidate list
            __syncthreads();
            if (threadIdx.x < 2 * kRefSpan) fir[threadIdx.x / kRefSpan][threadIdx.x % kRefSpan] = 0.0f;
            for (int s = 0; s < u.n_slices; ++s) {
                if (u.sl_level[s] != k) continue;
                for (int j = u.sl_item0[s]; j < u.sl_item0[s + 1]; ++j) {
                    if (ci < kRefSplitCap) {
                        if (threadIdx.x < 2 * kRefSpan)
                            fir[threadIdx.x / kRefSpan][threadIdx.x % kRefSpan] +=
                                staged ? sh.hs[j * 2 * kRefSpan + threadIdx.x] : zc_[j * 2 * kRefSpan + threadIdx.x];
                    } else {
                        float a0, a1, b0, b1;
                        ref_chunk_fir(u, s, i, lo[k], (j - u.sl_item0[s]) * kRefQC, sh, a0, a1, b0, b1);
                        ref_block_sum(sh, a0, a1, b0, b1, tmp[0], tmp[1]);
                        __syncthreads();
                        if (threadIdx.x < 2 * kRefSpan)
                            fir[threadIdx.x / kRefSpan][threadIdx.x % kRefSpan] +=
                                tmp[threadIdx.x / kRefSpan][threadIdx.x % kRefSpan];
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x < 2 * kRefSpan) {
                const int row = threadIdx.x / kRefSpan, mi = threadIdx.x % kRefSpan;
                const int64_t m = lo[k] + mi;
                float v = 0.0f;
                if (m <= hi[k] && m >= 0) {
                    v = fir[row][mi];
                    if (k < u.kmax) {                    // x2 interpolation of level k + 1
                        const float *zp = sh.z[cur][row];
                        const int64_t base = lo[k + 1];
                        if ((m & 1) == 0) {
                            v += zp[(m >> 1) - base];
                        } else {
                            const int64_t mlo = (m - 1) >> 1;
                            float acc = 0.0f;
#pragma unroll
                            for (int q = 0; q < kOddTaps; ++q)
                                acc = fmaf(2.0f * g.odd[q], zp[mlo - q - base] + zp[mlo + 1 + q - base], acc);
                            v += acc;
                        }
                    }
                }
                sh.z[cur ^ 1][row][mi] = v;
            }
            __syncthreads();
            cur ^= 1;
        }
        // sh.z[cur] holds level 0 over [lo_0, hi_0] (<= 2R + 1 + 2 kXiJ samples): maximum over
        // [slo, shi] (<= 2R + 1 <= 32 columns, lane l takes column c0 + l), first on ties; then the
        // sub-sample peak from its neighbours and xi^2 over the lags around it
        if (warp == 0) {
            const float *zc = sh.z[cur][0], *zs = sh.z[cur][1];
            const int len0 = (int)(hi[0] - lo[0] + 1), c0 = (int)(slo - lo[0]), c1 = (int)(shi - lo[0]);
            float best = -1.0f;
            int bc = -1;
            if (c0 + lane <= c1) {
                bc = c0 + lane;
                best = fmaf(zs[bc], zs[bc], zc[bc] * zc[bc]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                if (ob > best || (ob == best && oc >= 0 && (bc < 0 || oc < bc))) {
                    best = ob;
                    bc = oc;
                }
            }
            // xi^2 (every lane holds bc): all lags inside the computed range and n >= 0
            float xi = 0.0f;
            const bool has_xi = u.acorr && bc >= kXiJ && bc + kXiJ < len0 && lo[0] + bc - kXiJ >= 0;
            if (has_xi) {
                const float z0c = zc[bc], z0s = zs[bc];
                const float2 *Ri = u.acorr + (int64_t)i * kXiLags;
                float num = 0.0f, den = 0.0f;
                for (int j = lane; j < kXiLags; j += 32) {
                    const float2 r = Ri[j];
                    const float ec = zc[bc - kXiJ + j] - (z0c * r.x - z0s * r.y);
                    const float es = zs[bc - kXiJ + j] - (z0c * r.y + z0s * r.x);
                    num += fmaf(es, es, ec * ec);
                    den += 2.0f - 2.0f * fmaf(r.y, r.y, r.x * r.x);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    num += __shfl_xor_sync(0xffffffffu, num, off);
                    den += __shfl_xor_sync(0xffffffffu, den, off);
                }
                xi = num / den;
            }
            if (lane == 0 && bc >= 0) {
                rec.mag2 = best;
                rec.re = zc[bc];
                rec.im = zs[bc];
                rec.nr = (int32_t)(lo[0] + bc - u.first_n);
                rec.flags = SB_TRIG_REFINED_BIT;
                rec.pk = rec.dt = rec.xi2 = 0.0f;
                if (bc >= 1 && bc + 1 < len0) {
                    const float ym = fmaf(zs[bc - 1], zs[bc - 1], zc[bc - 1] * zc[bc - 1]);
                    const float yp = fmaf(zs[bc + 1], zs[bc + 1], zc[bc + 1] * zc[bc + 1]);
                    if (subsample_peak(ym, best, yp, rec.pk, rec.dt)) rec.flags |= SB_TRIG_SUBSAMPLE_BIT;
                }
                if (has_xi) {
                    rec.xi2 = xi;
                    rec.flags |= SB_TRIG_XI2_BIT;
                }
                u.part[idx] = rec;
            }
        }
        __syncthreads();                                // z is reused by the next candidate
    }
}

cudaError_t launch_refine(const RefUnit *d_units, int n_units, int64_t max_windows, RefCand *cands, int *counters,
                          unsigned long long *cum, float *zpart, int max_items, const Halfband &g, cudaStream_t s) {
    if (n_units == 0 || max_windows == 0) return cudaSuccess;
    const int fb = (int)((max_windows + 255) / 256);              // one thread per (template, window)
    // the window maxima were gathered by the top level's mixing epilogue
    cudaError_t e = launch_pdl(refine_flag_kernel, dim3(fb, n_units), dim3(256), 0, s, d_units, cands, counters,
                               kRefCandCap);
    if (e == cudaSuccess)
        // about twice the resident blocks (six per SM by registers) over the work items of one
        // candidate: blocks past the candidates exit at once, the rest fill the SMs as they free up
        e = launch_pdl(refine_fir_kernel, dim3((12 * 148 + max_items - 1) / max_items, max_items),
                       dim3(kRefWarps * 32), 0, s, d_units, (const int *)counters, (const RefCand *)cands,
                       kRefCandCap, zpart, max_items);
    if (e == cudaSuccess)
        e = launch_pdl(refine_candidate_kernel, dim3(8 * 148), dim3(kRefWarps * 32), 0, s, d_units,
                       (const int *)counters, (const RefCand *)cands, kRefCandCap, cum, (const float *)zpart,
                       max_items, g);
    return e;
}

}  // namespace lloid
