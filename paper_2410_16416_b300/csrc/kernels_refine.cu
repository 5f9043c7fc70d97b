// a6: FP32 refinement of candidate window maxima in the 16-bit modes.
//
// After the top level's partial maxima are known, every partial record whose
// |rho| exceeds the refine threshold is recomputed in FP32 over the samples
// within R = 8 of its maximum: for each 256-sample tile holding candidates, the
// union of those neighbourhoods is re-filtered from the FP32 decimated strain
// and the FP32 basis (a tiled FP32 Toeplitz GEMM, shared by every template with
// a candidate in the tile); then each candidate's two real filters are mixed
// with the FP32 coefficients, interpolated level by level in FP32, and the
// maximum is taken again within R of the old one.  The refined records go
// through the usual window bookkeeping and carry SB_TRIG_REFINED.
//
// Level ranges (absolute indices): the top level covers [n_lo, n_hi]; level
// k+1 needs [ceil((lo_k - 31)/2), floor((hi_k + 31)/2)] for the interpolation.
#include <algorithm>

#include "gemm_fp32_tile.cuh"
#include "lloid_internal.h"

namespace lloid {

__device__ __forceinline__ int64_t floor_div2(int64_t v) { return v >> 1; }
__device__ __forceinline__ int64_t ceil_div2(int64_t v) { return -((-v) >> 1); }

// level ranges of the refined neighbourhood of tile tt of unit u
__device__ __forceinline__ void tile_ranges(const RefUnit &u, int tt, const int *tlo, const int *thi, int64_t *lo,
                                            int64_t *hi) {
    lo[0] = u.first_n + tlo[u.flag_off + tt];
    hi[0] = u.first_n + thi[u.flag_off + tt];
    for (int k = 0; k < u.kmax; ++k) {
        lo[k + 1] = ceil_div2(lo[k] - (2 * kHalfK - 1));
        hi[k + 1] = floor_div2(hi[k] + (2 * kHalfK - 1));
    }
}

// R1a: flag tiles that hold a candidate record and widen the tile's column
// range to cover R samples on either side of the candidate's maximum.
__global__ void __launch_bounds__(256) refine_flag_kernel(const RefUnit *__restrict__ units, int n_units,
                                                          int *__restrict__ flags, int *__restrict__ tlo,
                                                          int *__restrict__ thi, RefCand *__restrict__ cands,
                                                          int *__restrict__ counters, int cand_cap) {
    const RefUnit &u = units[blockIdx.y];
    const int64_t total = (int64_t)u.M * u.n_rec;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const WinPart p = u.part[idx];
        if (!(p.mag2 > u.thr2)) continue;
        const int tt = (int)((idx % u.n_rec) / 4);
        const int c = (int)(p.n - u.first_n);
        const int c0 = kRefTile * tt, c1 = min(kRefTile * tt + kRefTile, u.B) - 1;
        flags[u.flag_off + tt] = 1;
        atomicMin(&tlo[u.flag_off + tt], max(c - kRefR, c0));
        atomicMax(&thi[u.flag_off + tt], min(c + kRefR, c1));
        const int slot = atomicAdd(&counters[1], 1);
        if (slot < cand_cap) cands[slot] = RefCand{(int)blockIdx.y, idx};
        else atomicExch(&counters[2], 1);
    }
}

// R1b: one thread per (unit, tile): flagged tiles get a slot (capacity-limited).
__global__ void __launch_bounds__(256) refine_slot_kernel(const RefUnit *__restrict__ units, int n_units,
                                                          int *__restrict__ flags, RefSlot *__restrict__ slots,
                                                          int *__restrict__ counters, int cap) {
    const RefUnit &u = units[blockIdx.y];
    const int tt = blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= u.tiles_t) return;
    int *f = flags + u.flag_off + tt;
    if (*f == 0) { *f = -1; return; }
    const int s = atomicAdd(&counters[0], 1);
    if (s < cap) {
        slots[s] = RefSlot{(int)blockIdx.y, tt};
        *f = s;
    } else {
        *f = -1;
        atomicExch(&counters[2], 1);                // not every candidate could be refined
    }
}

// R2: FP32 basis outputs of one slot's neighbourhood at every level,
// o[l][m - lo_k] (row stride kRefRange(k)), as FP32 Toeplitz GEMM tiles.
// Block (slot, work item = slice x 64 basis vectors x 128 samples).
__global__ void __launch_bounds__(256) refine_fir_kernel(const RefUnit *__restrict__ units,
                                                         const RefSlot *__restrict__ slots,
                                                         const int *__restrict__ counters, const int *__restrict__ tlo,
                                                         const int *__restrict__ thi, float *__restrict__ obuf,
                                                         int64_t slot_floats) {
    const int s = blockIdx.x;
    if (s >= counters[0]) return;
    const RefSlot sl = slots[s];
    const RefUnit &u = units[sl.unit];
    int64_t lo[kRefMaxLevels], hi[kRefMaxLevels];
    tile_ranges(u, sl.tt, tlo, thi, lo, hi);
    int item = blockIdx.y, si = 0, mb = 0, lb = 0;
    for (; si < u.n_slices; ++si) {
        const int k = u.sl_level[si];
        const int nm = (int)((hi[k] - lo[k] + kGemmTN) / kGemmTN), nl = (u.sl_L[si] + kGemmTM - 1) / kGemmTM;
        if (item < nm * nl) { lb = item / nm; mb = item % nm; break; }
        item -= nm * nl;
    }
    if (si >= u.n_slices) return;
    const int k = u.sl_level[si];
    GemmTask t{};
    t.A = u.sl_V[si];
    t.lda = u.sl_Q[si];
    t.B = u.lv_d[k];
    t.ldb = lo[k] - u.sl_D[si] - u.lv_origin[k];      // position of d[m - D - q] is ldb + (m - lo) - q
    t.C = obuf + (int64_t)s * slot_floats + u.lv_off[k] + (int64_t)u.sl_row[si] * kRefRange(k);
    t.ldc = kRefRange(k);
    t.M = u.sl_L[si];
    t.N = (int32_t)(hi[k] - lo[k] + 1);
    t.K = u.sl_Q[si];
    t.beta = 0;
    t.toeplitz = 1;
    gemm_fp32_tile<true>(t, lb * kGemmTM, mb * kGemmTN, u.lv_len[k]);
}

// R3: one block per candidate record: FP32 mixing + interpolation of its two
// real filters over the tile, then the record's maximum is taken again.
__global__ void __launch_bounds__(128) refine_candidate_kernel(const RefUnit *__restrict__ units, int n_units,
                                                               const int *__restrict__ flags,
                                                               const int *__restrict__ tlo, const int *__restrict__ thi,
                                                               const int *__restrict__ counters,
                                                               const RefCand *__restrict__ cands, int cand_cap,
                                                               const float *__restrict__ obuf, int64_t slot_floats,
                                                               Halfband g) {
    __shared__ float ya[2][kRefRange(0)], yb[2][kRefRange(0)];
    __shared__ float red_m[128];
    __shared__ int red_c[128];
    const int n_cand = min(counters[1], cand_cap);
    for (int ci = blockIdx.x; ci < n_cand; ci += gridDim.x) {
        const RefCand cand = cands[ci];
        const RefUnit &u = units[cand.unit];
        const int64_t idx = cand.idx;
        WinPart rec = u.part[idx];
        const int i = (int)(idx / u.n_rec), r = (int)(idx % u.n_rec);
        const int tt = r / 4;
        const int slot = flags[u.flag_off + tt];
        if (slot < 0) continue;
        int64_t lo[kRefMaxLevels], hi[kRefMaxLevels];
        tile_ranges(u, tt, tlo, thi, lo, hi);
        const float *ob = obuf + (int64_t)slot * slot_floats;
        float(*yc)[kRefRange(0)] = ya;      // level k (being built)
        float(*yp)[kRefRange(0)] = yb;      // level k+1
        for (int k = u.kmax; k >= 0; --k) {
            const int len = (int)(hi[k] - lo[k] + 1);
            for (int t = threadIdx.x; t < 2 * len; t += blockDim.x) {
                const int row = t / len, mi = t % len;
                const int64_t m = lo[k] + mi;
                float v = 0.0f;
                if (m >= 0) {
                    if (k < u.kmax) {           // interpolation from level k+1 (absolute index arithmetic)
                        const int64_t base = lo[k + 1];
                        if ((m & 1) == 0) {
                            v = yp[row][(m >> 1) - base];
                        } else {
                            const int64_t mlo = (m - 1) >> 1;
                            float acc = 0.0f;
#pragma unroll
                            for (int q = 0; q < kOddTaps; ++q)
                                acc = fmaf(2.0f * g.odd[q], yp[row][mlo - q - base] + yp[row][mlo + 1 + q - base], acc);
                            v = acc;
                        }
                    }
                    const int Lk = u.lv_Lk[k];
                    if (Lk > 0) {
                        const float *Mrow = u.lv_M[k] + (int64_t)(2 * i + row) * Lk;
                        const float *o = ob + u.lv_off[k] + mi;
                        float c = 0.0f;
                        for (int l = 0; l < Lk; ++l) c = fmaf(Mrow[l], o[(int64_t)l * kRefRange(k)], c);
                        v += c;
                    }
                }
                yc[row][mi] = v;
            }
            __syncthreads();
            float(*tmp)[kRefRange(0)] = yc;
            yc = yp;
            yp = tmp;
        }
        // yp holds level 0 over [lo[0], hi[0]]; the record covers one half and one window
        // search: this record's half and window, within R of its unrefined maximum
        const int h = (r / 2) % 2;
        const int64_t w = rec.n / u.win_len;
        const int64_t cstar = rec.n - lo[0];                       // index in the level-0 range
        const int64_t half0 = u.first_n + (int64_t)kRefTile * tt + 128 * h - lo[0];
        const int c_lo = (int)max(max(cstar - kRefR, half0), (int64_t)0);
        const int c_hi = (int)min(min(cstar + kRefR + 1, half0 + 128), hi[0] - lo[0] + 1);
        float best = -1.0f;
        int bc = -1;
        for (int c = c_lo + threadIdx.x; c < c_hi; c += blockDim.x) {
            const int64_t n = lo[0] + c;
            if (n < 0 || n / u.win_len != w) continue;
            const float m2 = fmaf(yp[1][c], yp[1][c], yp[0][c] * yp[0][c]);
            if (m2 > best) { best = m2; bc = c; }
        }
        red_m[threadIdx.x] = best;
        red_c[threadIdx.x] = bc;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 1; t < blockDim.x; ++t)
                if (red_m[t] > best || (red_m[t] == best && red_c[t] >= 0 && (bc < 0 || red_c[t] < bc))) {
                    best = red_m[t];
                    bc = red_c[t];
                }
            if (bc >= 0) {
                rec.mag2 = best;
                rec.re = yp[0][bc];
                rec.im = yp[1][bc];
                rec.n = lo[0] + bc;
                rec.flags = SB_TRIG_REFINED_BIT;
                u.part[idx] = rec;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_refine(const RefUnit *d_units, int n_units, int max_tiles, int64_t max_tiles_total,
                          int64_t max_records, int *flags, RefSlot *slots, int *counters, int cap, float *obuf,
                          int64_t slot_floats, int max_items, const Halfband &g, cudaStream_t s) {
    if (n_units == 0) return cudaSuccess;
    const int fb = (int)std::min<int64_t>(1024, (max_records + 255) / 256);
    int *tlo = flags + max_tiles_total, *thi = tlo + max_tiles_total;
    // candidate list after the three int arrays, 16-byte aligned (the allocation has 16 bytes of slack)
    RefCand *cands = reinterpret_cast<RefCand *>((reinterpret_cast<uintptr_t>(thi + max_tiles_total) + 15) &
                                                 ~uintptr_t(15));
    refine_flag_kernel<<<dim3(fb, n_units), 256, 0, s>>>(d_units, n_units, flags, tlo, thi, cands, counters,
                                                         kRefCandCap);
    refine_slot_kernel<<<dim3((max_tiles + 255) / 256, n_units), 256, 0, s>>>(d_units, n_units, flags, slots,
                                                                               counters, cap);
    refine_fir_kernel<<<dim3(cap, max_items), 256, 0, s>>>(d_units, slots, counters, tlo, thi, obuf, slot_floats);
    refine_candidate_kernel<<<4 * 148, 128, 0, s>>>(d_units, n_units, flags, tlo, thi, counters, cands,
                                                    kRefCandCap, obuf, slot_floats, g);
    return cudaGetLastError();
}

}  // namespace lloid
