// Tensor-core (tcgen05, sm_103a) kernels of the two GEMM-shaped steps in the
// 16-bit modes (SB_BF16, SB_FP16; FP32 accumulation in TMEM):
//
//  a2 basis FIR as a Hankel GEMM.  Output time m' = 8b + r (b = block of 8
//     samples, r = phase).  With X[b][j] = x[X0 + 8b + j] the FIR is
//         o[l][8b + r] = sum_j W[(l,r)][j] X[b][j],
//         W[(l,r)][j]  = v[l][r + Q - 1 + phi - j]   (0 outside the taps),
//     so the data operand is a Hankel matrix whose rows start 16 bytes apart.
//     A plain no-swizzle UMMA descriptor (core matrices 16 B apart along K,
//     8-row groups 128 B apart) reads it straight from one strain window in
//     shared memory: the strain is loaded once per tile, never expanded.  The
//     8-phase weights W (8 L_s rows) are expanded once at bank creation and
//     streamed by TMA with 128-byte swizzle.
//  a3 mixing GEMM with time on the TMEM lanes: D[m][a] = sum_l O[m][l] M[a][l],
//     so every epilogue store writes 32 consecutive time samples of one filter.
//
// One CTA = 4 warps: warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMAs, then
// all four warps drain TMEM (each warp owns 32 TMEM lanes).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lloid_internal.h"
#include "tc_ptx.cuh"

namespace lloid {

using namespace tc;

// Operand modes: element type, bytes, the Hankel block (phases = 16 bytes of
// samples), K per MMA instruction (32 bytes) and the instruction kind.
template <int MODE>
struct Op;
template <>
struct Op<kModeF16> {
    using T = __half;
    static constexpr int kBytes = 2, kPhases = 8, kMmaK = 16;
    static constexpr uint32_t kFmt = 0;
    static __device__ __forceinline__ T cvt(float v) { return __float2half_rn(v); }
};
template <>
struct Op<kModeBF16> {
    using T = __nv_bfloat16;
    static constexpr int kBytes = 2, kPhases = 8, kMmaK = 16;
    static constexpr uint32_t kFmt = 1;
    static __device__ __forceinline__ T cvt(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Op<kModeE4M3> {
    using T = __nv_fp8_e4m3;
    static constexpr int kBytes = 1, kPhases = 16, kMmaK = 32;
    static constexpr uint32_t kFmt = 0;
    static __device__ __forceinline__ T cvt(float v) { return __nv_fp8_e4m3(v); }   // saturating
};
template <int MODE>
__device__ __forceinline__ void mma_op(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == kModeE4M3) mma_f8(d, a, b, idesc, acc);
    else mma_f16(d, a, b, idesc, acc);
}
template <int MODE>
__host__ __device__ constexpr uint32_t idesc_op(int M, int N) {
    return (1u << 4) | (Op<MODE>::kFmt << 7) | (Op<MODE>::kFmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <class Task>
__device__ __forceinline__ int find_tile(const Task *tasks, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// ---------------------------------------------------------------------------
// FP32 -> 16-bit copies of the decimated strain (FIR data operand)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) to_half_kernel(const HalfConvTask *__restrict__ tasks) {
    const HalfConvTask t = tasks[blockIdx.y];
    using T = typename Op<MODE>::T;
    T *dst = reinterpret_cast<T *>(t.dst);
    float mul = 1.0f;
    if (MODE == kModeE4M3) {                  // per-buffer absmax scaling: samples map to [-448, 448]
        const float amax = t.amax[0];
        mul = amax > 0.0f ? 448.0f / amax : 1.0f;
        if (blockIdx.x == 0 && threadIdx.x == 0) t.amax_next[0] = 0.0f;   // reset for the next push
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = Op<MODE>::cvt(t.src[i] * mul);
}

// |x| maximum of each task's source (E4M3 mode), as the bits of a non-negative float.
__global__ void __launch_bounds__(256) absmax_kernel(const HalfConvTask *__restrict__ tasks) {
    const HalfConvTask t = tasks[blockIdx.y];
    float m = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(t.src[i]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(t.amax), __float_as_int(m));
}

// ---------------------------------------------------------------------------
// a2: Hankel-operand basis FIR
// ---------------------------------------------------------------------------
constexpr int kFirStages = 4;
constexpr int kFirStageBytes = kTcM * 64 * 2;             // 128 rows x 64 K x 2 B
constexpr int kTmemCols = 256;

template <int MODE>
__global__ void __launch_bounds__(128, 1) tc_fir_kernel(const TcFirTask *__restrict__ tasks, int n_tasks,
                                                        int *err) {
    using H = Op<MODE>;
    constexpr int kPh = H::kPhases, kB = H::kBytes, kKC = 128 / kB;   // K elements per 128-byte row
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kFirStages;
    uint64_t *winb = empty + kFirStages;
    uint64_t *accb = winb + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accb + 1);
    uint8_t *a_st = smem + 1024;
    uint8_t *win = a_st + kFirStages * kFirStageBytes;

    const TcFirTask &t = tasks[find_tile(tasks, n_tasks, blockIdx.x)];
    const int local = blockIdx.x - t.tile_begin;
    const int mt = local / t.tiles_n, nt = local % t.tiles_n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        tmem_alloc(tslot, kTmemCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kFirStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(winb, 1);
        mbar_init(accb, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nk = t.Kpad / kKC;

    if (warp == 0 && lane == 0) {
        prefetch_tmap(t.mapW);
        const uint32_t wbytes = (uint32_t)(kTcN * kPh + t.Kpad) * kB;
        mbar_expect_tx(winb, wbytes);
        bulk_load(win, reinterpret_cast<const uint8_t *>(t.x) + kB * (t.X0 + (int64_t)kPh * kTcN * nt), wbytes, winb);
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kFirStages;
            if (kc >= kFirStages && !mbar_wait(&empty[s], ((kc / kFirStages) - 1) & 1, err, 1)) break;
            mbar_expect_tx(&full[s], kFirStageBytes);
            tma_load_2d(a_st + s * kFirStageBytes, t.mapW, kc * kKC, mt * kTcM, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        if (mbar_wait(winb, 0, err, 2)) {
            const uint32_t idesc = idesc_op<MODE>(kTcM, kTcN);
            const uint32_t wa = smem_u32(win);
            bool ok = true;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int s = kc % kFirStages;
                if (!mbar_wait(&full[s], (kc / kFirStages) & 1, err, 3)) { ok = false; break; }
                tc_fence_after();
                const uint32_t aa = smem_u32(a_st + s * kFirStageBytes);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_op<MODE>(tmem, desc_k_sw128(aa + kk * 32), desc_hankel(wa + kc * 128 + kk * 32), idesc,
                                 (kc | kk) != 0);
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(accb);
        }
    }
    __syncwarp();
    const bool have = mbar_wait(accb, 0, err, 4);
    tc_fence_after();
    if (have) {
        // TMEM lane R = lpt r + l_loc (row of W in this tile), column c = block b - 256 nt
        constexpr int lpt = kTcM / kPh;                      // basis vectors per tile
        const int R = warp * 32 + lane;
        const int r = R / lpt;
        const int col = t.o_col + mt * lpt + (R % lpt);
        typename H::T *O = reinterpret_cast<typename H::T *>(t.O);
        const int64_t m_base = (int64_t)kPh * kTcN * nt + r;
        float oscale = 1.0f;                                 // E4M3: strain scale x basis/output scales
        if (MODE == kModeE4M3) oscale = t.xamax[0] * (1.0f / 448.0f) * t.colscale[col];
#pragma unroll 1
        for (int c0 = 0; c0 < kTcN; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t m = m_base + kPh * (c0 + j);
                if (m < t.Bk) O[m * t.ldo + col] = H::cvt(__uint_as_float(v[j]) * oscale);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// a3 + a4 (+ a5 partials at the top level): mixing GEMM with the x2
// interpolation of the coarser level fused into its epilogue.
//   D[a][m] = sum_l M[a][l] O[m][l]   (TMEM lanes = filters, columns = time)
//   y_k[a][m] = D[a][m] + sum_j 2 g[j] y_{k+1}[a][(m - j)/2]
// Tile = 128 filters x 256 samples.  Persistent CTAs (one per SM), warp roles:
//   warp 0   TMA producer: per tile, the K chunks of M and O into a ring of
//            n_stages stage buffers, then the coarser level's window for each
//            half tile (128 filters x 100 samples, FP32) into a ring of n_win
//            window buffers;
//   warp 1   MMA issuer into one of two TMEM accumulators (256 columns each),
//            so the next tile's GEMM runs while this tile's epilogue drains;
//   warps 4-11  epilogue: warp w reads TMEM lanes 32 (w % 4) (its 32 filters)
//            for half tile (w / 4 - 1), takes each filter's 52 coarser samples
//            per 32 outputs from shared memory and interpolates from registers.
// At the top level the epilogue does not store the SNR: it reduces |rho|^2
// over its columns into per-window partial maxima.
// ---------------------------------------------------------------------------
constexpr int kMixRows = 128;                            // filters per tile (MMA M)
constexpr int kMixCols = 256;                            // time samples per tile (MMA N)
constexpr int kMixABytes = kMixRows * 128;               // mixing tile: 128 filters x 128 bytes of K
constexpr int kMixBBytes = kMixCols * 128;               // basis-output tile: 256 time x 128 bytes of K
constexpr int kMixStageBytes = kMixABytes + kMixBBytes;
constexpr int kMixWinCols = 100;                         // coarser samples of a half tile: 64 + 32 taps + 4
constexpr int kMixWinBytes = kMixRows * kMixWinCols * 4;
constexpr int kMixThreads = 384;
constexpr int kMixStBytes = 32 * 32 * 4;                 // store staging: 32 filters x 32 samples, 128-byte swizzle
constexpr int kMixMaxStages = 2, kMixMaxWin = 3;

// x[j] += interpolated coarser level at column c0 + j.  w[i] holds the staged
// coarser sample at register index i; PAR = parity of the first column's
// relative index, REM = offset of the first needed sample inside w; g2 holds
// the doubled odd taps 2 g[2t+1].  Even outputs add the coarser sample itself
// (2 g[0] = 1); odd outputs add 16 symmetric tap pairs, taps outermost so the
// 16 odd outputs of the chunk are independent multiply-add chains.
template <int PAR, int REM>
__device__ __forceinline__ void add_interp(float (&x)[32], const float (&w)[52], const Halfband &g2) {
#pragma unroll
    for (int j = PAR; j < 32; j += 2) x[j] += w[REM + 16 + ((j + PAR) >> 1)];
#pragma unroll
    for (int t = 0; t < kOddTaps; ++t) {
#pragma unroll
        for (int j = 1 - PAR; j < 32; j += 2) {
            const int base = REM + 16 + ((j + PAR) >> 1);
            x[j] = fmaf(g2.odd[t], w[base - t] + w[base + 1 + t], x[j]);
        }
    }
}

__device__ __forceinline__ void add_interp_dispatch(int sel, float (&x)[32], const float (&w)[52],
                                                    const Halfband &g2) {
    switch (sel) {
        case 0: add_interp<0, 0>(x, w, g2); break;
        case 1: add_interp<0, 1>(x, w, g2); break;
        case 2: add_interp<0, 2>(x, w, g2); break;
        case 3: add_interp<0, 3>(x, w, g2); break;
        case 4: add_interp<1, 0>(x, w, g2); break;
        case 5: add_interp<1, 1>(x, w, g2); break;
        case 6: add_interp<1, 2>(x, w, g2); break;
        default: add_interp<1, 3>(x, w, g2); break;
    }
}

struct SegBest {
    float mag2, re, im;
    int64_t n;
};
__device__ __forceinline__ void seg_update(SegBest &b, float m2, float re, float im, int64_t n) {
    if (m2 > b.mag2) {
        b.mag2 = m2;
        b.re = re;
        b.im = im;
        b.n = n;
    }
}
// Takes the other lane's maximum of the same segment when larger (the earlier sample on ties).
__device__ __forceinline__ void seg_merge_pair(SegBest &b) {
    const float om = __shfl_xor_sync(0xffffffffu, b.mag2, 1);
    const float ore = __shfl_xor_sync(0xffffffffu, b.re, 1);
    const float oim = __shfl_xor_sync(0xffffffffu, b.im, 1);
    const long long on = __shfl_xor_sync(0xffffffffu, (long long)b.n, 1);
    if (om > b.mag2 || (om == b.mag2 && om >= 0.0f && on < b.n)) {
        b.mag2 = om;
        b.re = ore;
        b.im = oim;
        b.n = on;
    }
}

// Geometry of one tile, identical for every role.
struct MixTile {
    const TcMixUpTask *t;
    int tt, at, nk;
    int64_t xs0;        // first coarser position of the tile's window (16-byte aligned)
    int rem, par;
};
__device__ __forceinline__ MixTile mix_tile(const TcMixUpTask *tasks, int n_tasks, int tile, int kc_elems) {
    MixTile m;
    m.t = &tasks[find_tile(tasks, n_tasks, tile)];
    const int local = tile - m.t->tile_begin;
    m.tt = local / m.t->tiles_a;
    m.at = local % m.t->tiles_a;
    m.nk = (m.t->Lk_pad + kc_elems - 1) / kc_elems;
    // coarser-level window of column c0 starts at position A0 - 16 + c0/2 (A0: position of
    // relative column 0 halved); loads start 16-byte aligned at xs0 + c0/2, rem floats earlier
    const int64_t rel0 = (int64_t)kMixCols * m.tt - m.t->lam;
    const int64_t A0 = (rel0 >> 1) + m.t->in_off;
    m.xs0 = (A0 - 16) & ~int64_t(3);
    m.rem = (int)((A0 - 16) - m.xs0);
    m.par = (int)(rel0 & 1);
    return m;
}

template <int MODE>
__global__ void __launch_bounds__(kMixThreads, 1) tc_mixup_kernel(const TcMixUpTask *__restrict__ tasks, int n_tasks,
                                                                   int total_tiles, int n_stages, int n_win,
                                                                   int n_stbuf, Halfband g2, int *err) {
    constexpr int kKC = 128 / Op<MODE>::kBytes, kMK = Op<MODE>::kMmaK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kMixMaxStages;
    uint64_t *wfull = empty + kMixMaxStages;
    uint64_t *wempty = wfull + kMixMaxWin;
    uint64_t *afull = wempty + kMixMaxWin;
    uint64_t *aempty = afull + 2;
    uint64_t *mdrain = aempty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mdrain + 1);
    uint8_t *stage = smem + 1024;
    float *win = reinterpret_cast<float *>(stage + n_stages * kMixStageBytes);
    float *stbuf = win + n_win * (kMixWinBytes / 4);      // 1024-byte aligned: n_stbuf per epilogue warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        tmem_alloc(tslot, 2 * kMixCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kMixMaxStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < kMixMaxWin; ++s) {
            mbar_init(&wfull[s], 1);
            mbar_init(&wempty[s], 4);                        // the 4 warps of one half
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&afull[b], 1);
            mbar_init(&aempty[b], 8);                        // all 8 epilogue warps
        }
        mbar_init(mdrain, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        uint32_t su = 0, wu = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
            const MixTile m = mix_tile(tasks, n_tasks, tile, kKC);
            const TcMixUpTask &t = *m.t;
            for (int kc = 0; kc < m.nk; ++kc) {
                const int s = su % n_stages;
                if (su >= (uint32_t)n_stages && !mbar_wait(&empty[s], ((su / n_stages) - 1) & 1, err, 5)) {
                    ok = false;
                    break;
                }
                uint8_t *sa = stage + s * kMixStageBytes;
                mbar_expect_tx(&full[s], kMixStageBytes);
                tma_load_2d(sa, t.mapM, kc * kKC, m.at * kMixRows, &full[s]);
                tma_load_2d(sa + kMixABytes, t.mapO, kc * kKC, m.tt * kMixCols, &full[s]);
                ++su;
            }
            if (!ok || !t.mapY) continue;
            for (int h = 0; h < 2; ++h) {
                const int ws = wu % n_win;
                if (wu >= (uint32_t)n_win && !mbar_wait(&wempty[ws], ((wu / n_win) - 1) & 1, err, 8)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&wfull[ws], kMixWinBytes);
                tma_load_2d(win + ws * (kMixWinBytes / 4), t.mapY, (int)(m.xs0 + 64 * h), m.at * kMixRows,
                            &wfull[ws]);
                ++wu;
            }
        }
        if (!ok) {
            // copies still in flight land before the CTA leaves: wait for the last load of each buffer
            // (the last use of slot s is use s + n ((used - 1 - s) / n); its phase parity is that quotient's)
            for (int s = 0; s < n_stages && s < (int)su; ++s)
                mbar_wait_bounded(&full[s], ((su - 1 - s) / n_stages) & 1);
            for (int s = 0; s < n_win && s < (int)wu; ++s)
                mbar_wait_bounded(&wfull[s], ((wu - 1 - s) / n_win) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        uint32_t su = 0, au = 0;
        bool issued = false;
        const uint32_t idesc = idesc_op<MODE>(kMixRows, kMixCols);
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            const MixTile m = mix_tile(tasks, n_tasks, tile, kKC);
            if (m.nk == 0) continue;
            const int b = au & 1;
            if (au >= 2 && !mbar_wait(&aempty[b], ((au >> 1) - 1) & 1, err, 9)) break;
            tc_fence_after();
            const uint32_t d = tmem + b * kMixCols;
            bool ok = true;
            for (int kc = 0; kc < m.nk; ++kc) {
                const int s = su % n_stages;
                if (!mbar_wait(&full[s], (su / n_stages) & 1, err, 6)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(stage + s * kMixStageBytes);
                const int nmma = min(128 / (kMK * Op<MODE>::kBytes), (m.t->Lk_pad - kc * kKC) / kMK);
                for (int kk = 0; kk < nmma; ++kk)
                    mma_op<MODE>(d, desc_k_sw128(sa + kk * 32), desc_k_sw128(sa + kMixABytes + kk * 32), idesc,
                                 (kc | kk) != 0);
                issued = true;
                mma_commit(&empty[s]);
                ++su;
            }
            if (!ok) break;
            mma_commit(&afull[b]);
            ++au;
        }
        if (issued) {                                        // every MMA has completed before TMEM is freed
            mma_commit(mdrain);
            mbar_wait_bounded(mdrain, 0);
        }
    } else if (warp >= 4) {
        // ---- epilogue ----
        const int q = warp & 3, h = (warp >> 2) - 1;
        const int R = 32 * q + lane;                         // TMEM lane = filter row in the tile
        uint32_t au = 0, wu = 0, stu = 0;                    // stu: staged stores issued by this warp
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            const MixTile m = mix_tile(tasks, n_tasks, tile, kKC);
            const TcMixUpTask &t = *m.t;
            const int b = au & 1;
            bool ok = true;
            if (m.nk > 0) {
                ok = mbar_wait(&afull[b], (au >> 1) & 1, err, 7);
                tc_fence_after();
            }
            int ws = 0;
            if (ok && t.mapY) {
                const uint32_t idx = wu + h;
                ws = idx % n_win;
                ok = mbar_wait(&wfull[ws], (idx / n_win) & 1, err, 10);
            }
            if (!ok) break;
            const int a = kMixRows * m.at + R;
            const bool row_ok = a < t.M2;
            // E4M3: mixing-row scale (levels without slices have no mixing and no scale)
            const float rsc = (MODE == kModeE4M3 && row_ok && t.rscale) ? t.rscale[a] : 1.0f;
            const bool top = t.part != nullptr;
            const float *wrow = win + ws * (kMixWinBytes / 4) + R * kMixWinCols;
            SegBest b0{-1.0f, 0.0f, 0.0f, -1}, b1{-1.0f, 0.0f, 0.0f, -1};
            // top level: columns [vlo, vhi) of this half are real samples (n >= 0, inside the push);
            // columns >= cb belong to the next window (window length >= 128 columns)
            int vlo = 0, vhi = 0, cb = 1 << 30;
            if (top) {
                const int64_t hcol0 = (int64_t)kMixCols * m.tt + 128 * h;
                const int64_t half_first = t.first_n + hcol0;
                vlo = half_first < 0 ? (int)min((int64_t)128, -half_first) : 0;
                vhi = (int)min((int64_t)128, (int64_t)t.Bk - hcol0);
                const int64_t a0 = half_first + vlo;
                const int64_t wend = (a0 >= 0 ? a0 / t.win_len + 1 : 1) * t.win_len;
                cb = (int)min((int64_t)(1 << 30), wend - half_first);
            }
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int c0 = 128 * h + 32 * c;
                float x[32];
                if (m.nk > 0) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * kMixCols + c0, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]) * rsc;
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) x[j] = 0.0f;
                }
                if (t.mapY) {
                    float w[52];
                    const float4 *s4 = reinterpret_cast<const float4 *>(wrow + 16 * c);
#pragma unroll
                    for (int i = 0; i < 13; ++i) {
                        const float4 f = s4[i];
                        w[4 * i] = f.x; w[4 * i + 1] = f.y; w[4 * i + 2] = f.z; w[4 * i + 3] = f.w;
                    }
                    add_interp_dispatch(m.par * 4 + m.rem, x, w, g2);
                }
                const int64_t col0 = (int64_t)kMixCols * m.tt + c0;
                const int64_t n0 = t.first_n + col0;
                if (n0 < 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (n0 + j < 0) x[j] = 0.0f;         // every rate starts at index 0
                }
                if (t.mapYst && n_stbuf > 0) {
                    // staged store: row `lane` of a 32 x 32 tile with 128-byte swizzle (16-byte chunk
                    // i of row r at chunk i ^ (r & 7)), then one TMA store of the whole tile
                    float *sb = stbuf + ((warp - 4) * n_stbuf + (stu & 1)) * (kMixStBytes / 4);
                    if (stu >= 2) {
                        if (lane == 0) bulk_wait_read_1();           // this buffer's previous store has read it
                        __syncwarp();
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        *reinterpret_cast<float4 *>(sb + lane * 32 + ((i ^ (lane & 7)) * 4)) =
                            make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(t.mapYst, sb, (int)(t.yst_col0 + col0), kMixRows * m.at + 32 * q);
                        bulk_commit();
                    }
                    ++stu;
                } else if (t.Y && row_ok) {
                    float *dst = t.Y + (int64_t)a * t.ldy + col0;
                    if (col0 + 32 <= t.Bk) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(dst + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < t.Bk) dst[j] = x[j];
                    }
                }
                if (top) {
                    // lanes 2i, 2i+1 hold the two phases (re, im) of template i
                    const int cl = c0 - 128 * h;
                    const bool odd = lane & 1;
                    if (cl >= vlo && cl + 32 <= vhi && (cl + 32 <= cb || cl >= cb)) {
                        // whole chunk valid and in one window: the even lane takes columns 0-15, the
                        // odd lane 16-31; one exchange gives each lane the other phase of its columns
                        float own[16], oth[16], m2[16];
                        int id[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float lo = x[j], hi = x[j + 16];
                            own[j] = odd ? hi : lo;
                            oth[j] = __shfl_xor_sync(0xffffffffu, odd ? lo : hi, 1);
                            m2[j] = fmaf(oth[j], oth[j], own[j] * own[j]);
                            id[j] = j;
                        }
                        // maximum by a tree, the lower column on ties
#pragma unroll
                        for (int st = 1; st < 16; st *= 2)
#pragma unroll
                            for (int j = 0; j < 16; j += 2 * st)
                                if (m2[j + st] > m2[j]) {
                                    m2[j] = m2[j + st];
                                    id[j] = id[j + st];
                                    own[j] = own[j + st];
                                    oth[j] = oth[j + st];
                                }
                        const float re = odd ? oth[0] : own[0], im = odd ? own[0] : oth[0];
                        const int64_t nb = n0 + id[0] + (odd ? 16 : 0);
                        if (cl >= cb) seg_update(b1, m2[0], re, im, nb);
                        else seg_update(b0, m2[0], re, im, nb);
                    } else {
                        // chunk at a push edge or a window boundary: both lanes scan every column
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float p = __shfl_xor_sync(0xffffffffu, x[j], 1);   // other phase
                            const int cc = cl + j;
                            if (cc < vlo || cc >= vhi) continue;
                            const float mm = fmaf(p, p, x[j] * x[j]);
                            const float re = odd ? p : x[j], im = odd ? x[j] : p;
                            if (cc < cb) seg_update(b0, mm, re, im, n0 + j);
                            else seg_update(b1, mm, re, im, n0 + j);
                        }
                    }
                }
            }
            if (top) {
                seg_merge_pair(b0);                  // the two lanes' maxima of each segment
                seg_merge_pair(b1);
                if ((a & 1) == 0 && row_ok) {
                    WinPart *base = t.part + (int64_t)(a >> 1) * t.n_rec + (m.tt * 2 + h) * 2;
                    base[0] = WinPart{b0.mag2, b0.re, b0.im, 0, b0.n};
                    base[1] = WinPart{b1.mag2, b1.re, b1.im, 0, b1.n};
                }
            }
            // release the accumulator and the window buffer (TMEM reads and shared loads are done)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (m.nk > 0) mbar_arrive(&aempty[b]);
                if (t.mapY) mbar_arrive(&wempty[ws]);
            }
            if (m.nk > 0) ++au;
            if (t.mapY) wu += 2;
        }
        if (stu > 0 && lane == 0) bulk_wait_all();           // stores done before shared memory is released
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kMixCols);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t tc_fir_smem_bytes(int kpad_max, int mode) {
    const int ph = mode == kModeE4M3 ? 16 : 8, by = mode == kModeE4M3 ? 1 : 2;
    return 1024 + 1024 + kFirStages * kFirStageBytes + (size_t)(kTcN * ph + kpad_max) * by;
}
size_t tc_mixup_smem_bytes(int n_stages, int n_win, int n_stbuf) {
    return 1024 + 1024 + (size_t)n_stages * kMixStageBytes + (size_t)n_win * kMixWinBytes +
           (size_t)8 * n_stbuf * kMixStBytes;
}

template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_to_half(const HalfConvTask *d_tasks, int n_tasks, int mode, cudaStream_t s) {
    if (n_tasks == 0) return cudaSuccess;
    dim3 grid(64, n_tasks);
    if (mode == kModeBF16) to_half_kernel<kModeBF16><<<grid, 256, 0, s>>>(d_tasks);
    else if (mode == kModeF16) to_half_kernel<kModeF16><<<grid, 256, 0, s>>>(d_tasks);
    else {
        absmax_kernel<<<grid, 256, 0, s>>>(d_tasks);
        to_half_kernel<kModeE4M3><<<grid, 256, 0, s>>>(d_tasks);
    }
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t fir_launch(const TcFirTask *d_tasks, int n_tasks, int total_tiles, int kpad_max, int *err,
                              cudaStream_t s) {
    const size_t smem = tc_fir_smem_bytes(kpad_max, MODE);
    cudaError_t e = set_smem(tc_fir_kernel<MODE>, smem);
    if (e != cudaSuccess) return e;
    tc_fir_kernel<MODE><<<total_tiles, 128, smem, s>>>(d_tasks, n_tasks, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_fir(const TcFirTask *d_tasks, int n_tasks, int total_tiles, int kpad_max, int mode, int *err,
                          cudaStream_t s) {
    if (n_tasks == 0 || total_tiles == 0) return cudaSuccess;
    if (mode == kModeBF16) return fir_launch<kModeBF16>(d_tasks, n_tasks, total_tiles, kpad_max, err, s);
    if (mode == kModeF16) return fir_launch<kModeF16>(d_tasks, n_tasks, total_tiles, kpad_max, err, s);
    return fir_launch<kModeE4M3>(d_tasks, n_tasks, total_tiles, kpad_max, err, s);
}

static int sm_count() {
    static int count[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (count[dev] == 0 && cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        count[dev] = 148;
    return count[dev];
}

template <int MODE>
static cudaError_t mixup_launch(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, int max_nk,
                                bool tma_store, const Halfband &g, int *err, cudaStream_t s) {
    // shared memory (<= 227 KB): stage, window and store-staging buffers.  Several K chunks per
    // tile: 2 stages, 2 windows, plain stores; one K chunk and stored y: 1, 2 and two staging
    // buffers per epilogue warp; one K chunk at the top level (nothing stored): 1, 3, none
    int n_stages = 1, n_win = 3, n_stbuf = 0;
    if (max_nk >= 2) n_stages = 2, n_win = 2;
    else if (tma_store) n_win = 2, n_stbuf = 2;
    const size_t smem = tc_mixup_smem_bytes(n_stages, n_win, n_stbuf);
    cudaError_t e = set_smem(tc_mixup_kernel<MODE>, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(total_tiles, sm_count());
    Halfband g2;                                     // doubled odd taps 2 g[2t+1] (exact)
    for (int t = 0; t < kOddTaps; ++t) g2.odd[t] = 2.0f * g.odd[t];
    tc_mixup_kernel<MODE><<<grid, kMixThreads, smem, s>>>(d_tasks, n_tasks, total_tiles, n_stages, n_win, n_stbuf,
                                                          g2, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_mixup(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, int max_nk, bool tma_store,
                            const Halfband &g, int mode, int *err, cudaStream_t s) {
    if (n_tasks == 0 || total_tiles == 0) return cudaSuccess;
    if (mode == kModeBF16) return mixup_launch<kModeBF16>(d_tasks, n_tasks, total_tiles, max_nk, tma_store, g, err, s);
    if (mode == kModeF16) return mixup_launch<kModeF16>(d_tasks, n_tasks, total_tiles, max_nk, tma_store, g, err, s);
    return mixup_launch<kModeE4M3>(d_tasks, n_tasks, total_tiles, max_nk, tma_store, g, err, s);
}

}  // namespace lloid
