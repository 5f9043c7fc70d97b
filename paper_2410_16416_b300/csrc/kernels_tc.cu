// Tensor-core (tcgen05, sm_103a) kernels of the GEMM-shaped steps in the
// reduced-precision modes (SB_BF16, SB_FP16, SB_FP8; FP32 accumulation in TMEM):
//
//  a2 basis FIR as a Hankel GEMM (tc_fir_kernel).  Output time m' = ph b + r
//     (b = block of ph samples, r = phase; ph = 8 for 16-bit operands, 16 for
//     E4M3).  With X[b][j] = x[X0 + ph b + j] the FIR is
//         o[l][ph b + r] = sum_j W[(l,r)][j] X[b][j],
//         W[(l,r)][j]    = v[l][r + Q - 1 + phi - j]   (0 outside the taps),
//     so the data operand is a Hankel matrix whose rows start 16 bytes apart.
//     A plain no-swizzle UMMA descriptor (core matrices 16 B apart along K,
//     8-row groups 128 B apart) reads it straight from one strain window in
//     shared memory: the strain is loaded once per tile, never expanded.  The
//     ph-phase weights W are expanded once at bank creation and streamed by TMA
//     with 128-byte swizzle.  In E4M3 the strain is two terms (hi + lo, one
//     MMA each into the same accumulator) and the outputs are written in BF16.
//     One CTA = 4 warps: warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMAs,
//     then all four warps drain TMEM (each warp owns 32 TMEM lanes).
//  a3 + a4 (+ a5 partials) mixing GEMM and the x2 interpolation of the coarser
//     level in one persistent warp-specialised kernel (tc_mixup_kernel,
//     described at its definition), FP16 or BF16 operands.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

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
// a2: Hankel-operand basis FIR
// ---------------------------------------------------------------------------
constexpr int kFirStages = 4;
constexpr int kFirStageBytes = kTcM * 64 * 2;             // 128 rows x 64 K x 2 B
constexpr int kTmemCols = 256;

template <int MODE>
__global__ void __launch_bounds__(128, 1) tc_fir_kernel(const TcFirTask *__restrict__ tasks, int n_tasks,
                                                        int *err, uint64_t wait_ns, int skip_chunk) {
    // wait_ns: bound of every wait (kWaitLimitNs in normal operation).  skip_chunk >= 0 is a test
    // hook: tile 0's producer does not issue that K chunk's load, so its consumer's wait runs out
    // (nothing is in flight for it) and the failure path below runs.
    using H = Op<MODE>;
    constexpr int kPh = H::kPhases, kB = H::kBytes, kKC = 128 / kB;   // K elements per 128-byte row
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kFirStages;
    uint64_t *winb = empty + kFirStages;
    uint64_t *accb = winb + 1;
    uint64_t *drain = accb + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(drain + 1);
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
        mbar_init(drain, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    griddep_wait();                                  // the prologue above overlaps the previous kernel's tail
    const int nk = t.Kpad / kKC;
    // E4M3: the strain's second term sits right after the first (both windows a multiple of 16 bytes)
    constexpr int kXTerms = MODE == kModeE4M3 ? 2 : 1;
    const uint32_t wbytes = (uint32_t)(kTcN * kPh + t.Kpad) * kB;

    if (warp == 0 && lane == 0) {
        prefetch_tmap(t.mapW);
        const int64_t xoff = kB * (t.X0 + (int64_t)kPh * kTcN * nt);
        mbar_expect_tx(winb, kXTerms * wbytes);
        bulk_load(win, reinterpret_cast<const uint8_t *>(t.x) + xoff, wbytes, winb);
        if (kXTerms == 2) bulk_load(win + wbytes, reinterpret_cast<const uint8_t *>(t.x_lo) + xoff, wbytes, winb);
        int last[kFirStages] = {-1, -1, -1, -1};            // last K chunk whose load was issued, per stage
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kFirStages;
            if (kc >= kFirStages && !mbar_wait(&empty[s], ((kc / kFirStages) - 1) & 1, err, 1, wait_ns)) {
                ok = false;
                break;
            }
            if (kc == skip_chunk && blockIdx.x == 0) continue;   // test hook: this load is never issued
            mbar_expect_tx(&full[s], kFirStageBytes);
            tma_load_2d(a_st + s * kFirStageBytes, t.mapW, kc * kKC, mt * kTcM, &full[s]);
            last[s] = kc;
        }
        // every copy issued into this CTA's shared memory lands before the CTA leaves, also when a
        // wait gave up here or in another role (normally these waits return at once)
        (void)ok;
        mbar_wait_bounded(winb, 0);
        for (int s = 0; s < kFirStages; ++s)
            if (last[s] >= 0) mbar_wait_bounded(&full[s], (last[s] / kFirStages) & 1);
    } else if (warp == 1 && lane == 0) {
        if (mbar_wait(winb, 0, err, 2, wait_ns)) {
            const uint32_t idesc = idesc_op<MODE>(kTcM, kTcN);
            const uint32_t wa = smem_u32(win);
            bool ok = true, issued = false;
            for (int kc = 0; kc < nk && ok; ++kc) {
                const int s = kc % kFirStages;
                if (!mbar_wait(&full[s], (kc / kFirStages) & 1, err, 3, wait_ns)) { ok = false; break; }
                issued = true;
                tc_fence_after();
                const uint32_t aa = smem_u32(a_st + s * kFirStageBytes);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    mma_op<MODE>(tmem, desc_k_sw128(aa + kk * 32), desc_hankel(wa + kc * 128 + kk * 32), idesc,
                                 (kc | kk) != 0);
                    if (kXTerms == 2)
                        mma_op<MODE>(tmem, desc_k_sw128(aa + kk * 32), desc_hankel(wa + wbytes + kc * 128 + kk * 32),
                                     idesc, 1u);
                }
                mma_commit(&empty[s]);
            }
            if (ok) {
                mma_commit(accb);
            } else if (issued) {                             // the issued MMAs finish before TMEM is freed
                mma_commit(drain);
                mbar_wait_bounded(drain, 0);
            }
        }
    }
    __syncwarp();
    const bool have = mbar_wait(accb, 0, err, 4, wait_ns);
    tc_fence_after();
    if (have) {
        // TMEM lane R = lpt r + l_loc (row of W in this tile), column c = block b - 256 nt
        constexpr int lpt = kTcM / kPh;                      // basis vectors per tile
        const int R = warp * 32 + lane;
        const int r = R / lpt;
        const int col = t.o_col + mt * lpt + (R % lpt);
        // basis outputs in the mixing kernel's operand type (E4M3 FIR: BF16)
        using OT = typename Op<mix_mode(MODE)>::T;
        OT *O = reinterpret_cast<OT *>(t.O);
        const int64_t m_base = (int64_t)kPh * kTcN * nt + r;
        float oscale = 1.0f;                                 // E4M3: strain scale x basis-vector scale
        if (MODE == kModeE4M3) oscale = t.xamax[0] * (1.0f / 448.0f) * t.colscale[col];
#pragma unroll 1
        for (int c0 = 0; c0 < kTcN; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t m = m_base + kPh * (c0 + j);
                if (m < t.Bk) O[m * t.ldo + col] = Op<mix_mode(MODE)>::cvt(__uint_as_float(v[j]) * oscale);
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
// a3 + a4 (+ a5 partials at the top level): mixing GEMM and the x2
// interpolation of the coarser level, both on the tensor cores, accumulated
// into one TMEM tile:
//   D[a][m] = sum_l M[a][l] O[m][l] + sum_i y_{k+1}[a][i] U[m][i]
// (TMEM lanes = filters, columns = time; U[m][i] = 2 g[m - 2i] is the banded
// halfband interpolator of step a4).  U is split into two terms U = U_hi + U_lo.
// BF16 mode (also the mixing of SB_FP8 units) stores y as one FP16 plane and
// D takes y U_hi + y U_lo;
// FP16 mode stores y = y_hi + y_lo (BF16) and D takes y_hi U_hi + y_hi U_lo +
// y_lo U_hi (the y_lo U_lo term is below 2^-16 of the result).  Every level
// stores its y in the form the next finer level reads, so no conversion
// happens on the read side.
//
// Tile = 128 filters x 256 samples.  Stored levels cut it into four 64-sample
// blocks (block j reads coarser samples [32 j, 32 j + 80) of the tile's
// window, U is one 64 x 80 matrix); the top level into two 128-sample blocks
// (U is 128 x 112).  U is one of 16 variants: the parity of the tile's first
// sample and the window's offset inside its 16-byte-aligned start.
// Persistent CTAs (one per SM), warp roles:
//   warp 0      TMA producer: mixing chunks (stage ring), the tile's U
//               variant (bulk copy, ring of n_u) and its three window chunks
//               of 64 coarser samples, one or two planes (ring of n_win);
//   warp 1      MMA issuer into one of two TMEM accumulators (256 columns each);
//   warps 4-11  epilogue: warp w reads TMEM lanes 32 (w % 4) for half tile
//               (w / 4 - 1); at the top level it reduces |rho|^2 into
//               per-window partial maxima, below it stores y through a
//               swizzled staging buffer with coalesced 16-byte stores.
// ---------------------------------------------------------------------------
constexpr int kMixRows = 128;                            // filters per tile (MMA M)
constexpr int kMixCols = 256;                            // time samples per tile (MMA N)
// One mixing stage: the mixing tile (128 filters) and the basis-output tile (256 time rows), each row
// `kbytes` of K (32, 64 or 128 bytes: the chunk's swizzle span), rounded to the 1024-byte swizzle atom
constexpr int kMixMaxSt = 6;
constexpr int kWinHalfBytes = kMixRows * 128;            // one plane: 64 coarser samples (16-bit) x 128 filters
constexpr int kWinChunks = 3;                            // 192 >= 7 + 176 coarser samples per tile
// Interpolation block geometry: UB outputs per block (MMA N); a block reads UB/2 + 48 coarser
// samples (its own UB/2, 16 + 16 taps and up to 7 + 1 of alignment), rounded to whole MMA K steps.
template <int UB>
struct UGeo {
    static constexpr int kBlk = UB;
    static constexpr int kK = UB == 64 ? 80 : 112;
    static constexpr int kBytes = kBlk * kK * 2;         // one BF16 term, no-swizzle K-major core matrices
    static constexpr int kVarBytes = 2 * kBytes;         // hi + lo
    static constexpr int kBlocks = 256 / UB;
};
constexpr int kUVariants = 16;                           // (parity, offset 0..7)
// operand table: BF16 hi / lo terms of the 16 variants of the 64-wide blocks, then of the 128-wide
// blocks (FP16 mode, BF16 hi + lo y); then the same two parts as FP16 hi / lo terms (one-plane FP16
// y, BF16 mode)
constexpr size_t kUTab128 = (size_t)kUVariants * UGeo<64>::kVarBytes;
constexpr size_t kUTabPart = kUTab128 + (size_t)kUVariants * UGeo<128>::kVarBytes;
constexpr int kMixStPlane = 32 * 64;                     // store staging per plane: 32 filters x 32 samples
constexpr int kMixThreads = 384;
constexpr int kMixMaxWin = 6;
size_t tc_mixup_stage_bytes(int kbytes) { return ((size_t)(kMixRows + kMixCols) * kbytes + 1023) / 1024 * 1024; }
constexpr size_t kMixSmemMax = 227 * 1024;               // dynamic shared memory per CTA (opt-in maximum)

size_t tc_interp_table_bytes() { return 2 * kUTabPart; }

// U for variant (par, rem): output c of a block takes coarser sample
// i = rem + 16 + ((c + par) >> 1) (even c + par: weight 1 = 2 g[0]) or the
// pairs i - t, i + 1 + t with weight 2 g[2t+1] (odd c + par).  Stored as hi and
// lo terms (BF16, or FP16 with f16) in the no-swizzle K-major layout: element
// (c, i) at byte ((c / 8) * (K / 8) + i / 8) * 128 + (c % 8) * 16 + (i % 8) * 2.
template <int UB>
static void interp_table_part(const Halfband &g, uint16_t *out, bool f16, float gain) {
    using G = UGeo<UB>;
    auto bf16_bits = [](float v) {                       // round to nearest even
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u += 0x7fffu + ((u >> 16) & 1u);
        return (uint16_t)(u >> 16);
    };
    auto bf16_val = [](uint16_t h) {
        const uint32_t u = (uint32_t)h << 16;
        float v;
        std::memcpy(&v, &u, 4);
        return v;
    };
    auto bits = [&](float v) {
        if (!f16) return bf16_bits(v);
        const __half_raw r = __float2half_rn(v);
        return (uint16_t)r.x;
    };
    auto val = [&](uint16_t h) {
        if (!f16) return bf16_val(h);
        __half_raw r;
        r.x = h;
        return __half2float(__half(r));
    };
    for (int var = 0; var < kUVariants; ++var) {
        const int par = var / 8, rem = var % 8;
        uint16_t *hi = out + (size_t)var * (G::kVarBytes / 2), *lo = hi + G::kBytes / 2;
        std::vector<float> U((size_t)G::kBlk * G::kK, 0.0f);
        for (int c = 0; c < G::kBlk; ++c) {
            const int i = rem + 16 + ((c + par) >> 1);
            if (((c + par) & 1) == 0) {
                U[(size_t)c * G::kK + i] = 1.0f;
            } else {
                for (int t = 0; t < kOddTaps; ++t) {
                    U[(size_t)c * G::kK + i - t] = 2.0f * g.odd[t];
                    U[(size_t)c * G::kK + i + 1 + t] = 2.0f * g.odd[t];
                }
            }
        }
        for (int c = 0; c < G::kBlk; ++c)
            for (int i = 0; i < G::kK; ++i) {
                const size_t at = ((size_t)(c / 8) * (G::kK / 8) + i / 8) * 64 + (c % 8) * 8 + (i % 8);
                const float u = U[(size_t)c * G::kK + i] * gain;
                const uint16_t h = bits(u);
                hi[at] = h;
                lo[at] = bits(u - val(h));
            }
    }
}

void tc_interp_table(const Halfband &g, void *host_out) {
    uint8_t *out = static_cast<uint8_t *>(host_out);
    for (int f = 0; f < 2; ++f) {
        interp_table_part<64>(g, reinterpret_cast<uint16_t *>(out + f * kUTabPart), f == 1, 1.0f);
        interp_table_part<128>(g, reinterpret_cast<uint16_t *>(out + f * kUTabPart + kUTab128), f == 1, 1.0f);
    }
}

// Running maximum of one window segment; col is the column within the tile (32-bit arithmetic
// in the per-sample path; the absolute sample is formed once, when the record is written).
struct SegBest {
    float mag2, re, im;
    int col;
};
__device__ __forceinline__ void seg_update(SegBest &b, float m2, float re, float im, int col) {
    if (m2 > b.mag2) {
        b.mag2 = m2;
        b.re = re;
        b.im = im;
        b.col = col;
    }
}
// Takes the other lane's maximum of the same segment when larger (the earlier sample on ties).
__device__ __forceinline__ void seg_merge_pair(SegBest &b) {
    const float om = __shfl_xor_sync(0xffffffffu, b.mag2, 1);
    const float ore = __shfl_xor_sync(0xffffffffu, b.re, 1);
    const float oim = __shfl_xor_sync(0xffffffffu, b.im, 1);
    const int oc = __shfl_xor_sync(0xffffffffu, b.col, 1);
    if (om > b.mag2 || (om == b.mag2 && om >= 0.0f && oc < b.col)) {
        b.mag2 = om;
        b.re = ore;
        b.im = oim;
        b.col = oc;
    }
}

// Geometry of one tile, identical for every role.
struct MixTile {
    const TcMixUpTask *t;
    int tt, at, nk, var;
    int64_t xs0;        // first coarser position of the tile's window (16-byte aligned)
};
// Per-role cursor over the task list.  A CTA's tiles come in increasing order (stride gridDim.x),
// so each role walks the tasks forward and keeps the current task's tile-geometry fields in
// registers, instead of searching the list and re-reading the fields for every tile.
struct MixCursor {
    const TcMixUpTask *t = nullptr;
    int idx = -1, next = 0, begin = 0, tiles_a = 1, nk = 0, lam = 0, in_off = 0, kbytes = 32, Lk_pad = 0;
    bool has_y = false;
    __device__ __forceinline__ void seek(const TcMixUpTask *tasks, int n_tasks, int tile, int kc_elems) {
        if (idx >= 0 && tile < next) return;
        if (idx < 0) idx = find_tile(tasks, n_tasks, tile);
        while (idx + 1 < n_tasks && tasks[idx + 1].tile_begin <= tile) ++idx;
        t = &tasks[idx];
        next = idx + 1 < n_tasks ? tasks[idx + 1].tile_begin : 0x7fffffff;
        begin = t->tile_begin;
        tiles_a = t->tiles_a;
        nk = (t->Lk_pad + kc_elems - 1) / kc_elems;
        lam = t->lam;
        in_off = t->in_off;
        kbytes = t->kbytes;
        Lk_pad = t->Lk_pad;
        has_y = t->mapY != nullptr;
    }
    __device__ __forceinline__ MixTile tile_of(int tile) const {
        MixTile m;
        m.t = t;
        const int local = tile - begin;
        m.tt = local / tiles_a;
        m.at = local % tiles_a;
        m.nk = nk;
        // output column c of the tile interpolates around coarser position A0 + (c + par) / 2
        // (A0: position of relative column 0 halved); the window starts 16-byte aligned at xs0
        const int64_t rel0 = (int64_t)kMixCols * m.tt - lam;
        const int64_t A0 = (rel0 >> 1) + in_off;
        m.xs0 = (A0 - 16) & ~int64_t(7);
        m.var = (int)(rel0 & 1) * 8 + (int)((A0 - 16) - m.xs0);
        return m;
    }
};

// no-swizzle K-major descriptor of U (core matrices 128 B apart along K, (K / 8) 128 B along N)
template <int UB>
__device__ __forceinline__ uint64_t desc_u(uint32_t saddr) {
    return smem_desc(saddr, 128, (UGeo<UB>::kK / 8) * 128, 0);
}

template <int MODE, int UB, bool TOP>
__global__ void __launch_bounds__(kMixThreads, 1) tc_mixup_kernel(const TcMixUpTask *__restrict__ tasks, int n_tasks,
                                                                   int total_tiles, int n_st, int n_win, int n_u,
                                                                   int n_stbuf, int st_bytes,
                                                                   const uint8_t *__restrict__ utab, int *err) {
    constexpr int kKC = 128 / Op<MODE>::kBytes, kMK = Op<MODE>::kMmaK;
    constexpr int NP = y_planes(MODE);                   // 1: FP16 y; 2: BF16 hi + lo
    constexpr int kWinBytes = NP * kWinHalfBytes;
    using G = UGeo<UB>;
    static_assert(MODE != kModeE4M3, "the mixing kernel runs in FP16 or BF16 (mix_mode)");
    utab += (NP == 2 ? 0 : kUTabPart) + (UB == 128 ? kUTab128 : 0);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kMixMaxSt;
    uint64_t *wfull = empty + kMixMaxSt;
    uint64_t *wempty = wfull + kMixMaxWin;
    uint64_t *ufull = wempty + kMixMaxWin;
    uint64_t *uempty = ufull + 2;
    uint64_t *afull = uempty + 2;
    uint64_t *aempty = afull + 2;
    uint64_t *mdrain = aempty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mdrain + 1);
    uint8_t *stage = smem + 1024;                                  // n_st mixing stages
    uint8_t *win = stage + n_st * st_bytes;                        // n_win window chunks
    uint8_t *ubuf = win + n_win * kWinBytes;                       // n_u U variants
    uint8_t *stbuf = ubuf + n_u * G::kVarBytes;                    // n_stbuf per epilogue warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        tmem_alloc(tslot, 2 * kMixCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kMixMaxSt; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < kMixMaxWin; ++s) {
            mbar_init(&wfull[s], 1);
            mbar_init(&wempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ufull[b], 1);
            mbar_init(&uempty[b], 1);
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
    griddep_wait();                                  // the prologue above overlaps the previous kernel's tail

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        uint32_t su = 0, wu = 0, uu = 0;
        int uvar = -1;                                       // U variant in the newest U buffer
        bool ok = true;
        MixCursor cur;
        for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
            cur.seek(tasks, n_tasks, tile, kKC);
            const MixTile m = cur.tile_of(tile);
            const TcMixUpTask &t = *m.t;
            for (int kc = 0; kc < m.nk; ++kc) {
                const int s = su % n_st;
                if (su >= (uint32_t)n_st && !mbar_wait(&empty[s], ((su / n_st) - 1) & 1, err, 5)) {
                    ok = false;
                    break;
                }
                uint8_t *sa = stage + s * st_bytes;
                mbar_expect_tx(&full[s], 3 * kMixRows * t.kbytes);
                tma_load_2d(sa, t.mapM, kc * kKC, m.at * kMixRows, &full[s]);
                tma_load_2d(sa + kMixRows * t.kbytes, t.mapO, kc * kKC, m.tt * kMixCols, &full[s]);
                ++su;
            }
            if (!ok || !t.mapY) continue;
            if (m.var != uvar) {                             // a new U variant (tiles of one task share it)
                const int us = uu % n_u;
                if (uu >= (uint32_t)n_u && !mbar_wait(&uempty[us], ((uu / n_u) - 1) & 1, err, 11)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&ufull[us], G::kVarBytes);
                bulk_load(ubuf + us * G::kVarBytes, utab + (size_t)m.var * G::kVarBytes, G::kVarBytes, &ufull[us]);
                ++uu;
                uvar = m.var;
            }
            for (int wc = 0; wc < kWinChunks; ++wc) {
                const int ws = wu % n_win;
                if (wu >= (uint32_t)n_win && !mbar_wait(&wempty[ws], ((wu / n_win) - 1) & 1, err, 8)) {
                    ok = false;
                    break;
                }
                uint8_t *dst = win + ws * kWinBytes;
                mbar_expect_tx(&wfull[ws], kWinBytes);
                const int x = (int)(m.xs0 + 64 * wc);
                tma_load_2d(dst, t.mapY, x, m.at * kMixRows, &wfull[ws]);                         // (hi)
                if (NP == 2) tma_load_2d(dst + kWinHalfBytes, t.mapY, x, t.M2 + m.at * kMixRows, &wfull[ws]);  // lo
                ++wu;
            }
        }
        {
            // copies still in flight land before the CTA leaves (also when another role or CTA gave up;
            // normally these waits return at once): wait for the last load of each buffer
            // (the last use of slot s of a ring of n is use s + n ((used - 1 - s) / n))
            for (int s = 0; s < n_st && s < (int)su; ++s) mbar_wait_bounded(&full[s], ((su - 1 - s) / n_st) & 1);
            for (int s = 0; s < n_u && s < (int)uu; ++s) mbar_wait_bounded(&ufull[s], ((uu - 1 - s) / n_u) & 1);
            for (int s = 0; s < n_win && s < (int)wu; ++s)
                mbar_wait_bounded(&wfull[s], ((wu - 1 - s) / n_win) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        uint32_t su = 0, wu = 0, uu = 0, au = 0;
        int uvar = -1;
        bool issued = false;
        MixCursor cur;
        const uint32_t idesc = idesc_op<MODE>(kMixRows, kMixCols);
        const uint32_t idesc_u = idesc_op<NP == 1 ? kModeF16 : kModeBF16>(kMixRows, G::kBlk);
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            cur.seek(tasks, n_tasks, tile, kKC);
            const MixTile m = cur.tile_of(tile);
            const bool has_src = cur.has_y;
            const int b = au & 1;
            if (au >= 2 && !mbar_wait(&aempty[b], ((au >> 1) - 1) & 1, err, 9)) break;
            tc_fence_after();
            const uint32_t d = tmem + b * kMixCols;
            bool ok = true;
            for (int kc = 0; kc < m.nk; ++kc) {
                const int s = su % n_st;
                if (!mbar_wait(&full[s], (su / n_st) & 1, err, 6)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int kb = cur.kbytes;
                // descriptors differ only in the start address field (address >> 4, no carry)
                const uint32_t sa = smem_u32(stage + s * st_bytes);
                const uint64_t da = desc_k_sw(sa, kb), db = desc_k_sw(sa + kMixRows * kb, kb);
                const int nmma = min(kb / 32, (cur.Lk_pad - kc * kKC) / kMK);      // 32 bytes of K per MMA
                for (int kk = 0; kk < nmma; ++kk)
                    mma_op<MODE>(d, da + 2 * kk, db + 2 * kk, idesc, (kc | kk) != 0);
                issued = true;
                mma_commit(&empty[s]);
                ++su;
            }
            if (!ok) break;
            if (has_src) {
                if (m.var != uvar) {                         // switch to the next U buffer
                    if (uvar >= 0) {
                        mma_commit(&uempty[(uu - 1) % n_u]);   // released once the previous variant's MMAs complete
                    }
                    if (!mbar_wait(&ufull[uu % n_u], (uu / n_u) & 1, err, 12)) break;
                    ++uu;
                    uvar = m.var;
                }
                const int us = (uu - 1) % n_u;
                tc_fence_after();
                const uint64_t du_hi = desc_u<UB>(smem_u32(ubuf + us * G::kVarBytes)), du_lo = du_hi + (G::kBytes >> 4);
                const uint32_t first = m.nk > 0 ? 1u : 0u;           // no mixing: each block starts afresh
                // block j reads window samples [(UB/2) j, (UB/2) j + K): K step (j, s) sits at sample
                // (UB/2) j + 16 s, in window chunk ((UB/2) j + 16 s) / 64; fully unrolled, so the schedule
                // is fixed at compile time
#pragma unroll
                for (int wc = 0; wc < kWinChunks; ++wc) {
                    const int ws = wu % n_win;
                    if (!mbar_wait(&wfull[ws], (wu / n_win) & 1, err, 13)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da_hi = desc_k_sw128(smem_u32(win + ws * kWinBytes));
                    const uint64_t da_lo = da_hi + (kWinHalfBytes >> 4);
#pragma unroll
                    for (int j = 0; j < G::kBlocks; ++j)
#pragma unroll
                        for (int st = 0; st < G::kK / 16; ++st) {
                            const int kap = (UB / 2) * j + 16 * st;
                            if (kap / 64 != wc) continue;
                            const uint64_t ao = (uint64_t)((kap % 64) * 2 / 16), bo = (uint64_t)(256 * st / 16);
                            const uint32_t dj = d + UB * j;
                            mma_f16(dj, da_hi + ao, du_hi + bo, idesc_u, kap > (UB / 2) * j ? 1u : first);
                            mma_f16(dj, da_hi + ao, du_lo + bo, idesc_u, 1u);
                            if (NP == 2) mma_f16(dj, da_lo + ao, du_hi + bo, idesc_u, 1u);
                        }
                    issued = true;
                    mma_commit(&wempty[ws]);
                    ++wu;
                }
                if (!ok) break;
            }
            mma_commit(&afull[b]);
            ++au;
        }
        if (issued) {                                        // every MMA has completed before TMEM is freed
            mma_commit(mdrain);
            mbar_wait_bounded(mdrain, 0);
        }
    } else if (warp >= 4) {
        // ---- epilogue ----
        const int q = warp & 3, h = (warp >> 2) - 1;            // TMEM lane quarter (warp % 4), half tile
        const int R = 32 * q + lane;                         // TMEM lane = filter row in the tile
        uint8_t *sbuf = stbuf + (warp - 4) * (NP * kMixStPlane);
        uint32_t au = 0;
        MixCursor cur;
        for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
            cur.seek(tasks, n_tasks, tile, kKC);
            const MixTile m = cur.tile_of(tile);
            const TcMixUpTask &t = *m.t;
            const int b = au & 1;
            if (!mbar_wait(&afull[b], (au >> 1) & 1, err, 7)) break;
            tc_fence_after();
            // task fields used per chunk, read once per tile
            const int64_t first_n = t.first_n, Bk = t.Bk, ldy = t.ldy, yst_col0 = t.yst_col0, ldu = t.ldu;
            float *const Y = t.Y;
            uint16_t *const Yh = t.Yh;
            const int M2 = t.M2;
            const int a = kMixRows * m.at + R;
            const bool row_ok = a < M2;
            // 128-wide interpolation blocks run only at the top level (trigger partials, no y stored);
            // 64-wide blocks only below it (y stored): each instantiation keeps only its own epilogue
            constexpr bool kTopKernel = TOP;
            const bool top = kTopKernel && t.part != nullptr;
            SegBest b0{-1.0f, 0.0f, 0.0f, 0x7fffffff}, b1{-1.0f, 0.0f, 0.0f, 0x7fffffff};
            // top level: columns [vlo, vhi) of this half are real samples (n >= 0, inside the push);
            // columns >= cb belong to the next window (window length >= 128 columns)
            int vlo = 0, vhi = 0, cb = 1 << 30;
            if (top) {
                const int64_t hcol0 = (int64_t)kMixCols * m.tt + 128 * h;
                const int64_t half_first = first_n + hcol0;
                vlo = half_first < 0 ? (int)min((int64_t)128, -half_first) : 0;
                vhi = (int)min((int64_t)128, Bk - hcol0);
                const int64_t a0 = half_first + vlo;
                const int64_t wend = (a0 >= 0 ? a0 / t.win_len + 1 : 1) * t.win_len;
                cb = (int)min((int64_t)(1 << 30), wend - half_first);
            }
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int c0 = 128 * h + 32 * c;
                float x[32];
                {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * kMixCols + c0, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]);
                }
                const int64_t col0 = (int64_t)kMixCols * m.tt + c0;
                const int64_t n0 = first_n + col0;
                if (n0 < 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (n0 + j < 0) x[j] = 0.0f;         // every rate starts at index 0
                }
                if (!kTopKernel && Yh && n_stbuf > 0) {
                    // y (FP16, or BF16 hi / lo) through a per-warp staging buffer: row `lane` of one
                    // 32 x 32 tile per plane (64-byte rows, 16-byte chunk i at chunk i ^ ((r >> 1) & 3):
                    // no bank conflicts), then each store instruction writes 8 whole 64-byte row segments
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float y0 = x[2 * j], y1 = x[2 * j + 1];
                        if constexpr (NP == 1) {
                            // one packed conversion that saturates instead of overflowing to infinity
                            // (|SNR| > 65504): y0 to the low half, y1 to the high half
                            uint32_t hv;
                            asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(hv) : "f"(y1), "f"(y0));
                            hw[j] = hv;
                            lw[j] = 0u;
                        } else {
                            const __nv_bfloat162 hv = __floats2bfloat162_rn(y0, y1);   // hi: one packed convert
                            const float2 hf = __bfloat1622float2(hv);
                            const __nv_bfloat162 lv = __floats2bfloat162_rn(y0 - hf.x, y1 - hf.y);
                            hw[j] = *reinterpret_cast<const uint32_t *>(&hv);
                            lw[j] = *reinterpret_cast<const uint32_t *>(&lv);
                        }
                    }
                    __syncwarp();                                   // the previous chunk's reads are done
                    const int sw = (lane >> 1) & 3;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        *reinterpret_cast<uint4 *>(sbuf + lane * 64 + ((i ^ sw) * 16)) =
                            make_uint4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
                        if (NP == 2)
                            *reinterpret_cast<uint4 *>(sbuf + kMixStPlane + lane * 64 + ((i ^ sw) * 16)) =
                                make_uint4(lw[4 * i], lw[4 * i + 1], lw[4 * i + 2], lw[4 * i + 3]);
                    }
                    __syncwarp();
                    const int ch = lane & 3;
                    const int64_t col = yst_col0 + col0 + 8 * ch;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = (lane >> 2) + 8 * i;          // row of the warp's 32
                        const int arow = kMixRows * m.at + 32 * q + r;
                        const int pc = ch ^ ((r >> 1) & 3);
                        const uint4 vh = *reinterpret_cast<const uint4 *>(sbuf + r * 64 + pc * 16);
                        if (arow < M2 && col + 8 <= ldu) {
                            *reinterpret_cast<uint4 *>(Yh + (int64_t)arow * ldu + col) = vh;
                            if (NP == 2)
                                *reinterpret_cast<uint4 *>(Yh + ((int64_t)M2 + arow) * ldu + col) =
                                    *reinterpret_cast<const uint4 *>(sbuf + kMixStPlane + r * 64 + pc * 16);
                        }
                    }
                } else if (kTopKernel && Y && row_ok) {
                    float *dst = Y + (int64_t)a * ldy + col0;
                    if (col0 + 32 <= Bk) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(dst + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < Bk) dst[j] = x[j];
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
                        const int cb_ = c0 + id[0] + (odd ? 16 : 0);       // column within the tile
                        if (cl >= cb) seg_update(b1, m2[0], re, im, cb_);
                        else seg_update(b0, m2[0], re, im, cb_);
                    } else {
                        // chunk at a push edge or a window boundary: both lanes scan every column
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float p = __shfl_xor_sync(0xffffffffu, x[j], 1);   // other phase
                            const int cc = cl + j;
                            if (cc < vlo || cc >= vhi) continue;
                            const float mm = fmaf(p, p, x[j] * x[j]);
                            const float re = odd ? p : x[j], im = odd ? x[j] : p;
                            if (cc < cb) seg_update(b0, mm, re, im, c0 + j);
                            else seg_update(b1, mm, re, im, c0 + j);
                        }
                    }
                }
            }
            if (top) {
                seg_merge_pair(b0);                  // the two lanes' maxima of each segment
                seg_merge_pair(b1);
                if ((a & 1) == 0 && row_ok) {
                    WinPart *base = t.part + (int64_t)(a >> 1) * t.n_rec + (m.tt * 2 + h) * 2;
                    // sample offsets from the push's column 0 (empty records keep an unused offset)
                    const int32_t r0 = b0.mag2 >= 0.0f ? kMixCols * m.tt + b0.col : -1;
                    const int32_t r1 = b1.mag2 >= 0.0f ? kMixCols * m.tt + b1.col : -1;
                    base[0] = WinPart{b0.mag2, b0.re, b0.im, 0.0f, 0.0f, 0.0f, 0, r0};
                    base[1] = WinPart{b1.mag2, b1.re, b1.im, 0.0f, 0.0f, 0.0f, 0, r1};
                    if (t.wmax) {                    // window maxima for the refinement's candidate rule
                        uint32_t *wm = t.wmax + (int64_t)(a >> 1) * t.n_wslot - t.win0;
                        if (b0.mag2 > t.thr2) atomicMax(wm + (first_n + r0) / t.win_len, __float_as_uint(b0.mag2));
                        if (b1.mag2 > t.thr2) atomicMax(wm + (first_n + r1) / t.win_len, __float_as_uint(b1.mag2));
                    }
                }
            }
            // release the accumulator (TMEM reads are done)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&aempty[b]);
            ++au;
        }
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
    const int ph = mode == kModeE4M3 ? 16 : 8, by = mode == kModeE4M3 ? 1 : 2, terms = mode == kModeE4M3 ? 2 : 1;
    return 1024 + 1024 + kFirStages * kFirStageBytes + (size_t)terms * (kTcN * ph + kpad_max) * by;
}
size_t tc_mixup_smem_bytes(int n_st, int n_win, int n_u, int n_stbuf, int ublk, int np, int kbytes) {
    const size_t uvar = ublk == 128 ? UGeo<128>::kVarBytes : UGeo<64>::kVarBytes;
    return 1024 + 1024 + (size_t)n_st * tc_mixup_stage_bytes(kbytes) + (size_t)n_win * np * kWinHalfBytes +
           (size_t)n_u * uvar + (size_t)8 * n_stbuf * np * kMixStPlane;
}
// Opts a kernel into the full 227 KB of dynamic shared memory, once.  The attribute is a limit on
// the launches of the function, kept by the function rather than by a launch: lowering it to one
// launch's size would invalidate an earlier launch of the same function (a captured graph node,
// or a profiler's replay of it) that needs more.  So it is raised to the maximum and never lowered.
template <class K>
static cudaError_t set_smem(K kernel, size_t smem) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;   // (kernel, device) pairs already raised
    if (smem > kMixSmemMax) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const std::pair<const void *, int> id(reinterpret_cast<const void *>(kernel), dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(id)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixSmemMax);
    if (e == cudaSuccess) done.insert(id);
    return e;
}

template <int MODE>
static cudaError_t fir_launch(const TcFirTask *d_tasks, int n_tasks, int total_tiles, int kpad_max, int *err,
                              uint64_t wait_ns, int skip_chunk, cudaStream_t s) {
    const size_t smem = tc_fir_smem_bytes(kpad_max, MODE);
    cudaError_t e = set_smem(tc_fir_kernel<MODE>, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(tc_fir_kernel<MODE>, dim3(total_tiles), dim3(128), smem, s, d_tasks, n_tasks, err, wait_ns,
                      skip_chunk);
}

cudaError_t launch_tc_fir(const TcFirTask *d_tasks, int n_tasks, int total_tiles, int kpad_max, int mode, int *err,
                          cudaStream_t s, uint64_t wait_ns, int skip_chunk) {
    if (n_tasks == 0 || total_tiles == 0) return cudaSuccess;
    if (wait_ns == 0) wait_ns = kWaitLimitNs;
    if (mode == kModeBF16)
        return fir_launch<kModeBF16>(d_tasks, n_tasks, total_tiles, kpad_max, err, wait_ns, skip_chunk, s);
    if (mode == kModeF16)
        return fir_launch<kModeF16>(d_tasks, n_tasks, total_tiles, kpad_max, err, wait_ns, skip_chunk, s);
    return fir_launch<kModeE4M3>(d_tasks, n_tasks, total_tiles, kpad_max, err, wait_ns, skip_chunk, s);
}

static int sm_count() {
    static int count[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (count[dev] == 0 && cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        count[dev] = 148;
    return count[dev];
}

template <int MODE, int UB, bool TOP>
static cudaError_t mixup_launch_ub(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, const MixCfg &cfg,
                                   int n_stbuf, int kbytes, const void *utab, int *err, cudaStream_t s) {
    const size_t smem = tc_mixup_smem_bytes(cfg.n_st, cfg.n_win, cfg.n_u, n_stbuf, UB, y_planes(MODE), kbytes);
    cudaError_t e = set_smem(tc_mixup_kernel<MODE, UB, TOP>, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(total_tiles, sm_count());
    return launch_pdl(tc_mixup_kernel<MODE, UB, TOP>, dim3(grid), dim3(kMixThreads), smem, s, d_tasks, n_tasks,
                      total_tiles, cfg.n_st, cfg.n_win, cfg.n_u, n_stbuf, (int)tc_mixup_stage_bytes(kbytes),
                      static_cast<const uint8_t *>(utab), err);
}

uint32_t tc_mixup_shape_key(int mode, const MixLaunch &ml, int total_tiles) {
    int lg = 0;                                         // log4 of the tile count (coarse buckets)
    while ((1 << (2 * lg + 2)) <= total_tiles && lg < 15) ++lg;
    const uint32_t kb = ml.kbytes <= 32 ? 0u : ml.kbytes <= 64 ? 1u : 2u;
    return (uint32_t)mode | (ml.store_y ? 4u : 0u) | (ml.interp ? 8u : 0u) | ((uint32_t)std::min(ml.max_nk, 3) << 4) |
           (kb << 6) | ((uint32_t)lg << 8);
}

// Pipeline shapes that fit in shared memory (<= 227 KB): 1, 2, 3 or 4 mixing stages (each sized
// for the launch's widest K row), one staging buffer per epilogue warp when the level's y is
// stored, and, when a task interpolates a coarser level, 1-2 U buffers (1 for the wider top-level
// blocks) and a window ring of 2, 3 or 4 chunks (np planes each).  The first candidate is the
// built-in default: the most stages that fit beside a ring of 4.
static std::vector<MixCfg> mix_candidates(const MixLaunch &ml, int ub, int np) {
    std::vector<MixCfg> out;
    const int n_stbuf = ml.store_y ? 1 : 0;
    const int st_opts[] = {4, 3, 2, 1};
    const int win_opts[] = {4, 3, 2};
    for (int n_st : st_opts) {
        if (!ml.interp) {
            if (tc_mixup_smem_bytes(n_st, 0, 0, n_stbuf, ub, np, ml.kbytes) <= kMixSmemMax)
                out.push_back(MixCfg{n_st, 0, 0});
            continue;
        }
        for (int n_u = (ub == 128 ? 1 : 2); n_u >= 1; --n_u)
            for (int n_win : win_opts)
                if (tc_mixup_smem_bytes(n_st, n_win, n_u, n_stbuf, ub, np, ml.kbytes) <= kMixSmemMax)
                    out.push_back(MixCfg{n_st, n_u, n_win});
    }
    auto score = [](const MixCfg &c) { return c.n_st * 16 + c.n_win * 2 + c.n_u; };
    std::stable_sort(out.begin(), out.end(), [&](const MixCfg &a, const MixCfg &b) { return score(a) > score(b); });
    return out;
}

template <int MODE, int UB, bool TOP>
static cudaError_t mixup_launch_tuned(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, const MixLaunch &ml,
                                      const void *utab, int *err, MixTuner *tuner, bool may_tune, cudaStream_t s) {
    const int n_stbuf = ml.store_y ? 1 : 0;
    const std::vector<MixCfg> cands = mix_candidates(ml, UB, y_planes(MODE));
    if (cands.empty()) return cudaErrorInvalidValue;
    MixCfg cfg = cands.front();
    const uint32_t key = tc_mixup_shape_key(MODE, ml, total_tiles);
    const MixCfg *known = tuner ? tuner->find(key) : nullptr;
    if (known) cfg = *known;
    if (tuner && !known && may_tune && cands.size() == 1) tuner->best.emplace_back(key, cfg);
    if (tuner && !known && may_tune && cands.size() > 1) {
        // time every candidate on this push, in kTuneRounds interleaved rounds (each launch computes
        // the same result), and keep the candidate with the smallest of its times
        constexpr int kTuneRounds = 3;
        const size_t nc = cands.size();
        std::vector<cudaEvent_t> ev(kTuneRounds * nc + 1);
        for (auto &x : ev) cudaEventCreate(&x);
        cudaError_t e = cudaEventRecord(ev[0], s);
        for (size_t k = 0; k < kTuneRounds * nc && e == cudaSuccess; ++k) {
            e = mixup_launch_ub<MODE, UB, TOP>(d_tasks, n_tasks, total_tiles, cands[k % nc], n_stbuf, ml.kbytes, utab,
                                          err, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k + 1], s);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
        std::vector<float> best_ms(nc, 1e30f);
        for (size_t k = 0; k < kTuneRounds * nc && e == cudaSuccess; ++k) {
            float ms = 0.0f;
            e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            if (e == cudaSuccess) best_ms[k % nc] = std::min(best_ms[k % nc], ms);
        }
        for (auto &x : ev) cudaEventDestroy(x);
        if (e != cudaSuccess) return e;
        size_t bi = 0;
        for (size_t i = 1; i < nc; ++i)
            if (best_ms[i] < best_ms[bi]) bi = i;
        cfg = cands[bi];
        tuner->best.emplace_back(key, cfg);
        tuner->timed_launches += (int64_t)(kTuneRounds * nc);
        return cudaSuccess;
    }
    return mixup_launch_ub<MODE, UB, TOP>(d_tasks, n_tasks, total_tiles, cfg, n_stbuf, ml.kbytes, utab, err, s);
}

template <int MODE>
static cudaError_t mixup_launch(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, const MixLaunch &ml,
                                const void *utab, int *err, MixTuner *tuner, bool may_tune, cudaStream_t s) {
    // The top level (stores nothing) uses 128-wide interpolation blocks.  So do the stored levels of
    // the one-plane (FP16 y) modes: an N = 128 MMA runs at the full rate, an N = 64 one at about half,
    // and the 128 x 112 operand always fits beside one stage, two window chunks and the staging
    // buffers.  The two-plane FP16 mode keeps 64-wide blocks, which always fit as well.  The block
    // width depends on the operand mode only, so a unit's arithmetic never depends on its group.
    if (!ml.store_y)
        return mixup_launch_tuned<MODE, 128, true>(d_tasks, n_tasks, total_tiles, ml, utab, err, tuner, may_tune, s);
    if (y_planes(MODE) == 1)
        return mixup_launch_tuned<MODE, 128, false>(d_tasks, n_tasks, total_tiles, ml, utab, err, tuner, may_tune, s);
    return mixup_launch_tuned<MODE, 64, false>(d_tasks, n_tasks, total_tiles, ml, utab, err, tuner, may_tune, s);
}

cudaError_t launch_tc_mixup(const TcMixUpTask *d_tasks, int n_tasks, int total_tiles, const MixLaunch &ml,
                            const void *utab, int mode, int *err, MixTuner *tuner, bool may_tune, cudaStream_t s) {
    if (n_tasks == 0 || total_tiles == 0) return cudaSuccess;
    if (mode == kModeBF16) return mixup_launch<kModeBF16>(d_tasks, n_tasks, total_tiles, ml, utab, err, tuner, may_tune, s);
    if (mode == kModeF16) return mixup_launch<kModeF16>(d_tasks, n_tasks, total_tiles, ml, utab, err, tuner, may_tune, s);
    return cudaErrorInvalidValue;                        // E4M3 units mix in BF16 (mix_mode)
}

}  // namespace lloid
