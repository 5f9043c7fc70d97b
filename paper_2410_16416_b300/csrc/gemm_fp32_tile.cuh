// FP32 SIMT GEMM tile of the SB_FP32 mode's basis FIR (a2, Toeplitz B operand)
// and mixing step (a3): C[m0:m0+128, n0:n0+128] (+)= A * B for one GemmTask.
// 256 threads, 8 x 8 outputs per thread (rows 8 ty.., columns 4 tx.. and
// 64 + 4 tx..), K in steps of 8.  The next K step's operands are fetched into
// registers while the current one is multiplied out of shared memory (two
// shared-memory buffers, one barrier per K step), so global-load latency hides
// behind 512 FMAs per thread.  Each output's sum runs over k in increasing
// order, so results depend only on the operands.
#pragma once
#include "lloid_internal.h"

namespace lloid {

__device__ __forceinline__ void gemm_fp32_tile(const GemmTask &t, int m0, int n0) {
    constexpr int TM = kGemmTM, TN = kGemmTN, TK = kGemmTK;
    static_assert(TM == 128 && TN == 128 && TK == 8, "tile geometry of the loaders below");
    __shared__ __align__(16) float As[2][TK][TM + 4];      // padded: the loaders' stores hit 32 banks
    __shared__ __align__(16) float Bs[2][TK][TN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    // loaders: A rows a_r + 32 i (i < 4) at k a_k; B row b_k, columns b_n + 32 j (j < 4)
    const int a_r = tid >> 3, a_k = tid & 7;
    const int b_k = tid >> 5, b_n = tid & 31;
    float ra[4], rb[4];
    auto fetch = [&](int k0) {
        const int gk = k0 + a_k;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gm = m0 + a_r + 32 * i;
            ra[i] = (gm < t.M && gk < t.K) ? t.A[(int64_t)gm * t.lda + gk] : 0.0f;
        }
        const int bk = k0 + b_k;
        if (t.toeplitz) {
            const float *xb = t.B + (t.ldb - bk);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gn = n0 + b_n + 32 * j;
                rb[j] = (bk < t.K && gn < t.N) ? xb[gn] : 0.0f;
            }
        } else {
            const float *brow = t.B + (int64_t)bk * t.ldb;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gn = n0 + b_n + 32 * j;
                rb[j] = (bk < t.K && gn < t.N) ? brow[gn] : 0.0f;
            }
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 4; ++i) As[buf][a_k][a_r + 32 * i] = ra[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) Bs[buf][b_k][b_n + 32 * j] = rb[j];
    };

    fetch(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < t.K; k0 += TK) {
        const bool more = k0 + TK < t.K;
        if (more) fetch(k0 + TK);                       // in flight while this step multiplies
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) {
            stash(buf ^ 1);                              // the other buffer: last read one step ago
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + ty * 8 + i;
        if (gm >= t.M) continue;
        float *crow = t.C + (int64_t)gm * t.ldc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gn = n0 + 64 * h + tx * 4;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = acc[i][4 * h + j];
            if (t.beta) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (gn + j < t.N) v[j] += crow[gn + j];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (gn + j < t.N) crow[gn + j] = v[j];
        }
    }
}

}  // namespace lloid
