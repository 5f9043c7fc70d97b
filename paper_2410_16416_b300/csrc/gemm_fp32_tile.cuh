// FP32 SIMT GEMM tile shared by the FP32-mode basis FIR / mixing kernel and the
// FP32 refinement: C[m0:m0+64, n0:n0+128] (+)= A * B for one GemmTask (64 x 128
// tile, 256 threads, 4 x 8 outputs per thread, K in steps of 16).  With GUARD,
// Toeplitz positions outside [0, x_len) read as 0.
#pragma once
#include "lloid_internal.h"

namespace lloid {

template <bool GUARD>
__device__ __forceinline__ void gemm_fp32_tile(const GemmTask &t, int m0, int n0, int64_t x_len) {
    constexpr int TM = kGemmTM, TN = kGemmTN, TK = kGemmTK;
    __shared__ __align__(16) float As[TK][TM + 4];
    __shared__ __align__(16) float Bs[TK][TN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    // loader coordinates
    const int a_r = tid >> 2, a_c = (tid & 3) * 4;      // A: 64 rows x 16 k
    const int b_r = tid >> 4, b_c = (tid & 15) * 8;     // B: 16 k x 128 cols

    for (int k0 = 0; k0 < t.K; k0 += TK) {
        {
            const int gm = m0 + a_r;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gk = k0 + a_c + i;
                As[a_c + i][a_r] = (gm < t.M && gk < t.K) ? t.A[gm * t.lda + gk] : 0.0f;
            }
        }
        {
            const int gk = k0 + b_r;
            if (t.toeplitz) {
                const int64_t xb = t.ldb - gk;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int gn = n0 + b_c + j;
                    bool ok = gk < t.K && gn < t.N;
                    if (GUARD) ok = ok && xb + gn >= 0 && xb + gn < x_len;
                    Bs[b_r][b_c + j] = ok ? t.B[xb + gn] : 0.0f;
                }
            } else {
                const float *brow = t.B + (int64_t)gk * t.ldb;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int gn = n0 + b_c + j;
                    Bs[b_r][b_c + j] = (gk < t.K && gn < t.N) ? brow[gn] : 0.0f;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty * 4 + i;
        if (gm >= t.M) continue;
        float *crow = t.C + (int64_t)gm * t.ldc;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (gn < t.N) crow[gn] = t.beta ? crow[gn] + acc[i][j] : acc[i][j];
        }
    }
}

}  // namespace lloid
