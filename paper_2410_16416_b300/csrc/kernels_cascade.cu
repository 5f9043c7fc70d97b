// a1 in one launch: the decimation cascade of every unit of a push (level k ->
// k + 1 by the halfband, Sec. II.A "down-samples"), and, for the tensor-core
// units, the 16-bit operand copy of every level that the basis FIR reads.
//
// One cluster of kCascadeCtas CTAs per unit.  Level k + 1 needs level k's
// outputs across the whole push (the 65-tap halo crosses any split), so the
// CTAs of a cluster split each level's outputs and meet at a cluster barrier
// (release / acquire: the global-memory writes of one step are visible to every
// CTA of the cluster in the next).  The cluster's CTAs are resident together,
// so the barrier cannot wait on a CTA that has not started.  Every CTA of a
// cluster runs the same sequence of barriers (it depends only on the task).
//
// Arithmetic per output is the same as the one-level-per-launch form: the
// centre tap 1/2 first, then the 16 symmetric pairs in tap order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lloid_internal.h"

namespace lloid {

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// 1024 threads a CTA: the cascade runs on one cluster per unit, so each CTA keeps as many loads in
// flight as it can.
constexpr int kCascThreads = 1024;

// This CTA's share [lo, hi) of n items (contiguous, rounded to 32).
__device__ __forceinline__ void cta_share(int64_t n, int r, int64_t &lo, int64_t &hi) {
    const int64_t per = ((n + kCascadeCtas - 1) / kCascadeCtas + 31) / 32 * 32;
    lo = min(n, per * r);
    hi = min(n, lo + per);
}

constexpr int kCascChunk = 4096;                  // outputs per shared-memory pass
constexpr int kCascSeg = 2 * kCascChunk + 4 * kOddTaps;   // their input span (2 n + 61 samples)

// Decimation of this CTA's share, kCascChunk outputs at a time: the input span of the chunk is
// staged in shared memory with coalesced loads (the 2K - 1 halo on either side), then every
// output reads its 33 taps from there.  Only the samples that non-zero outputs read are loaded.
__device__ __forceinline__ void decimate_share(const DecimTask &t, int r, const Halfband &g, float *seg) {
    int64_t lo, hi;
    cta_share(t.n_out, r, lo, hi);
    for (int64_t p0 = lo; p0 < hi; p0 += kCascChunk) {
        const int n = (int)min((int64_t)kCascChunk, hi - p0);
        const int jv = (int)min((int64_t)n, max((int64_t)0, -(t.first_m + p0)));   // outputs [0, jv) are 0
        const float *src = t.in + t.in_base + 2 * p0 - (2 * kOddTaps - 1);
        if (jv < n)
            for (int i = 2 * jv + threadIdx.x; i < 2 * n + 4 * kOddTaps - 3; i += blockDim.x) seg[i] = src[i];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            float v = 0.0f;                    // every rate's signal starts at index 0
            if (j >= jv) {
                const float *c = seg + 2 * j + (2 * kOddTaps - 1);
                v = 0.5f * c[0];
#pragma unroll
                for (int k = 0; k < kOddTaps; ++k) v = fmaf(g.odd[k], c[-(2 * k + 1)] + c[2 * k + 1], v);
            }
            t.out[p0 + j] = v;
        }
        __syncthreads();                       // the next chunk overwrites the span
    }
}

// 16-bit copy of one level (history and this push): BF16 or FP16 rounding to nearest; E4M3 as two
// terms hi + lo of the samples scaled by 448 / max|x| (per-buffer absmax scaling).
__device__ void convert_share(const HalfConvTask &t, int mode, int r) {
    int64_t lo, hi;
    cta_share(t.n, r, lo, hi);
    if (mode == kModeBF16) {
        __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(t.dst);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) dst[i] = __float2bfloat16_rn(t.src[i]);
    } else if (mode == kModeF16) {
        __half *dst = static_cast<__half *>(t.dst);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) dst[i] = __float2half_rn(t.src[i]);
    } else {
        float m = 0.0f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) m = fmaxf(m, fabsf(t.src[i]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(t.amax), __float_as_int(m));
        cluster_sync_all();                  // this push's maximum is complete
        const float amax = *reinterpret_cast<volatile float *>(t.amax);
        const float mul = amax > 0.0f ? 448.0f / amax : 1.0f;
        __nv_fp8_e4m3 *dst = static_cast<__nv_fp8_e4m3 *>(t.dst);
        __nv_fp8_e4m3 *dlo = static_cast<__nv_fp8_e4m3 *>(t.dst_lo);
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float v = t.src[i] * mul;
            const __nv_fp8_e4m3 h(v);        // saturating
            dst[i] = h;
            dlo[i] = __nv_fp8_e4m3(v - static_cast<float>(h));
        }
        if (r == 0 && threadIdx.x == 0) t.amax_next[0] = 0.0f;   // the next push's accumulator
    }
}

__global__ void __launch_bounds__(kCascThreads) cascade_kernel(const CascadeTask *__restrict__ tasks, Halfband g) {
    griddep_wait();
    const CascadeTask &t = tasks[blockIdx.x / kCascadeCtas];
    const int r = cluster_rank();
    const int n_lev = t.n_lev, n_conv = t.n_conv, mode = t.mode;
    __shared__ float seg[kCascSeg];
    for (int k = 0; k <= n_lev; ++k) {
        // level k is complete here: its 16-bit copy and the next level both read it
        if (k < n_conv) convert_share(t.conv[k], mode, r);
        if (k < n_lev) {
            decimate_share(t.lev[k], r, g, seg);
            cluster_sync_all();
        }
    }
}

cudaError_t launch_cascade(const CascadeTask *d_tasks, int n_tasks, const Halfband &g, cudaStream_t s) {
    if (n_tasks == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_tasks * kCascadeCtas);
    cfg.blockDim = dim3(kCascThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCascadeCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, cascade_kernel, d_tasks, g);
}

}  // namespace lloid
