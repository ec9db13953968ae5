// Rate probes for the roofline of the narrow band (not part of the method).
//
// The narrow band's per-point work ends in a 64-bit atomicMin of the packed key (|d|, feature)
// (Algorithm 1's minimum-magnitude merge): in shared memory in the tile kernel, in global memory
// in the paper's own schedule (Section 9, one thread per region looping over its cells).  Neither
// rate has a published figure, so these kernels measure them, and the FP64 rate that bounds the
// filtered re-decision, on the device at hand.  Each launch runs a fixed number of operations; the
// caller times it (CUDA events on the same stream) and divides.
#include <stdint.h>

#include "sdf_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 4;
constexpr int SMEM_WORDS = 4096;  // 32 KB of keys per CTA

// 64-bit atomicMin in shared memory: lane l of a warp hits word l + 32 m (m drawn per step), the
// pattern of the tile kernel's merge, where the lanes of a warp hold consecutive points of a row.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_smem_min(unsigned long long *sink, int64_t iters) {
    __shared__ unsigned long long pool[SMEM_WORDS];
    for (int i = threadIdx.x; i < SMEM_WORDS; i += blockDim.x) pool[i] = ~0ull;
    __syncthreads();
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 1u;
    const int lane = threadIdx.x & 31;
    for (int64_t k = 0; k < iters; k++) {
        x = x * 1664525u + 1013904223u;  // LCG (Numerical Recipes constants)
        const int m = (int)(__shfl_sync(0xffffffffu, x, 0) >> 25);  // one row offset per warp, 0..127
        atomicMin(&pool[(lane + 32 * m) & (SMEM_WORDS - 1)], ((unsigned long long)x << 20) | (uint64_t)k);
    }
    __syncthreads();
    if (threadIdx.x == 0) sink[blockIdx.x] = pool[blockIdx.x & (SMEM_WORDS - 1)];
}

// 64-bit atomicMin in global memory on scattered words of a footprint of n_words (a power of
// two): every lane hits its own pseudo-random word, as the regions of the paper's schedule walk
// unrelated cells.  A footprint within L2 measures the L2 atomic units, a larger one adds DRAM.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_global_min(unsigned long long *buf, int64_t n_words,
                                                                     int64_t iters) {
    uint64_t x = (uint64_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B97F4A7C15ull + 1u;
    const uint64_t mask = (uint64_t)n_words - 1;
    for (int64_t k = 0; k < iters; k++) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;  // 64-bit LCG (Knuth's MMIX constants)
        atomicMin(&buf[(x >> 17) & mask], (x >> 8) | 1ull);
    }
}

// FP64 fused multiply-add throughput: 8 independent chains per thread.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fp64(double *sink, int64_t iters) {
    double a[8];
    const double b = 0.999999 + 1e-9 * threadIdx.x, c = 1e-7;
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = 1.0 + 1e-3 * j + 1e-6 * (blockIdx.x & 63);
    for (int64_t k = 0; k < iters; k++)
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += a[j];
    if (s == 12345.678) sink[0] = s;  // keeps the chains alive; never true for these inputs
}

}  // namespace

extern "C" int sdf_probe_rate(int32_t kind, void *buf, int64_t n_words, int64_t iters, int64_t *ops,
                              void *stream) {
    if (!buf || iters < 1 || !ops) return SDF_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SDF_ERR_CUDA;
    const int ctas = PROBE_CTAS_PER_SM * sms;
    const int64_t threads = (int64_t)ctas * PROBE_THREADS;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kind) {
    case SDF_PROBE_SMEM_ATOMIC_MIN:
        if (n_words < ctas) return SDF_ERR_INVALID_ARG;  // one sink word per CTA
        k_probe_smem_min<<<ctas, PROBE_THREADS, 0, s>>>(reinterpret_cast<unsigned long long *>(buf), iters);
        *ops = threads * iters;
        break;
    case SDF_PROBE_GLOBAL_ATOMIC_MIN:
        if (n_words < 1 || (n_words & (n_words - 1))) return SDF_ERR_INVALID_ARG;  // a power of two
        k_probe_global_min<<<ctas, PROBE_THREADS, 0, s>>>(reinterpret_cast<unsigned long long *>(buf), n_words, iters);
        *ops = threads * iters;
        break;
    case SDF_PROBE_FP64_FMA:
        if (n_words < 1) return SDF_ERR_INVALID_ARG;
        k_probe_fp64<<<ctas, PROBE_THREADS, 0, s>>>(reinterpret_cast<double *>(buf), iters);
        *ops = threads * iters * 8 * 2;  // flops: 8 chains, 2 per FMA
        break;
    default:
        return SDF_ERR_INVALID_ARG;
    }
    SDF_LAUNCHED(1);
    return cudaGetLastError() == cudaSuccess ? SDF_OK : SDF_ERR_CUDA;
}
