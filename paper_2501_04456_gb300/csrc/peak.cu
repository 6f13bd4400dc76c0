// peak.cu -- FP32 CUDA-core throughput microbenchmark: the denominator of the
// all-pairs kernel's roofline.
//
// The all-pairs pair body is FP32 arithmetic on the CUDA cores (no tensor
// cores), so its roofline is the rate at which the SMs retire FP32
// fused multiply-adds.  This kernel measures that rate directly: every thread
// runs CHAINS independent dependency chains a <- a * b + c, either as scalar
// FFMA (2 flops per lane per instruction) or as the packed float32x2 FFMA2
// that the pair kernels use (4 flops per lane per instruction), with enough
// chains and resident warps to hide the FMA latency.  The result is written
// only under a condition that never holds for the values used, so the chains
// cannot be removed by the compiler.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

constexpr int kPeakBlock = 256;

template <bool PACKED, int CHAINS>
__global__ void __launch_bounds__(kPeakBlock)
k_fma_peak(long long iters, float b, float c, float *__restrict__ sink)
{
    // starting values differ per thread and chain; every chain tends to
    // c / (1 - b) = 10 and stays finite and normal
    const float a0 = 1.0f + 1e-3f * (float)(threadIdx.x & 7);
    if (PACKED) {
        float2 a[CHAINS];
#pragma unroll
        for (int k = 0; k < CHAINS; ++k)
            a[k] = make_float2(a0 + (float)k, a0 - (float)k);
        const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll 16
        for (long long it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < CHAINS; ++k)
                a[k] = __ffma2_rn(a[k], bb, cc);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < CHAINS; ++k)
            s += a[k].x + a[k].y;
        if (s == -1.0f) // never: every chain stays positive
            sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else {
        float a[CHAINS];
#pragma unroll
        for (int k = 0; k < CHAINS; ++k)
            a[k] = a0 + (float)k;
#pragma unroll 16
        for (long long it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < CHAINS; ++k)
                a[k] = __fmaf_rn(a[k], b, c);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < CHAINS; ++k)
            s += a[k];
        if (s == -1.0f)
            sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

constexpr int kChains = 8;

template <bool PACKED>
cudaError_t launch_fma_peak(int grid, long long iters, float *sink, cudaStream_t st)
{
    // b < 1 and c > 0: every chain converges to c / (1 - b) > 0 and stays normal
    k_fma_peak<PACKED, kChains><<<grid, kPeakBlock, 0, st>>>(iters, 0.9999f, 1e-3f, sink);
    return cudaGetLastError();
}

cudaError_t fma_peak_run(int packed, long long iters, int *grid_out, double *flops,
                         float *ms, cudaStream_t st)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    e = packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<true, kChains>,
                                                               kPeakBlock, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<false, kChains>,
                                                               kPeakBlock, 0);
    if (e != cudaSuccess)
        return e;
    if (occ < 1)
        occ = 1;
    const int grid = sms * occ; // one full wave: every SM holds occ CTAs throughout
    float *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(float) * (size_t)grid * kPeakBlock);
    if (e != cudaSuccess)
        return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    auto launch = [&](long long n) {
        return packed ? launch_fma_peak<true>(grid, n, sink, st)
                      : launch_fma_peak<false>(grid, n, sink, st);
    };
    if (e == cudaSuccess)
        e = launch(iters / 8 + 1); // warm-up (clocks, instruction cache)
    if (e == cudaSuccess)
        e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
        e = launch(iters);
    if (e == cudaSuccess)
        e = cudaEventRecord(e1, st);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(e1);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(ms, e0, e1);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess)
        return e;
    *grid_out = grid;
    *flops = (double)grid * kPeakBlock * (double)iters * kChains * (packed ? 4.0 : 2.0);
    return cudaSuccess;
}
} // namespace

} // namespace npsim

extern "C" int npsim_fma_peak(int packed, int64_t iters, void *stream, double *flops, float *ms,
                              int *grid)
{
    using namespace npsim;
    if (!flops || !ms || iters < 1 || iters > (1ll << 40))
        return report_error(NPSIM_ERR_INVALID_ARG,
                            "flops and ms are required and iters must be in [1, 2^40]");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return report_error(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    int g = 0;
    const cudaError_t e = fma_peak_run(packed ? 1 : 0, (long long)iters, &g, flops, ms,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess)
        return report_error(e == cudaErrorMemoryAllocation ? NPSIM_ERR_OOM : NPSIM_ERR_CUDA,
                            "FMA microbenchmark failed: %s", cudaGetErrorString(e));
    if (grid)
        *grid = g;
    return NPSIM_OK;
}
