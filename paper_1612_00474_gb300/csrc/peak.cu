// peak.cu -- measured arithmetic peaks of the GPU the library runs on: independent chains of fused
// multiply-adds on every SM (packed float32x2 FFMA2, scalar FFMA, float64 DFMA), timed with CUDA
// events.  The pair kernels are bound by these pipes, so their roofline fractions are taken against
// what this device delivers, at the clocks it runs at, rather than against a nominal figure.
#include "rpb_internal.cuh"

namespace rpb {

constexpr int kPeakChains = 8;       // independent accumulators per thread (latency hidden by ILP)
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;  // 2048 threads per SM
static __device__ float g_peak_sink;  // written only if a chain's sum were -1 (never: all values stay positive)

// Each iteration does kPeakChains fused multiply-adds per thread (two per FFMA2).  The multiplier
// and addend keep the values bounded; the final store is guarded by a condition the compiler cannot
// decide, so no chain is removed.
__global__ void __launch_bounds__(kPeakThreads) peak_ffma2_kernel(int iters, float2 m, float2 c)
{
    float2 acc[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) acc[i] = make_float2(1e-3f * threadIdx.x + i, 0.5f * i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) acc[i] = __ffma2_rn(acc[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += acc[i].x + acc[i].y;
    if (s == -1.f) g_peak_sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma_kernel(int iters, float m, float c)
{
    float acc[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) acc[i] = 1e-3f * threadIdx.x + i;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) acc[i] = fmaf(acc[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += acc[i];
    if (s == -1.f) g_peak_sink = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_dfma_kernel(int iters, double m, double c)
{
    double acc[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) acc[i] = 1e-3 * threadIdx.x + i;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) acc[i] = fma(acc[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += acc[i];
    if (s == -1.0) g_peak_sink = (float)s;
}

}  // namespace rpb

extern "C" int rpb_fma_peak(int kind, void *stream, double *tflops, double *ms)
{
    using namespace rpb;
    if (kind < RPB_PEAK_FFMA2 || kind > RPB_PEAK_DFMA || !tflops) {
        set_error("rpb_fma_peak: unknown kind %d or null output", kind);
        return RPB_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, rc;
    if ((rc = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if ((rc = cuda_fail(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return rc;
    const unsigned grid = (unsigned)(sms * kPeakBlocksPerSm);
    // about 40 ms per launch at the expected rates (float32 ~80 TFLOP/s, float64 ~1 TFLOP/s)
    const int iters = kind == RPB_PEAK_DFMA ? 6000 : (kind == RPB_PEAK_FFMA2 ? 200000 : 400000);
    const double fl_per_iter = kind == RPB_PEAK_FFMA2 ? 4.0 * kPeakChains : 2.0 * kPeakChains;
    const double flops = fl_per_iter * iters * (double)grid * kPeakThreads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = cuda_fail(cudaEventCreate(&e0), "cudaEventCreate"))) return rc;
    if ((rc = cuda_fail(cudaEventCreate(&e1), "cudaEventCreate"))) {
        cudaEventDestroy(e0);
        return rc;
    }
    float best = 0.f;
    for (int rep = 0; rep < 4 && rc == RPB_OK; ++rep) {  // the first launch is a warm-up
        cudaEventRecord(e0, st);
        if (kind == RPB_PEAK_FFMA2)
            peak_ffma2_kernel<<<grid, kPeakThreads, 0, st>>>(iters, make_float2(0.9999999f, 0.9999998f),
                                                             make_float2(1e-7f, 2e-7f));
        else if (kind == RPB_PEAK_FFMA)
            peak_ffma_kernel<<<grid, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f);
        else
            peak_dfma_kernel<<<grid, kPeakThreads, 0, st>>>(iters, 0.9999999999, 1e-10);
        count_launches(1);
        cudaEventRecord(e1, st);
        if ((rc = cuda_fail(cudaEventSynchronize(e1), "peak kernel"))) break;
        float t = 0.f;
        if ((rc = cuda_fail(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime"))) break;
        if (rep > 0 && (best == 0.f || t < best)) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return RPB_OK;
}
