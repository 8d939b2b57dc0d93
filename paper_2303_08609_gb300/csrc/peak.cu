// Arithmetic peak of this GPU's FP64 and FP32 fused multiply-add pipes, for the
// roofline of kernels bound by arithmetic rather than memory (the FP64 hopping
// kernel on a part whose FP64 rate is a small fraction of its FP32 rate).
#include <algorithm>

#include "weo_internal.h"

namespace weo {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;
constexpr int kPeakChains = 8;

__device__ double g_peak_sink;

// Eight independent FMA chains per thread, unrolled four times per iteration.
// a <- a b + c with 0 < b < 1 stays bounded and positive, so the result is
// never the value tested below; the test keeps the chains live.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, T b, T c)
{
    T a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    if (s < T(0)) g_peak_sink = double(s);
}

template <typename T>
static int time_fma(int iters, int grid, cudaStream_t s, double *ms)
{
    cudaEvent_t e0, e1;
    WEO_CUDA(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail_cuda(err, "cudaEventCreate", __FILE__, __LINE__);
    }
    cudaEventRecord(e0, s);
    fma_peak_kernel<T><<<grid, kPeakThreads, 0, s>>>(iters, T(0.5), T(1));
    err = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float f = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail_cuda(err, "FMA peak kernel", __FILE__, __LINE__);
    *ms = f;
    return WEO_OK;
}

template <typename T>
static int fma_peak(double *flops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * kPeakBlocksPerSm;
    const double fma_per_iter = 4.0 * kPeakChains * (double)grid * kPeakThreads;
    // calibrate on a short run (also the warm-up), then time ~100 ms of work
    int iters = sizeof(T) == 8 ? 64 : 1024;
    double ms = 0.0;
    WEO_TRY(time_fma<T>(iters, grid, s, &ms));
    const double rate = fma_per_iter * iters / std::max(ms, 1e-3);  // FMA per ms
    iters = (int)std::min(std::max(100.0 * rate / fma_per_iter, 16.0), 1e7);
    WEO_TRY(time_fma<T>(iters, grid, s, &ms));
    *flops = 2.0 * fma_per_iter * iters / (ms * 1e-3);
    return WEO_OK;
}

}  // namespace weo

using namespace weo;

extern "C" int wilson_eo_alu_peak(int prec, double *flops_per_s, void *stream)
{
    try {
        if (!flops_per_s) return set_error(WEO_ERR_ARG, "flops_per_s is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (prec == WEO_F64) return fma_peak<double>(flops_per_s, s);
        if (prec == WEO_F32) return fma_peak<float>(flops_per_s, s);
        return set_error(WEO_ERR_ARG, "prec must be WEO_F64 or WEO_F32");
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_alu_peak");
    }
}
