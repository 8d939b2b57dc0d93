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

// ------------------------------------------------ L2 -> SM read bandwidth --
// Every thread reads 16-byte words of an L2-resident buffer with L2-only loads
// (ld.global.cg: no L1), grid-strided so each warp request is one contiguous
// 512-byte range, for `passes` passes; the sum keeps the loads live.
constexpr int kL2Threads = 512;
constexpr int kL2BlocksPerSm = 4;

__global__ void __launch_bounds__(kL2Threads) l2_read_kernel(const float4 *buf, long long n4, int passes)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 1234.5f) g_peak_sink = acc;  // the buffer holds zeros: never taken
}

static int l2_peak(double *bytes_per_s, cudaStream_t s)
{
    int dev = 0, sms = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // 48 MiB: well inside the L2 of this GPU (129 MB), far beyond its L1s
    const long long bytes = 48ll << 20, n4 = bytes / 16;
    Buffer buf;
    WEO_TRY(buf.ensure((size_t)bytes));
    int st = WEO_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        cudaError_t e = cudaMemsetAsync(buf.ptr, 0, (size_t)bytes, s);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            st = fail_cuda(e, "L2 probe set-up", __FILE__, __LINE__);
            break;
        }
        const int grid = sms * kL2BlocksPerSm;
        // warm: bring the buffer into L2
        l2_read_kernel<<<grid, kL2Threads, 0, s>>>(static_cast<const float4 *>(buf.ptr), n4, 2);
        const int passes = 40;
        cudaEventRecord(e0, s);
        l2_read_kernel<<<grid, kL2Threads, 0, s>>>(static_cast<const float4 *>(buf.ptr), n4, passes);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = fail_cuda(e, "L2 probe kernel", __FILE__, __LINE__);
            break;
        }
        *bytes_per_s = (double)bytes * passes / (ms * 1e-3);
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    buf.release();
    return st;
}

}  // namespace weo

using namespace weo;

extern "C" int wilson_eo_l2_peak(double *bytes_per_s, void *stream)
{
    try {
        if (!bytes_per_s) return set_error(WEO_ERR_ARG, "bytes_per_s is NULL");
        return l2_peak(bytes_per_s, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_l2_peak");
    }
}

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
