// Conversion between the two orderings of a single-parity spinor field:
//   site-major  psi[rhs][i][spin][colour]   (each site's 12 components together)
//   planar      psi[rhs][spin][colour][i]   (the library's external layout)
// with i = lex/2 the x-compacted parity index of Sec. 3.3 in both. The planar
// order lets a warp read one component of 32 consecutive sites as one
// contiguous request, which is what every hopping kernel here is built on;
// callers that hold the site-major order convert once on the device.
//
// One CTA moves 128 sites of one right-hand side: the contiguous block on the
// site-major side goes through shared memory, so both the load and the store
// of every element are coalesced.
#include "weo_internal.h"

namespace weo {

constexpr int kLayoutSites = 128;
constexpr int kLayoutPad = 13;  // shared-memory row of 12 components + 1 (fewer bank conflicts)

template <typename T, bool ToPlanar>
__global__ void __launch_bounds__(kLayoutSites) layout_kernel(T *dst, const T *src, long long vh)
{
    __shared__ T buf[kLayoutSites * kLayoutPad];
    const long long s0 = (long long)blockIdx.x * kLayoutSites;
    const long long rhs = blockIdx.y;
    const int n = (int)min((long long)kLayoutSites, vh - s0);
    const T *in = src + rhs * 12 * vh;
    T *out = dst + rhs * 12 * vh;
    if (ToPlanar) {
        // contiguous block of n sites x 12 components
        for (int e = threadIdx.x; e < 12 * n; e += blockDim.x)
            buf[(e / 12) * kLayoutPad + e % 12] = in[s0 * 12 + e];
        __syncthreads();
        if ((int)threadIdx.x < n)
#pragma unroll
            for (int k = 0; k < 12; ++k) out[k * vh + s0 + threadIdx.x] = buf[threadIdx.x * kLayoutPad + k];
    } else {
        if ((int)threadIdx.x < n)
#pragma unroll
            for (int k = 0; k < 12; ++k) buf[threadIdx.x * kLayoutPad + k] = in[k * vh + s0 + threadIdx.x];
        __syncthreads();
        for (int e = threadIdx.x; e < 12 * n; e += blockDim.x)
            out[s0 * 12 + e] = buf[(e / 12) * kLayoutPad + e % 12];
    }
}

static bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace weo

using namespace weo;

extern "C" int wilson_eo_spinor_layout(long long half_volume, int nrhs, int elem_bytes, int to_planar,
                                       void *dst, const void *src, void *stream)
{
    try {
        if (!dst || !src) return set_error(WEO_ERR_ARG, "NULL array");
        if (half_volume < 1 || nrhs < 1 || nrhs > 65535)
            return set_error(WEO_ERR_ARG, "half_volume must be >= 1 and nrhs in 1..65535");
        if (elem_bytes != 8 && elem_bytes != 16)
            return set_error(WEO_ERR_ARG, "elem_bytes must be 8 (complex64) or 16 (complex128)");
        if (to_planar != 0 && to_planar != 1) return set_error(WEO_ERR_ARG, "to_planar must be 0 or 1");
        const long long bytes = half_volume * 12 * nrhs * elem_bytes;
        const char *d = static_cast<const char *>(dst), *s0 = static_cast<const char *>(src);
        if (d < s0 + bytes && s0 < d + bytes) return set_error(WEO_ERR_ARG, "dst and src overlap");
        if (!on_device(dst) || !on_device(src))
            return set_error(WEO_ERR_ARG, "wilson_eo_spinor_layout takes device arrays only");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const dim3 grid((unsigned)((half_volume + kLayoutSites - 1) / kLayoutSites), (unsigned)nrhs);
        if (elem_bytes == 8) {
            if (to_planar)
                layout_kernel<float2, true><<<grid, kLayoutSites, 0, s>>>((float2 *)dst, (const float2 *)src, half_volume);
            else
                layout_kernel<float2, false><<<grid, kLayoutSites, 0, s>>>((float2 *)dst, (const float2 *)src, half_volume);
        } else {
            if (to_planar)
                layout_kernel<double2, true><<<grid, kLayoutSites, 0, s>>>((double2 *)dst, (const double2 *)src, half_volume);
            else
                layout_kernel<double2, false><<<grid, kLayoutSites, 0, s>>>((double2 *)dst, (const double2 *)src, half_volume);
        }
        WEO_CUDA(cudaGetLastError());
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_spinor_layout");
    }
}
