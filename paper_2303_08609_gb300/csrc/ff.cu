// Float-float operator support: conversions between canonical complex128
// spinors and the SpFF layout, and the lazily packed float-float gauge field.
#include "weo_internal.h"

namespace weo {

// src: nrhs x [12][vh] double2 ; dst: nrhs x ([12][vh] float2 high parts, [12][vh] low parts)
__global__ void k_f64_to_ff(float2 *__restrict__ dst, const double2 *__restrict__ src, long long vh,
                            long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long per = 12 * vh, r = e / per, k = e - r * per;
        const double2 v = src[e];
        const float hx = float(v.x), hy = float(v.y);
        float2 *d = dst + r * 2 * per + k;
        d[0] = make_float2(hx, hy);
        d[per] = make_float2(float(v.x - double(hx)), float(v.y - double(hy)));
    }
}

__global__ void k_ff_to_f64(double2 *__restrict__ dst, const float2 *__restrict__ src, long long vh,
                            long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long per = 12 * vh, r = e / per, k = e - r * per;
        const float2 *s = src + r * 2 * per + k;
        const float2 h = s[0], l = s[per];
        dst[e] = make_double2(double(h.x) + double(l.x), double(h.y) + double(l.y));
    }
}

static unsigned conv_grid(long long n)
{
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

int ff_from_f64(void *dst, const void *src, long long vh, int nrhs, cudaStream_t s)
{
    const long long n = 12 * vh * nrhs;
    k_f64_to_ff<<<conv_grid(n), 256, 0, s>>>(static_cast<float2 *>(dst), static_cast<const double2 *>(src), vh, n);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

int ff_to_f64(void *dst, const void *src, long long vh, int nrhs, cudaStream_t s)
{
    const long long n = 12 * vh * nrhs;
    k_ff_to_f64<<<conv_grid(n), 256, 0, s>>>(static_cast<double2 *>(dst), static_cast<const float2 *>(src), vh, n);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

int ff_gauge(wilson_eo_s *h, const PackedGauge **g, cudaStream_t s)
{
    if (!h->gauge_ff.valid)
        WEO_TRY(pack_gauge(h, h->gauge_ff, kPrecFF, WEO_LINK18, h->canon_gauge.ptr, h->canon_is_f64, s));
    *g = &h->gauge_ff;
    return WEO_OK;
}

}  // namespace weo
