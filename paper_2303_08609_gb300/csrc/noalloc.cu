// wilson_eo_apply_noalloc: M_eo / M_eo^dag in FP32 for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted --
// inside a region that a framework's caching allocator owns, inside a
// real-time loop that must not touch the driver's allocator, or in a plug-in
// that only receives buffers from its host application. Such a caller owns its
// gauge field and spinors already; the only extra memory M_eo needs is the
// odd-site intermediate H_oe in_e, and here that lives in a fixed array that
// is part of the library's device image, not in memory this call allocates.
//
// The scratch array below is a file-scope __device__ variable: every GPU that
// loads this library holds its NOALLOC_SCRATCH_BYTES until the process exits.
// Its host-side name is only a stand-in; host code must not pass it to a
// kernel. The device address is looked up with cudaGetSymbolAddress once per
// device (the first call of the entry point on that device does it) and that
// address is what the kernels receive. The cached address belongs to the
// device's current primary context: after cudaDeviceReset (or any other end of
// that context) it is stale, so the entry point must not be called on a device
// once that device has been reset in this process.
#include <mutex>

#include "weo_internal.h"

namespace weo {

// 32 MiB: one FP32 odd-site spinor of up to NOALLOC_MAX_HALF_VOLUME sites.
constexpr long long NOALLOC_SCRATCH_BYTES = 32LL << 20;
constexpr long long NOALLOC_MAX_HALF_VOLUME = NOALLOC_SCRATCH_BYTES / 96;

static __device__ __align__(256) float2 g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(float2)];

constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (set-up on first use).
static int scratch_address(int device, void **addr)
{
    if (device < 0 || device >= kMaxDevices) return set_error(WEO_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_scratch_addr[device] = p;
    }
    *addr = g_scratch_addr[device];
    return WEO_OK;
}

// Canonical complex64 link U_mu at lexicographic site lex: 9 complex, row-major.
// Each link is read by two sites of a hop and again by the other hop: plain
// cached loads, so the repeat reads can hit in L2.
__device__ __forceinline__ void load_canonical_link(const float2 *gauge, long long V, int mu,
                                                    long long lex, cx<float> U[3][3])
{
    const float2 *p = gauge + 9 * (mu * V + lex);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float2 v = __ldg(p + k);
        U[k / 3][k % 3] = {v.x, v.y};
    }
}

template <int MU, bool FWD, int S0>
__device__ __forceinline__ void noalloc_dir(cx<float> acc[12], const float2 *in, long long vh,
                                            long long nb, const float2 *gauge, long long V,
                                            long long link_lex)
{
    constexpr int S = FWD ? S0 : -S0;
    cx<float> U[3][3];
    load_canonical_link(gauge, V, MU, link_lex, U);
    cx<float> v[12];
    SpF32::load(in, vh, nb, v);
    cx<float> h[2][3], w[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) project<MU, S>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<float> z = {0.f, 0.f};
#pragma unroll
            for (int b = 0; b < 3; ++b) z = FWD ? cfma(U[a][b], h[s][b], z) : cfmaconj(U[b][a], h[s][b], z);
            w[s][a] = z;
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) reconstruct<MU, S>(acc[c], acc[3 + c], acc[6 + c], acc[9 + c], w[0][c], w[1][c]);
}

// One hopping term onto the sites of out_parity (Eq. 1), optionally with the
// axpy of Eq. 4; links read from the canonical layout. A site with parity index
// i and x-parity p has lexicographic index 2 i + p.
template <bool Dag, bool Axpy>
__global__ void __launch_bounds__(128) noalloc_hop_kernel(int lxh, int ly, int lz, int lt,
                                                          int out_parity, const float2 *gauge,
                                                          const float2 *in, float2 *out,
                                                          const float2 *x, float a)
{
    const long long vh = (long long)lxh * ly * lz * lt;
    const long long V = 2 * vh;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    constexpr int S0 = Dag ? -1 : 1;
    int rem = i;
    const int xh = rem % lxh;
    rem /= lxh;
    const int y = rem % ly;
    rem /= ly;
    const int z = rem % lz;
    const int t = rem / lz;
    const int par = (y + z + t + out_parity) & 1;
    const int sy = lxh, sz = lxh * ly, st = lxh * ly * lz;
    const int row = i - xh;
    const int xp = par ? (xh + 1 == lxh ? 0 : xh + 1) : xh;
    const int xm = par ? xh : (xh == 0 ? lxh - 1 : xh - 1);
    const long long n_xp = row + xp, n_xm = row + xm;
    const long long n_yp = i + (y + 1 == ly ? -(ly - 1) * sy : sy);
    const long long n_ym = i + (y == 0 ? (ly - 1) * sy : -sy);
    const long long n_zp = i + (z + 1 == lz ? -(lz - 1) * sz : sz);
    const long long n_zm = i + (z == 0 ? (lz - 1) * sz : -sz);
    const long long n_tp = i + (t + 1 == lt ? -(long long)(lt - 1) * st : st);
    const long long n_tm = i + (t == 0 ? (long long)(lt - 1) * st : -st);
    const long long own = 2LL * i + par;  // lex of this site
    // lex of the backward neighbours: same x-parity except in the x direction
    const long long b_x = 2 * n_xm + (1 - par), b_y = 2 * n_ym + par, b_z = 2 * n_zm + par,
                    b_t = 2 * n_tm + par;

    cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
    noalloc_dir<0, true, S0>(acc, in, vh, n_xp, gauge, V, own);
    noalloc_dir<0, false, S0>(acc, in, vh, n_xm, gauge, V, b_x);
    noalloc_dir<1, true, S0>(acc, in, vh, n_yp, gauge, V, own);
    noalloc_dir<1, false, S0>(acc, in, vh, n_ym, gauge, V, b_y);
    noalloc_dir<2, true, S0>(acc, in, vh, n_zp, gauge, V, own);
    noalloc_dir<2, false, S0>(acc, in, vh, n_zm, gauge, V, b_z);
    noalloc_dir<3, true, S0>(acc, in, vh, n_tp, gauge, V, own);
    noalloc_dir<3, false, S0>(acc, in, vh, n_tm, gauge, V, b_t);
    if (Axpy) {
        cx<float> xv[12];
        SpF32::load(x, vh, i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[k].r = fmaf(a, acc[k].r, xv[k].r);
            acc[k].i = fmaf(a, acc[k].i, xv[k].i);
        }
    }
    SpF32::store(out, vh, i, acc);
}

// Device memory of `device` itself, or managed memory. Device memory of another
// GPU is refused: without peer access the kernels would fault on it.
static bool device_accessible(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace weo

using namespace weo;

extern "C" int wilson_eo_apply_noalloc(const int dims[4], double kappa, const void *gauge,
                                       void *out_e, const void *in_e, int dag, void *stream)
{
    try {
        if (!dims || !gauge || !out_e || !in_e) return set_error(WEO_ERR_ARG, "NULL argument");
        if (out_e == in_e) return set_error(WEO_ERR_ARG, "out_e must not alias in_e");
        long long v = 1;
        for (int mu = 0; mu < 4; ++mu) {
            if (dims[mu] < 2 || dims[mu] % 2)
                return set_error(WEO_ERR_DIMS, "every lattice extent must be even and >= 2");
            v *= dims[mu];
        }
        const long long vh = v / 2;
        if (vh > NOALLOC_MAX_HALF_VOLUME)
            return set_error(WEO_ERR_DIMS,
                             "lattice too large for wilson_eo_apply_noalloc: V/2 must be <= 349525 "
                             "sites (its fixed scratch holds one FP32 odd-site spinor, 32 MiB)");
        int device = 0;
        WEO_CUDA(cudaGetDevice(&device));
        if (!device_accessible(gauge, device) || !device_accessible(out_e, device) ||
            !device_accessible(in_e, device))
            return set_error(WEO_ERR_ARG,
                             "wilson_eo_apply_noalloc takes device arrays of the current device only");
        void *scratch = nullptr;
        WEO_TRY(scratch_address(device, &scratch));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int threads = 128;
        const unsigned blocks = (unsigned)((vh + threads - 1) / threads);
        const int lxh = dims[0] / 2;
        const float2 *g = static_cast<const float2 *>(gauge);
        const float2 *in = static_cast<const float2 *>(in_e);
        float2 *out = static_cast<float2 *>(out_e);
        float2 *tmp = static_cast<float2 *>(scratch);
        const float a = (float)(-kappa * kappa);
        // tmp_o = H_oe in_e (every odd site written before it is read)
        if (dag)
            noalloc_hop_kernel<true, false><<<blocks, threads, 0, s>>>(lxh, dims[1], dims[2], dims[3], 1, g, in, tmp, nullptr, 0.f);
        else
            noalloc_hop_kernel<false, false><<<blocks, threads, 0, s>>>(lxh, dims[1], dims[2], dims[3], 1, g, in, tmp, nullptr, 0.f);
        WEO_CUDA(cudaGetLastError());
        // out_e = in_e - kappa^2 H_eo tmp_o
        if (dag)
            noalloc_hop_kernel<true, true><<<blocks, threads, 0, s>>>(lxh, dims[1], dims[2], dims[3], 0, g, tmp, out, in, a);
        else
            noalloc_hop_kernel<false, true><<<blocks, threads, 0, s>>>(lxh, dims[1], dims[2], dims[3], 0, g, tmp, out, in, a);
        WEO_CUDA(cudaGetLastError());
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply_noalloc");
    }
}
