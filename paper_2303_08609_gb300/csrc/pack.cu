// Gauge packing (canonical lexicographic AoS -> per-(mu, parity) planar formats),
// device buffers and error reporting.
#include <stdio.h>

#include <string>

#include "weo_internal.h"

namespace weo {

// ------------------------------------------------------------------ errors --

static thread_local std::string g_last_error;

int set_error(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}

const char *last_error_message() { return g_last_error.c_str(); }

int fail_cuda(cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s) at %s:%d", what, cudaGetErrorName(e),
             cudaGetErrorString(e), file, line);
    (void)cudaGetLastError();  // clear a non-sticky error so later calls can proceed
    return set_error(e == cudaErrorMemoryAllocation ? WEO_ERR_OOM : WEO_ERR_CUDA, buf);
}

// ----------------------------------------------------------------- buffers --

int Buffer::ensure(size_t n)
{
    if (n <= bytes && ptr) return WEO_OK;
    release();
    if (n == 0) return WEO_OK;
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return fail_cuda(e, "cudaMalloc", __FILE__, __LINE__);
    }
    bytes = n;
    return WEO_OK;
}

void Buffer::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

// ----------------------------------------------------------------- packing --

// One thread per link (mu, lex): read the canonical 3x3 complex matrix and store
// it at parity index lex/2 of the (mu, parity) field.
template <class Lk, typename In>
__global__ void pack_gauge_kernel(const In *__restrict__ canon, char *__restrict__ out,
                                  long long pb, int lx, int ly, int lz, long long V)
{
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= 4 * V) return;
    const int mu = (int)(l / V);
    const long long lex = l - mu * V;
    long long r = lex;
    const int x = (int)(r % lx);
    r /= lx;
    const int y = (int)(r % ly);
    r /= ly;
    const int z = (int)(r % lz);
    const int t = (int)(r / lz);
    const int parity = (x + y + z + t) & 1;
    const In *src = canon + 18 * l;
    cx<double> U[3][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) U[k / 3][k % 3] = {double(src[2 * k]), double(src[2 * k + 1])};
    Lk::store(out + (2 * mu + parity) * pb, V / 2, lex / 2, U);
}

template <class Lk>
static int pack_with(PackedGauge &g, const wilson_eo_s *h, const void *canon, int is_f64,
                     cudaStream_t s)
{
    const long long V = 2 * h->vh;
    const int threads = 256;
    const long long n = 4 * V;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    char *out = static_cast<char *>(g.buf.ptr);
    if (is_f64)
        pack_gauge_kernel<Lk, double><<<blocks, threads, 0, s>>>(
            static_cast<const double *>(canon), out, g.pb, h->dims[0], h->dims[1], h->dims[2], V);
    else
        pack_gauge_kernel<Lk, float><<<blocks, threads, 0, s>>>(
            static_cast<const float *>(canon), out, g.pb, h->dims[0], h->dims[1], h->dims[2], V);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

int pack_gauge(wilson_eo_s *h, PackedGauge &g, int prec, int fmt, const void *canon, int is_f64,
               cudaStream_t s)
{
    g.valid = false;
    g.prec = prec;
    g.fmt = fmt;
    g.pb = h->vh * link_site_bytes(prec, fmt);
    WEO_TRY(g.buf.ensure((size_t)(8 * g.pb)));
    const bool c = fmt == WEO_LINK12;
    int st;
    switch (prec) {
    case WEO_F64: st = c ? pack_with<LkF64_12>(g, h, canon, is_f64, s) : pack_with<LkF64_18>(g, h, canon, is_f64, s); break;
    case WEO_F32: st = c ? pack_with<LkF32_12>(g, h, canon, is_f64, s) : pack_with<LkF32_18>(g, h, canon, is_f64, s); break;
    case WEO_F16: st = c ? pack_with<LkH16_12>(g, h, canon, is_f64, s) : pack_with<LkH16_18>(g, h, canon, is_f64, s); break;
    case WEO_BF16: st = c ? pack_with<LkB16_12>(g, h, canon, is_f64, s) : pack_with<LkB16_18>(g, h, canon, is_f64, s); break;
    case kPrecFF: st = pack_with<LkFF18>(g, h, canon, is_f64, s); break;
    default: return set_error(WEO_ERR_ARG, "unknown precision");
    }
    if (st == WEO_OK) {
        g.valid = true;
        ++g.gen;
    }
    return st;
}

int launch_hop(int prec, int fmt, int io, bool dag, bool axpy, const HopParams &p,
               const LaunchCfg &cfg, cudaStream_t s)
{
    if (p.vh == 0 || p.nrhs == 0) return WEO_OK;
    switch (prec) {
    case WEO_F64: return launch_hop_f64(fmt, dag, axpy, p, cfg, s);
    case WEO_F32: return launch_hop_f32(fmt, dag, axpy, p, cfg, s);
    case WEO_F16: return launch_hop_h16(fmt, io, dag, axpy, p, cfg, s);
    case WEO_BF16: return launch_hop_b16(fmt, io, dag, axpy, p, cfg, s);
    case kPrecFF: return launch_hop_ff(dag, axpy, p, cfg, s);
    default: return set_error(WEO_ERR_ARG, "unknown precision");
    }
}

}  // namespace weo
