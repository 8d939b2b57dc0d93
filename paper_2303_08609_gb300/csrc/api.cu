// C ABI of libwilson_eo.so: handle life cycle, M_eo, M_eo^dag and single hops.
#include <limits.h>
#include <string.h>

#include <new>
#include <string>

#include "weo_internal.h"

namespace weo {

const char *last_error_message();

HopParams geom_params(const wilson_eo_s *h)
{
    HopParams p;
    memset(&p, 0, sizeof(p));
    p.lxh = h->dims[0] / 2;
    p.ly = h->dims[1];
    p.lz = h->dims[2];
    p.lt = h->dims[3];
    p.vh = (int)h->vh;
    return p;
}

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    int want = -1;
    explicit DeviceGuard(int dev) : want(dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            return;
        }
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

static bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// page-locked host memory (cudaHostAlloc / cudaHostRegister / torch pin_memory)
static bool is_pinned_host_pointer(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Input array: device pointers pass through, host arrays are copied into `buf`
// on the stream. No host synchronisation is needed: the next call on the
// handle's stream runs after the kernels that read `buf`, and a pageable
// source may be reused as soon as cudaMemcpyAsync returns.
static int stage_in(Buffer &buf, const void *p, size_t bytes, cudaStream_t s, const void **dev)
{
    if (is_device_pointer(p)) {
        *dev = p;
        return WEO_OK;
    }
    WEO_TRY(buf.ensure(bytes));
    WEO_CUDA(cudaMemcpyAsync(buf.ptr, p, bytes, cudaMemcpyHostToDevice, s));
    *dev = buf.ptr;
    return WEO_OK;
}

// Output array: device pointers pass through, host arrays get a device buffer
// whose contents finish_out copies back on the stream.
static int stage_out(Buffer &buf, void *p, size_t bytes, void **dev, bool *host)
{
    *host = !is_device_pointer(p);
    if (!*host) {
        *dev = p;
        return WEO_OK;
    }
    WEO_TRY(buf.ensure(bytes));
    *dev = buf.ptr;
    return WEO_OK;
}

// Copy a staged output back. Pinned host memory: asynchronous like device
// memory (the caller synchronises the stream before reading). Pageable host
// memory: the call returns once the result is there.
static int finish_out(void *host_ptr, const void *dev, size_t bytes, bool host, cudaStream_t s)
{
    if (!host) return WEO_OK;
    WEO_CUDA(cudaMemcpyAsync(host_ptr, dev, bytes, cudaMemcpyDeviceToHost, s));
    if (!is_pinned_host_pointer(host_ptr)) WEO_CUDA(cudaStreamSynchronize(s));
    return WEO_OK;
}

// bytes of one external (canonical) spinor of the handle
static size_t ext_spinor_bytes(const wilson_eo_s *h)
{
    return (size_t)h->vh * (h->prec == WEO_F64 ? 192 : 96);
}

static int check_dims(const int *dims, long long *vh)
{
    if (!dims) return set_error(WEO_ERR_ARG, "dims is NULL");
    long long v = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] % 2)
            return set_error(WEO_ERR_DIMS, "every lattice extent must be even and >= 2");
        v *= dims[mu];
        if (v > (long long)INT_MAX * 2) return set_error(WEO_ERR_DIMS, "volume too large");
    }
    *vh = v / 2;
    return WEO_OK;
}

static int upload_gauge(wilson_eo_s *h, const void *gauge, int gauge_is_f64, cudaStream_t s)
{
    const size_t bytes = (size_t)(2 * h->vh) * 4 * 9 * (gauge_is_f64 ? 16 : 8);
    WEO_TRY(h->canon_gauge.ensure(bytes));
    const cudaMemcpyKind kind =
        is_device_pointer(gauge) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    WEO_CUDA(cudaMemcpyAsync(h->canon_gauge.ptr, gauge, bytes, kind, s));
    h->canon_is_f64 = gauge_is_f64 ? 1 : 0;
    h->gauge_f64.valid = false;
    h->gauge_lo.valid = false;
    h->gauge_ff.valid = false;
    WEO_TRY(pack_gauge(h, h->gauge, h->prec, h->fmt, h->canon_gauge.ptr, h->canon_is_f64, s));
    WEO_CUDA(cudaStreamSynchronize(s));
    return WEO_OK;
}

int handle_hop(wilson_eo_s *h, int prec, int fmt, int io, bool dag, bool axpy, const HopParams &p,
               cudaStream_t s)
{
    // staged 1: single-RHS hops; 2: multi-RHS hops too
    const int sm = h->cfg[prec].staged;
    const bool staged = (p.nrhs == 1 ? sm >= 1 : sm == 2) && prec == WEO_F32 && fmt == WEO_LINK18 &&
                        io == IO_SAME && staged_arrays_ok(p, axpy) && staged_ready(h, p, s);
    int tok = -1;
    if (h->prof) {
        const char *kind = staged ? "hop_staged"
                           : io == IO_TO16   ? "hop_to16"
                           : io == IO_FROM16 ? "hop_from16"
                                             : "hop";
        tok = prof_begin(h, kernel_label(kind, prec, fmt, dag, axpy).c_str(), s);
    }
    int st = staged ? launch_hop_staged(h, dag, axpy, p, s)
                    : launch_hop(prec, fmt, io, dag, axpy, p, h->cfg[prec], s);
    prof_end(h, tok, s);
    return st;
}

// M_eo (dag = false) or M_eo^dag on device pointers, for a packed gauge field
// in precision `prec`, with the odd-site intermediate in `tmp`. FP64 / FP32
// operators read and write spinors of their own precision; 16-bit operators
// read and write FP32 spinors and keep the intermediate in 16-bit.
int meo_with(wilson_eo_s *h, const PackedGauge &g, Buffer &tmp, void *out, const void *in,
             int nrhs, bool dag, cudaStream_t s)
{
    const int prec = g.prec;
    if (h->algo == 2 && prec == WEO_F32 && g.fmt == WEO_LINK18) {
        const long long ext32 = h->vh * 96;
        WEO_TRY(tmp.ensure((size_t)ext32));
        for (int r = 0; r < nrhs; ++r)
            WEO_TRY(meo_fstaged(h, g, tmp.ptr, static_cast<char *>(out) + r * ext32,
                                static_cast<const char *>(in) + r * ext32, dag, s));
        return WEO_OK;
    }
    if (h->algo == 1 && prec != WEO_F64 && prec != kPrecFF) {
        const long long ext32 = h->vh * 96;
        WEO_TRY(tmp.ensure((size_t)h->vh * (prec == WEO_F32 ? 96 : spinor_site_bytes(SK_H16))));
        for (int r = 0; r < nrhs; ++r)
            WEO_TRY(meo_fused(h, g, tmp.ptr, static_cast<char *>(out) + r * ext32,
                              static_cast<const char *>(in) + r * ext32, dag, s));
        return WEO_OK;
    }
    HopParams p = geom_params(h);
    p.nrhs = nrhs;
    p.gauge = static_cast<const char *>(g.buf.ptr);
    p.gauge_pb = g.pb;
    const long long ext = h->vh * (prec == WEO_F64 || prec == kPrecFF ? 192 : 96);
    if (prec == WEO_F64 || prec == WEO_F32 || prec == kPrecFF) {
        WEO_TRY(tmp.ensure((size_t)ext * nrhs));
        p.out_parity = 1;
        p.in = in;
        p.in_stride = ext;
        p.out = tmp.ptr;
        p.out_stride = ext;
        WEO_TRY(handle_hop(h, prec, g.fmt, IO_SAME, dag, false, p, s));
        p.out_parity = 0;
        p.in = tmp.ptr;
        p.out = out;
        p.x = in;
        p.x_stride = ext;
        p.a = -h->kappa * h->kappa;
        p.reverse = h->alternate;  // read the intermediate's most recent part first
        return handle_hop(h, prec, g.fmt, IO_SAME, dag, true, p, s);
    }
    const long long s16 = h->vh * spinor_site_bytes(SK_H16);
    WEO_TRY(tmp.ensure((size_t)s16 * nrhs));
    p.out_parity = 1;
    p.in = in;
    p.in_stride = ext;
    p.out = tmp.ptr;
    p.out_stride = s16;
    WEO_TRY(handle_hop(h, prec, g.fmt, IO_TO16, dag, false, p, s));
    p.out_parity = 0;
    p.in = tmp.ptr;
    p.in_stride = s16;
    p.out = out;
    p.out_stride = ext;
    p.x = in;
    p.x_stride = ext;
    p.a = -h->kappa * h->kappa;
    p.reverse = h->alternate;
    return handle_hop(h, prec, g.fmt, IO_FROM16, dag, true, p, s);
}

int meo_device(wilson_eo_s *h, void *out, const void *in, int nrhs, bool dag, cudaStream_t s)
{
    return meo_with(h, h->gauge, h->tmp, out, in, nrhs, dag, s);
}

static int apply_common(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, bool dag,
                        void *stream)
{
    if (!h || !out_e || !in_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
    if (nrhs < 1) return set_error(WEO_ERR_ARG, "nrhs must be >= 1");
    if (out_e == in_e) return set_error(WEO_ERR_ARG, "out_e must not alias in_e");
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = ext_spinor_bytes(h) * (size_t)nrhs;
    const void *in = nullptr;
    void *out = nullptr;
    bool out_host = false;
    WEO_TRY(stage_in(h->stage_in, in_e, bytes, s, &in));
    WEO_TRY(stage_out(h->stage_out, out_e, bytes, &out, &out_host));
    WEO_TRY(meo_device(h, out, in, nrhs, dag, s));
    return finish_out(out_e, out, bytes, out_host, s);
}

static int apply_ff_common(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, bool dag,
                           void *stream)
{
    if (!h || !out_e || !in_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
    if (nrhs < 1) return set_error(WEO_ERR_ARG, "nrhs must be >= 1");
    if (out_e == in_e) return set_error(WEO_ERR_ARG, "out_e must not alias in_e");
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)h->vh * 192 * (size_t)nrhs;  // complex128 and float-float alike
    const void *in = nullptr;
    void *out = nullptr;
    bool out_host = false;
    WEO_TRY(stage_in(h->stage_in, in_e, bytes, s, &in));
    WEO_TRY(stage_out(h->stage_out, out_e, bytes, &out, &out_host));
    const PackedGauge *gf = nullptr;
    WEO_TRY(ff_gauge(h, &gf, s));
    WEO_TRY(h->ff_in.ensure(bytes));
    WEO_TRY(h->ff_out.ensure(bytes));
    WEO_TRY(ff_from_f64(h->ff_in.ptr, in, h->vh, nrhs, s));
    WEO_TRY(meo_with(h, *gf, h->ff_tmp, h->ff_out.ptr, h->ff_in.ptr, nrhs, dag, s));
    WEO_TRY(ff_to_f64(out, h->ff_out.ptr, h->vh, nrhs, s));
    return finish_out(out_e, out, bytes, out_host, s);
}

}  // namespace weo

using namespace weo;

extern "C" {

int wilson_eo_apply_ff64(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, int dag, void *stream)
{
    try {
        return apply_ff_common(h, out_e, in_e, nrhs, dag != 0, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply_ff64");
    }
}

int wilson_eo_create(wilson_eo_t *out, const int dims[4], double kappa, int prec, int linkfmt,
                     const void *gauge, int gauge_is_f64, void *stream)
{
    try {
        if (!out) return set_error(WEO_ERR_ARG, "out is NULL");
        *out = nullptr;
        long long vh = 0;
        WEO_TRY(check_dims(dims, &vh));
        if (prec < WEO_F64 || prec > WEO_BF16) return set_error(WEO_ERR_ARG, "unknown precision");
        if (linkfmt != WEO_LINK18 && linkfmt != WEO_LINK12)
            return set_error(WEO_ERR_ARG, "unknown link format");
        if (!gauge) return set_error(WEO_ERR_ARG, "gauge is NULL");
        wilson_eo_s *h = new (std::nothrow) wilson_eo_s();
        if (!h) return set_error(WEO_ERR_OOM, "host allocation failed");
        for (int mu = 0; mu < 4; ++mu) h->dims[mu] = dims[mu];
        h->vh = vh;
        h->kappa = kappa;
        h->prec = prec;
        h->fmt = linkfmt;
        if (cudaGetDevice(&h->device) != cudaSuccess) {
            delete h;
            return fail_cuda(cudaGetLastError(), "cudaGetDevice", __FILE__, __LINE__);
        }
        int st = upload_gauge(h, gauge, gauge_is_f64, static_cast<cudaStream_t>(stream));
        if (st != WEO_OK) {
            wilson_eo_destroy(h);
            return st;
        }
        *out = h;
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_create");
    }
}

int wilson_eo_set_gauge(wilson_eo_t h, const void *gauge, int gauge_is_f64, void *stream)
{
    try {
        if (!h || !gauge) return set_error(WEO_ERR_ARG, "NULL handle or gauge");
        DeviceGuard g(h->device);
        return upload_gauge(h, gauge, gauge_is_f64, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_set_gauge");
    }
}

int wilson_eo_set_kappa(wilson_eo_t h, double kappa)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    h->kappa = kappa;
    return WEO_OK;
}

int wilson_eo_hop_split(wilson_eo_t h, int ranks, int out_parity, int dag, void *out,
                        const void *in, void *stream)
{
    try {
        if (!h || !out || !in) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (out == in) return set_error(WEO_ERR_ARG, "out must not alias in");
        if (out_parity != 0 && out_parity != 1) return set_error(WEO_ERR_ARG, "out_parity must be 0 or 1");
        if (!is_device_pointer(out) || !is_device_pointer(in))
            return set_error(WEO_ERR_ARG, "wilson_eo_hop_split takes device arrays");
        DeviceGuard dg(h->device);
        return hop_split_device(h, ranks, out_parity, dag != 0, out, in, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_hop_split");
    }
}

int wilson_eo_set_launch(wilson_eo_t h, int threads, int rhs_block, int order)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (order != 0 && order != 1) return set_error(WEO_ERR_ARG, "order must be 0 or 1");
    if (threads < 32 || threads > 1024 || threads % 32)
        return set_error(WEO_ERR_ARG, "threads must be a multiple of 32 in [32, 1024]");
    if (rhs_block != 1 && rhs_block != 2 && rhs_block != 4)
        return set_error(WEO_ERR_ARG, "rhs_block must be 1, 2 or 4");
    if (rhs_block != 1 && h->prec == WEO_F64)
        return set_error(WEO_ERR_UNSUPPORTED, "rhs_block > 1 needs an FP32 or 16-bit handle");
    if (threads > 256) return set_error(WEO_ERR_UNSUPPORTED, "hopping kernels are built for <= 256 threads");
    h->cfg[h->prec].threads = threads;
    h->cfg[h->prec].rhs_block = rhs_block;
    h->alternate = order;
    return WEO_OK;
}

int wilson_eo_set_rhs_lanes(wilson_eo_t h, int lanes)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
        return set_error(WEO_ERR_ARG, "lanes must be 1, 2, 4 or 8");
    if (lanes != 1 && h->prec == WEO_F64)
        return set_error(WEO_ERR_UNSUPPORTED, "lanes > 1 needs an FP32 or 16-bit handle");
    h->cfg[h->prec].lanes = lanes;
    return WEO_OK;
}

int wilson_eo_set_site_blocks(wilson_eo_t h, int blocked)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (blocked != 0 && blocked != 1) return set_error(WEO_ERR_ARG, "blocked must be 0 or 1");
    for (auto &c : h->cfg) c.blocked = blocked;
    return WEO_OK;
}

int wilson_eo_set_tile_links(wilson_eo_t h, int groups, int rhs_per_thread)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (groups != 0 && groups != 2 && groups != 4 && groups != 8)
        return set_error(WEO_ERR_ARG, "groups must be 0, 2, 4 or 8");
    if (rhs_per_thread != 1 && rhs_per_thread != 2)
        return set_error(WEO_ERR_ARG, "rhs_per_thread must be 1 or 2");
    if (groups && h->prec == WEO_F64)
        return set_error(WEO_ERR_UNSUPPORTED, "tile-shared links need an FP32 or 16-bit handle");
    h->cfg[h->prec].tile_links = groups;
    h->cfg[h->prec].tile_rhs_per_thread = rhs_per_thread;
    if (groups) h->cfg[h->prec].rhs_block = 1;
    return WEO_OK;
}

int wilson_eo_get_tile_links(wilson_eo_t h, int *groups, int *rhs_per_thread)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (groups) *groups = h->cfg[h->prec].tile_links;
    if (rhs_per_thread) *rhs_per_thread = h->cfg[h->prec].tile_rhs_per_thread;
    return WEO_OK;
}

int wilson_eo_set_staging(wilson_eo_t h, int staged, int rows, int depth)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        if (staged < 0 || staged > 2) return set_error(WEO_ERR_ARG, "staged must be 0, 1 or 2");
        if (rows < 0 || depth < 0 || depth == 1 || depth > 5)
            return set_error(WEO_ERR_ARG, "rows >= 0, depth 0 or 2..5");
        const int old_rows = h->staged_rows, old_depth = h->staged_depth;
        h->staged_rows = rows;
        h->staged_depth = depth;
        if (staged && !staged_eligible(h)) {
            h->staged_rows = old_rows;
            h->staged_depth = old_depth;
            return set_error(WEO_ERR_UNSUPPORTED,
                             "staged hop: needs Lx/2 even and R >= 2 dividing Ly with R Lx/2 <= 64, "
                             "and the requested stages in 227 KB of shared memory");
        }
        DeviceGuard dg(h->device);
        h->cfg[WEO_F32].staged = staged;
        if (staged) {
            WEO_TRY(fused_prepare(h, 0));  // error word of the bounded waits
            if (h->gauge.prec == WEO_F32) {
                WEO_TRY(staged_prepare(h, h->gauge, 0));
                WEO_CUDA(cudaStreamSynchronize(0));
            }
        } else {
            h->staged_links.release();
            h->staged_valid = false;
        }
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_set_staging");
    }
}

int wilson_eo_get_staging(wilson_eo_t h, int *staged, int *rows, int *depth)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    int r = 0, d = 0;
    staged_shape(h, &r, &d);
    if (staged) *staged = h->cfg[WEO_F32].staged;
    if (rows) *rows = r;
    if (depth) *depth = d;
    return WEO_OK;
}

int wilson_eo_inject_staged_timeout(wilson_eo_t h, void *out_o, const void *in_e, void *stream)
{
    try {
        if (!h || !out_o || !in_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (h->prec != WEO_F32 || h->fmt != WEO_LINK18 || !staged_eligible(h))
            return set_error(WEO_ERR_UNSUPPORTED, "staged hop: FP32 18-real handle on an eligible lattice");
        if (!is_device_pointer(out_o) || !is_device_pointer(in_e))
            return set_error(WEO_ERR_ARG, "device arrays only");
        DeviceGuard dg(h->device);
        WEO_TRY(fused_prepare(h, static_cast<cudaStream_t>(stream)));
        HopParams p = geom_params(h);
        p.nrhs = 1;
        p.gauge = static_cast<const char *>(h->gauge.buf.ptr);
        p.gauge_pb = h->gauge.pb;
        p.out_parity = 1;
        p.in = in_e;
        p.in_stride = h->vh * 96;
        p.out = out_o;
        p.out_stride = h->vh * 96;
        if (!staged_arrays_ok(p, false)) return set_error(WEO_ERR_ARG, "arrays must be 16-byte aligned");
        const bool was = h->cfg[WEO_F32].staged;
        h->cfg[WEO_F32].staged = 1;
        const int st = staged_prepare(h, h->gauge, static_cast<cudaStream_t>(stream));
        h->cfg[WEO_F32].staged = was;
        WEO_TRY(st);
        return launch_hop_staged(h, false, false, p, static_cast<cudaStream_t>(stream), true);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_inject_staged_timeout");
    }
}

int wilson_eo_set_algorithm(wilson_eo_t h, int algo, int lookahead, int threads)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (algo < 0 || algo > 2)
        return set_error(WEO_ERR_ARG, "algo must be 0 (two launches), 1 (fused) or 2 (fused staged)");
    if (algo == 1 && h->prec == WEO_F64)
        return set_error(WEO_ERR_UNSUPPORTED, "the fused M_eo has FP32 arithmetic only");
    if (algo == 2 && !fstaged_eligible(h))
        return set_error(WEO_ERR_UNSUPPORTED,
                         "the fused staged M_eo needs an FP32 handle with 18-real links and a lattice "
                         "the staged tiles cover (Lx/2 even, rows of at most 64 sites dividing Ly)");
    if (lookahead != 0 && (lookahead < 1 || lookahead > 64))
        return set_error(WEO_ERR_ARG, "lookahead must be 0 or in 1..64");
    if (threads != 0 && threads != 128 && threads != 256)
        return set_error(WEO_ERR_ARG, "threads must be 0, 128 or 256");
    h->algo = algo;
    if (lookahead) h->fused_lookahead = lookahead;
    if (threads) h->fused_threads = threads;
    return WEO_OK;
}

int wilson_eo_inject_fused_timeout(wilson_eo_t h, void *out_e, const void *in_e, void *stream)
{
    try {
        if (!h || !out_e || !in_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (h->prec == WEO_F64) return set_error(WEO_ERR_UNSUPPORTED, "the fused M_eo has FP32 arithmetic only");
        if (!is_device_pointer(out_e) || !is_device_pointer(in_e))
            return set_error(WEO_ERR_ARG, "device arrays only");
        DeviceGuard dg(h->device);
        WEO_TRY(h->tmp.ensure((size_t)h->vh * (h->prec == WEO_F32 ? 96 : spinor_site_bytes(SK_H16))));
        if (h->algo == 2)
            return meo_fstaged(h, h->gauge, h->tmp.ptr, out_e, in_e, false, static_cast<cudaStream_t>(stream),
                               true);
        return meo_fused(h, h->gauge, h->tmp.ptr, out_e, in_e, false, static_cast<cudaStream_t>(stream), true);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_inject_fused_timeout");
    }
}

int wilson_eo_check(wilson_eo_t h, void *stream)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        DeviceGuard dg(h->device);
        unsigned int err = 0;
        WEO_TRY(fused_take_error(h, static_cast<cudaStream_t>(stream), &err));
        if (err) return set_error(WEO_ERR_TIMEOUT, "a bounded wait in the fused M_eo or staged hop kernel gave up; results of the calls since the last check are invalid");
        return WEO_OK;
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_check");
    }
}

int wilson_eo_info(wilson_eo_t h, int dims_out[4], long long *half_volume, int *prec,
                   int *linkfmt, double *kappa, size_t *device_bytes)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    if (dims_out)
        for (int mu = 0; mu < 4; ++mu) dims_out[mu] = h->dims[mu];
    if (half_volume) *half_volume = h->vh;
    if (prec) *prec = h->prec;
    if (linkfmt) *linkfmt = h->fmt;
    if (kappa) *kappa = h->kappa;
    if (device_bytes)
        *device_bytes = h->gauge.buf.bytes + h->gauge_f64.buf.bytes + h->gauge_lo.buf.bytes +
                        h->gauge_ff.buf.bytes + h->ff_in.bytes + h->ff_out.bytes + h->ff_tmp.bytes +
                        h->canon_gauge.bytes + h->tmp.bytes + h->tmp2.bytes + h->tmp3.bytes +
                        h->even1.bytes + h->fused_ctrl.bytes + h->halo.bytes + h->staged_links.bytes + h->fs_links.bytes +
                        h->stage_in.bytes +
                        h->stage_out.bytes + h->stage_aux.bytes;
    return WEO_OK;
}

int wilson_eo_apply(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, void *stream)
{
    try {
        return apply_common(h, out_e, in_e, nrhs, false, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply");
    }
}

int wilson_eo_apply_dag(wilson_eo_t h, void *out_e, const void *in_e, int nrhs, void *stream)
{
    try {
        return apply_common(h, out_e, in_e, nrhs, true, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply_dag");
    }
}

int wilson_eo_hop(wilson_eo_t h, int out_parity, int dag, void *out, const void *in, int nrhs,
                  void *stream)
{
    try {
        if (!h || !out || !in) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (nrhs < 1) return set_error(WEO_ERR_ARG, "nrhs must be >= 1");
        if (out_parity != 0 && out_parity != 1) return set_error(WEO_ERR_ARG, "out_parity must be 0 or 1");
        if (out == in) return set_error(WEO_ERR_ARG, "out must not alias in");
        if (h->prec != WEO_F64 && h->prec != WEO_F32)
            return set_error(WEO_ERR_UNSUPPORTED, "wilson_eo_hop needs an FP64 or FP32 handle");
        DeviceGuard g(h->device);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t ext = ext_spinor_bytes(h);
        const size_t bytes = ext * (size_t)nrhs;
        const void *din = nullptr;
        void *dout = nullptr;
        bool out_host = false;
        WEO_TRY(stage_in(h->stage_in, in, bytes, s, &din));
        WEO_TRY(stage_out(h->stage_out, out, bytes, &dout, &out_host));
        HopParams p = geom_params(h);
        p.nrhs = nrhs;
        p.gauge = static_cast<const char *>(h->gauge.buf.ptr);
        p.gauge_pb = h->gauge.pb;
        p.out_parity = out_parity;
        p.in = din;
        p.in_stride = (long long)ext;
        p.out = dout;
        p.out_stride = (long long)ext;
        WEO_TRY(handle_hop(h, h->prec, h->fmt, IO_SAME, dag != 0, false, p, s));
        return finish_out(out, dout, bytes, out_host, s);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_hop");
    }
}

int wilson_eo_link_grad(wilson_eo_t h, void *grad, const void *g_e, const void *phi_e,
                        void *stream)
{
    try {
        if (!h || !grad || !g_e || !phi_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (h->prec != WEO_F64 && h->prec != WEO_F32)
            return set_error(WEO_ERR_UNSUPPORTED, "link gradient needs an FP64 or FP32 handle");
        DeviceGuard dg(h->device);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t sb = ext_spinor_bytes(h);
        const size_t gb = (size_t)(2 * h->vh) * 4 * 9 * (h->prec == WEO_F64 ? 16 : 8);
        const void *g = nullptr, *phi = nullptr;
        void *out = nullptr;
        bool out_host = false;
        WEO_TRY(stage_in(h->stage_in, g_e, sb, s, &g));
        WEO_TRY(stage_in(h->even1, phi_e, sb, s, &phi));
        WEO_TRY(stage_out(h->stage_aux, grad, gb, &out, &out_host));
        WEO_TRY(link_grad_device(h, out, g, phi, 0, s));
        return finish_out(grad, out, gb, out_host, s);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_link_grad");
    }
}

int wilson_eo_force(wilson_eo_t h, void *force, void *dS_dphi_e, const void *phi_e, void *stream)
{
    try {
        if (!h || !force || !phi_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (h->prec != WEO_F64 && h->prec != WEO_F32)
            return set_error(WEO_ERR_UNSUPPORTED, "force needs an FP64 or FP32 handle");
        DeviceGuard dg(h->device);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t sb = ext_spinor_bytes(h);
        const size_t gb = (size_t)(2 * h->vh) * 4 * 9 * (h->prec == WEO_F64 ? 16 : 8);
        const void *phi = nullptr;
        void *out = nullptr, *dphi = nullptr;
        bool out_host = false, dphi_host = false;
        WEO_TRY(stage_in(h->stage_in, phi_e, sb, s, &phi));
        WEO_TRY(stage_out(h->stage_aux, force, gb, &out, &out_host));
        if (dS_dphi_e) WEO_TRY(stage_out(h->stage_out, dS_dphi_e, sb, &dphi, &dphi_host));
        WEO_TRY(h->even1.ensure(sb));
        // g = dS/dchi = 2 M_eo phi; its first hop leaves t = H_oe phi in h->tmp
        WEO_TRY(meo_device(h, h->even1.ptr, phi, 1, false, s));
        WEO_TRY(scale_spinor(h, h->even1.ptr, 1, 2.0, s));
        WEO_TRY(link_grad_device(h, out, h->even1.ptr, phi, 1, s, h->tmp.ptr));
        if (dphi) WEO_TRY(meo_device(h, dphi, h->even1.ptr, 1, true, s));  // 2 M^dag M phi
        if (dphi) WEO_TRY(finish_out(dS_dphi_e, dphi, sb, dphi_host, s));
        return finish_out(force, out, gb, out_host, s);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_force");
    }
}

int wilson_eo_solve(wilson_eo_t h, void *x_e, const void *b_e, double tol, int maxiter, int mixed,
                    int *iters_out, double *true_relres_out, void *stream)
{
    try {
        if (iters_out) *iters_out = 0;
        if (true_relres_out) *true_relres_out = -1.0;
        if (!h || !x_e || !b_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (x_e == b_e) return set_error(WEO_ERR_ARG, "x_e must not alias b_e");
        if (!(tol > 0.0) || tol >= 1.0) return set_error(WEO_ERR_ARG, "tol must be in (0, 1)");
        if (maxiter < 0) return set_error(WEO_ERR_ARG, "maxiter must be >= 0");
        DeviceGuard dg(h->device);
        const bool xh = !is_device_pointer(x_e), bh = !is_device_pointer(b_e);
        return solve_device(h, x_e, b_e, xh, bh, 1, tol, maxiter, mixed, iters_out, true_relres_out,
                            static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solve");
    }
}

int wilson_eo_solve_multi(wilson_eo_t h, void *x_e, const void *b_e, int nrhs, double tol,
                          int maxiter, int mixed, int *iters_out, double *true_relres_out,
                          void *stream)
{
    try {
        if (!h || !x_e || !b_e) return set_error(WEO_ERR_ARG, "NULL handle or array");
        if (nrhs < 1 || nrhs > 64) return set_error(WEO_ERR_ARG, "nrhs must be in 1..64");
        for (int r = 0; r < nrhs; ++r) {
            if (iters_out) iters_out[r] = 0;
            if (true_relres_out) true_relres_out[r] = -1.0;
        }
        if (x_e == b_e) return set_error(WEO_ERR_ARG, "x_e must not alias b_e");
        if (!(tol > 0.0) || tol >= 1.0) return set_error(WEO_ERR_ARG, "tol must be in (0, 1)");
        if (maxiter < 0) return set_error(WEO_ERR_ARG, "maxiter must be >= 0");
        DeviceGuard dg(h->device);
        const bool xh = !is_device_pointer(x_e), bh = !is_device_pointer(b_e);
        return solve_device(h, x_e, b_e, xh, bh, nrhs, tol, maxiter, mixed, iters_out,
                            true_relres_out, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solve_multi");
    }
}

// out = x + kappa H in, in the handle's precision (prepare / reconstruct)
static int source_op(wilson_eo_t h, void *out, const void *in_a, const void *in_b, bool prepare,
                     void *stream)
{
    if (!h || !out || !in_a || !in_b) return set_error(WEO_ERR_ARG, "NULL handle or array");
    if (h->prec != WEO_F64 && h->prec != WEO_F32)
        return set_error(WEO_ERR_UNSUPPORTED, "needs an FP64 or FP32 handle");
    if (out == in_a || out == in_b) return set_error(WEO_ERR_ARG, "output must not alias an input");
    DeviceGuard dg(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t b = ext_spinor_bytes(h);
    const void *a = nullptr, *c = nullptr;
    void *o = nullptr;
    bool oh = false;
    WEO_TRY(stage_in(h->stage_in, in_a, b, s, &a));
    WEO_TRY(stage_in(h->even1, in_b, b, s, &c));
    WEO_TRY(stage_out(h->stage_out, out, b, &o, &oh));
    WEO_TRY(prepare ? prepare_source_device(h, o, a, c, s) : reconstruct_device(h, o, a, c, s));
    return finish_out(out, o, b, oh, s);
}

int wilson_eo_prepare_source(wilson_eo_t h, void *rhs_e, const void *eta_e, const void *eta_o,
                             void *stream)
{
    try {
        return source_op(h, rhs_e, eta_e, eta_o, true, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_prepare_source");
    }
}

int wilson_eo_reconstruct(wilson_eo_t h, void *xi_o, const void *eta_o, const void *xi_e,
                          void *stream)
{
    try {
        return source_op(h, xi_o, eta_o, xi_e, false, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_reconstruct");
    }
}

int wilson_eo_solve_full(wilson_eo_t h, void *xi_e, void *xi_o, const void *eta_e,
                         const void *eta_o, double tol, int maxiter, int mixed, int *iters_out,
                         double *relres_out, void *stream)
{
    try {
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = -1.0;
        if (!h || !xi_e || !xi_o || !eta_e || !eta_o) return set_error(WEO_ERR_ARG, "NULL handle or array");
        const void *ptrs[4] = {xi_e, xi_o, eta_e, eta_o};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < i; ++j)
                if (ptrs[i] == ptrs[j]) return set_error(WEO_ERR_ARG, "arrays must not alias");
        if (!(tol > 0.0) || tol >= 1.0) return set_error(WEO_ERR_ARG, "tol must be in (0, 1)");
        if (maxiter < 0) return set_error(WEO_ERR_ARG, "maxiter must be >= 0");
        DeviceGuard dg(h->device);
        bool host[4];
        for (int i = 0; i < 4; ++i) host[i] = !is_device_pointer(ptrs[i]);
        return solve_full_device(h, xi_e, xi_o, eta_e, eta_o, host, tol, maxiter, mixed, iters_out,
                                 relres_out, static_cast<cudaStream_t>(stream));
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solve_full");
    }
}

int wilson_eo_solver_config(wilson_eo_t h, double delta, int chunk, int use_graphs)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        DeviceGuard dg(h->device);
        return solver_configure(h, delta, chunk, use_graphs);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solver_config");
    }
}

int wilson_eo_solve_stats(wilson_eo_t h, int *iterations, int *reliable_updates,
                          int *fp64_applies, int *ff_applies, double *seconds)
{
    if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
    return solver_stats(h, iterations, reliable_updates, fp64_applies, ff_applies, seconds);
}

int wilson_eo_solver_residual(wilson_eo_t h, int mode)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        DeviceGuard dg(h->device);
        return solver_residual_mode(h, mode);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solver_residual");
    }
}

int wilson_eo_solver_restart(wilson_eo_t h, int restart)
{
    try {
        if (!h) return set_error(WEO_ERR_ARG, "NULL handle");
        DeviceGuard dg(h->device);
        return solver_restart_mode(h, restart);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_solver_restart");
    }
}

void wilson_eo_destroy(wilson_eo_t h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    h->gauge.buf.release();
    h->gauge_f64.buf.release();
    h->gauge_lo.buf.release();
    h->gauge_ff.buf.release();
    h->ff_in.release();
    h->ff_out.release();
    h->ff_tmp.release();
    h->canon_gauge.release();
    h->tmp.release();
    h->tmp2.release();
    h->tmp3.release();
    h->staged_links.release();
    h->fs_links.release();
    h->even1.release();
    h->stage_in.release();
    h->stage_out.release();
    h->stage_aux.release();
    h->fused_ctrl.release();
    h->halo.release();
    solver_destroy(h);
    prof_destroy(h);
    delete h;
}

const char *wilson_eo_strerror(int status)
{
    switch (status) {
    case WEO_OK: return "success";
    case WEO_ERR_ARG: return "invalid argument";
    case WEO_ERR_DIMS: return "invalid lattice dimensions";
    case WEO_ERR_UNSUPPORTED: return "unsupported combination";
    case WEO_ERR_CUDA: return "CUDA error";
    case WEO_ERR_NOT_CONVERGED: return "solver did not converge";
    case WEO_ERR_NONFINITE: return "non-finite value in solver";
    case WEO_ERR_TIMEOUT: return "bounded device wait timed out";
    case WEO_ERR_OOM: return "out of memory";
    default: return "unknown status";
    }
}

const char *wilson_eo_last_error(void) { return last_error_message(); }

}  // extern "C"
