// Fused M_eo: both hops of Eq. 4 in one persistent kernel, with the odd-site
// intermediate kept in a small ring of t-slices that stays in L2.
//
// Work is a queue of items (hop, t-slice, chunk of CTA size). Slice tasks are
// ordered as a wavefront:
//     A(Lt-1), A(0), A(1), B(0), A(2), B(1), ..., A(Lt-2), B(Lt-3), B(Lt-2), B(Lt-1)
// where A(t) = H_oe onto the odd sites of slice t (written to the ring) and
// B(t) = in - kappa^2 H_eo tmp onto the even sites of slice t (read from the
// ring slices t-1, t, t+1). CTAs take items from an atomic ticket in queue
// order. An item may only wait for items earlier in the queue:
//   B(t) waits until A(t-1), A(t), A(t+1) are complete;
//   A(t) (ring slot t mod R) waits until the three B tasks that read the
//        slot's previous slice (t-R) are complete (needs R >= 3).
// Because a ticket is only handed out after all earlier ones, the earliest
// unfinished item never waits, so the queue always progresses. Every wait is
// bounded: after `spin_limit` polls the CTA records an error code and gives up,
// and every other wait gives up as soon as it sees the error; the host reports
// WEO_ERR_TIMEOUT.
//
// Slices 0 and Lt-1 keep dedicated slots (they are read at both ends of the
// periodic wavefront). The ring is read with L2-only loads (ld.global.cg): its
// slots are rewritten during the launch, so L1 copies could be stale.
//
// DRAM traffic per M_eo approaches the minimum -- the even input once, every
// link once (A(t) and B(t) read the same slice's links within a short window)
// and the output once -- instead of two full passes with the intermediate
// written to and read back from HBM.
#include <algorithm>

#include "weo_internal.h"

namespace weo {

struct FusedParams {
    int lxh, ly, lz, lt;
    int vs;          // sites of one parity in one t-slice
    int vh;
    int chunks;      // CTA-sized chunks per slice
    int ring;        // ring slots R (>= 3) for slices 1 .. Lt-2
    int total;       // items in the queue
    const float2 *in;
    float2 *out;
    float2 *tmp;     // (ring + 2) slots of [12][vs] complex64
    const char *gauge;
    long long gauge_pb;
    float a;         // -kappa^2
    unsigned int *ctrl;  // [0] sticky error (kept across launches), [1] ticket,
                         // [2] this launch's error, [3 .. 3+Lt) done A, [3+Lt .. 3+2Lt) done B
    unsigned int spin_limit;
    int inject;      // test of the failure path: first-hop items never publish completion
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ring_slot(const FusedParams &f, int t)
{
    return t == 0 ? 0 : (t == f.lt - 1 ? 1 : 2 + t % f.ring);
}

// slice task k -> (phase B?, t)
__device__ __forceinline__ void slice_task(const FusedParams &f, int k, bool &phase_b, int &t)
{
    const int L = f.lt;
    if (k == 0) {
        phase_b = false;
        t = L - 1;
    } else if (k == 1) {
        phase_b = false;
        t = 0;
    } else if (k < 2 * (L - 1)) {
        phase_b = k & 1;
        t = phase_b ? (k >> 1) - 1 : (k >> 1);
    } else {
        phase_b = true;
        t = k == 2 * (L - 1) ? L - 2 : L - 1;
    }
}

// Wait (thread 0) until ctrl[idx] >= target; false on timeout or a prior error.
__device__ __forceinline__ bool wait_count(const FusedParams &f, int idx, unsigned int target)
{
    unsigned int n = 0;
    while (ld_acquire(f.ctrl + idx) < target) {
        if (ld_acquire(f.ctrl + 2) != 0u) return false;
        if (++n > f.spin_limit) {
            atomicExch(f.ctrl + 2, 1u);
            atomicOr(f.ctrl + 0, 1u);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

template <class Lk, int MU, bool FWD, int S0, bool PB>
__device__ __forceinline__ void fused_dir(cx<float> acc[12], const FusedParams &f, int t_nb,
                                          long long nb_global, long long link_idx, int link_par)
{
    constexpr int S = FWD ? S0 : -S0;
    cx<float> U[3][3];
    Lk::load(f.gauge + (2 * MU + link_par) * f.gauge_pb, f.vh, link_idx, U);
    cx<float> v[12];
    if (PB) {
        // odd intermediate from the ring slot of slice t_nb, local index
        const float2 *base = f.tmp + (long long)ring_slot(f, t_nb) * 12 * f.vs;
        const long long local = nb_global - (long long)t_nb * f.vs;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 d = __ldcg(base + (long long)k * f.vs + local);
            v[k] = {d.x, d.y};
        }
    } else {
        SpF32::load(f.in, f.vh, nb_global, v);
    }
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

// One site of an A (PB = false: odd output into the ring) or B item (PB = true:
// even output with the axpy of Eq. 4).
template <class Lk, bool Dag, bool PB>
__device__ __forceinline__ void fused_site(const FusedParams &f, int t, int s)
{
    constexpr int S0 = Dag ? -1 : 1;
    const int out_parity = PB ? 0 : 1;
    const int in_par = out_parity ^ 1;
    int rem = s;
    const int xh = rem % f.lxh;
    rem /= f.lxh;
    const int y = rem % f.ly;
    const int z = rem / f.ly;
    const int par = (y + z + t + out_parity) & 1;
    const long long i = (long long)t * f.vs + s;
    const int sy = f.lxh, sz = f.lxh * f.ly;
    const int row = s - xh;
    const int xp = par ? (xh + 1 == f.lxh ? 0 : xh + 1) : xh;
    const int xm = par ? xh : (xh == 0 ? f.lxh - 1 : xh - 1);
    const long long base = (long long)t * f.vs;
    const long long n_xp = base + row + xp, n_xm = base + row + xm;
    const long long n_yp = base + s + (y + 1 == f.ly ? -(f.ly - 1) * sy : sy);
    const long long n_ym = base + s + (y == 0 ? (f.ly - 1) * sy : -sy);
    const long long n_zp = base + s + (z + 1 == f.lz ? -(f.lz - 1) * sz : sz);
    const long long n_zm = base + s + (z == 0 ? (f.lz - 1) * sz : -sz);
    const int tp = t + 1 == f.lt ? 0 : t + 1, tm = t == 0 ? f.lt - 1 : t - 1;
    const long long n_tp = (long long)tp * f.vs + s, n_tm = (long long)tm * f.vs + s;

    cx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
    fused_dir<Lk, 0, true, S0, PB>(acc, f, t, n_xp, i, out_parity);
    fused_dir<Lk, 0, false, S0, PB>(acc, f, t, n_xm, n_xm, in_par);
    fused_dir<Lk, 1, true, S0, PB>(acc, f, t, n_yp, i, out_parity);
    fused_dir<Lk, 1, false, S0, PB>(acc, f, t, n_ym, n_ym, in_par);
    fused_dir<Lk, 2, true, S0, PB>(acc, f, t, n_zp, i, out_parity);
    fused_dir<Lk, 2, false, S0, PB>(acc, f, t, n_zm, n_zm, in_par);
    fused_dir<Lk, 3, true, S0, PB>(acc, f, tp, n_tp, i, out_parity);
    fused_dir<Lk, 3, false, S0, PB>(acc, f, tm, n_tm, n_tm, in_par);

    if (PB) {
        cx<float> xv[12];
        SpF32::load(f.in, f.vh, i, xv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[k].r = fmaf(f.a, acc[k].r, xv[k].r);
            acc[k].i = fmaf(f.a, acc[k].i, xv[k].i);
        }
        SpF32::store(f.out, f.vh, i, acc);
    } else {
        float2 *dst = f.tmp + (long long)ring_slot(f, t) * 12 * f.vs;
#pragma unroll
        for (int k = 0; k < 12; ++k) __stcg(dst + (long long)k * f.vs + s, make_float2(acc[k].r, acc[k].i));
    }
}

template <class Lk, bool Dag, int THREADS>
__global__ void __launch_bounds__(THREADS) fused_meo_kernel(const FusedParams f)
{
    __shared__ int sh_item;
    __shared__ int sh_ok;
    const int L = f.lt;
    while (true) {
        if (threadIdx.x == 0) sh_item = (int)atomicAdd(f.ctrl + 1, 1u);
        __syncthreads();
        const int q = sh_item;
        if (q >= f.total) break;
        const int k = q / f.chunks, c = q - k * f.chunks;
        bool pb;
        int t;
        slice_task(f, k, pb, t);
        if (threadIdx.x == 0) {
            bool ok = true;
            const unsigned int full = (unsigned int)f.chunks;
            if (pb) {
                const int tm = t == 0 ? L - 1 : t - 1, tp = t + 1 == L ? 0 : t + 1;
                ok = wait_count(f, 3 + tm, full) && wait_count(f, 3 + t, full) &&
                     wait_count(f, 3 + tp, full);
            } else if (t >= 1 && t <= L - 2 && t - f.ring >= 1) {
                const int prev = t - f.ring;  // previous slice in this ring slot
                ok = wait_count(f, 3 + L + prev - 1, full) && wait_count(f, 3 + L + prev, full) &&
                     wait_count(f, 3 + L + prev + 1, full);
            }
            sh_ok = ok;
        }
        __syncthreads();
        if (!sh_ok) break;  // give up after a recorded error
        const int s = c * THREADS + threadIdx.x;
        if (s < f.vs) {
            if (pb) fused_site<Lk, Dag, true>(f, t, s);
            else fused_site<Lk, Dag, false>(f, t, s);
        }
        __syncthreads();
        if (threadIdx.x == 0 && !(f.inject && !pb)) {
            __threadfence();
            atomicAdd(f.ctrl + 3 + (pb ? L : 0) + t, 1u);
        }
    }
}

template <class Lk, bool Dag>
static int launch_fused_t(const FusedParams &f0, int threads, cudaStream_t s)
{
    FusedParams f = f0;
    f.chunks = (f.vs + threads - 1) / threads;
    f.total = 2 * f.lt * f.chunks;
    int dev = 0, sms = 0, per_sm = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (threads == 256) {
        WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_meo_kernel<Lk, Dag, 256>, 256, 0));
        fused_meo_kernel<Lk, Dag, 256><<<sms * per_sm, 256, 0, s>>>(f);
    } else {
        WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_meo_kernel<Lk, Dag, 128>, 128, 0));
        fused_meo_kernel<Lk, Dag, 128><<<sms * per_sm, 128, 0, s>>>(f);
    }
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <class Lk>
static int launch_fused_d(const FusedParams &f, bool dag, int threads, cudaStream_t s)
{
    return dag ? launch_fused_t<Lk, true>(f, threads, s) : launch_fused_t<Lk, false>(f, threads, s);
}

// Size the ring and control words (outside any stream capture).
int fused_prepare(wilson_eo_s *h, cudaStream_t s)
{
    const int L = h->dims[3];
    const long long vs = (long long)(h->dims[0] / 2) * h->dims[1] * h->dims[2];
    const int ring = std::max(3, h->fused_ring);
    WEO_TRY(h->fused_tmp.ensure((size_t)(2 + ring) * 12 * vs * sizeof(float2)));
    const size_t nctrl = (size_t)(3 + 2 * L);
    if (!h->fused_ctrl.ptr || h->fused_ctrl.bytes < nctrl * sizeof(unsigned int)) {
        WEO_TRY(h->fused_ctrl.ensure(nctrl * sizeof(unsigned int)));
        WEO_CUDA(cudaMemsetAsync(h->fused_ctrl.ptr, 0, nctrl * sizeof(unsigned int), s));
    }
    return WEO_OK;
}

// M_eo (or M_eo^dag) with FP32 spinors through the fused kernel, links from `g`
// (FP32, FP16 or BF16; 18 or 12 reals).
int meo_fused(wilson_eo_s *h, const PackedGauge &g, void *out, const void *in, bool dag,
              cudaStream_t s, bool inject_timeout)
{
    if (g.prec == WEO_F64) return set_error(WEO_ERR_UNSUPPORTED, "the fused kernel has FP32 arithmetic only");
    const int L = h->dims[3];
    FusedParams f;
    f.lxh = h->dims[0] / 2;
    f.ly = h->dims[1];
    f.lz = h->dims[2];
    f.lt = L;
    f.vs = f.lxh * f.ly * f.lz;
    f.vh = (int)h->vh;
    f.ring = std::max(3, h->fused_ring);
    const int threads = h->fused_threads == 256 ? 256 : 128;
    WEO_TRY(fused_prepare(h, s));
    const size_t nctrl = (size_t)(3 + 2 * L);
    // reset the ticket, this launch's error and the completion counters
    WEO_CUDA(cudaMemsetAsync(static_cast<unsigned int *>(h->fused_ctrl.ptr) + 1, 0,
                             (nctrl - 1) * sizeof(unsigned int), s));
    f.in = static_cast<const float2 *>(in);
    f.out = static_cast<float2 *>(out);
    f.tmp = static_cast<float2 *>(h->fused_tmp.ptr);
    f.gauge = static_cast<const char *>(g.buf.ptr);
    f.gauge_pb = g.pb;
    f.a = (float)(-h->kappa * h->kappa);
    f.ctrl = static_cast<unsigned int *>(h->fused_ctrl.ptr);
    f.spin_limit = 1u << 24;  // at least ~1 s of polling (64 ns sleeps) before giving up
    f.inject = inject_timeout ? 1 : 0;
    if (inject_timeout) f.spin_limit = 1u << 12;  // give up after ~0.3 ms
    f.chunks = f.total = 0;
    const bool c = g.fmt == WEO_LINK12;
    int tok = prof_begin(h, kernel_label("fused", g.prec, g.fmt, dag, true).c_str(), s);
    int st;
    switch (g.prec) {
    case WEO_F32: st = c ? launch_fused_d<LkF32_12>(f, dag, threads, s) : launch_fused_d<LkF32_18>(f, dag, threads, s); break;
    case WEO_F16: st = c ? launch_fused_d<LkH16_12>(f, dag, threads, s) : launch_fused_d<LkH16_18>(f, dag, threads, s); break;
    default: st = c ? launch_fused_d<LkB16_12>(f, dag, threads, s) : launch_fused_d<LkB16_18>(f, dag, threads, s); break;
    }
    prof_end(h, tok, s);
    return st;
}

// Sticky error word of the fused kernel (set when a bounded wait gave up):
// blocks on the stream, returns it and clears it.
int fused_take_error(wilson_eo_s *h, cudaStream_t s, unsigned int *err)
{
    *err = 0;
    if (!h->fused_ctrl.ptr) return WEO_OK;
    WEO_CUDA(cudaMemcpyAsync(err, h->fused_ctrl.ptr, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    WEO_CUDA(cudaStreamSynchronize(s));
    if (*err) WEO_CUDA(cudaMemsetAsync(h->fused_ctrl.ptr, 0, sizeof(unsigned int), s));
    return WEO_OK;
}

}  // namespace weo
