// Fused M_eo: both hops of Eq. 4 in one persistent launch over a wavefront of
// t-slices, each site computed by the same per-site code as the two-launch
// kernels.
//
// Work is a queue of items (hop, t-slice, CTA-sized chunk). Slice tasks are
// ordered as a wavefront over t with lookahead D:
//     A(Lt-1), A(0) .. A(D-1), A(D), B(0), A(D+1), B(1), ..., A(Lt-2), B(Lt-2-D), B(..), .., B(Lt-1)
// where A(t) = H_oe onto the odd sites of slice t (into the full-size odd
// intermediate) and B(t) = in - kappa^2 H_eo mid onto the even sites of slice t,
// which reads the intermediate at slices t-1, t and t+1. CTAs take items from an
// atomic ticket in queue order; B(t) waits until A(t-1), A(t) and A(t+1) are
// complete, A items never wait (every slice has its own intermediate storage).
// A ticket is only handed out after all earlier ones and every wait is for an
// earlier item, so the earliest unfinished item never waits and the queue
// always progresses. Every wait is bounded: after `spin_limit` polls the CTA
// records an error code and gives up, every other wait gives up as soon as it
// sees the error, and the host reports WEO_ERR_TIMEOUT.
//
// What this saves against two launches: B(t) runs D slices behind A, so the
// links of slice t, which A(t) read a few slices earlier, and the intermediate
// slices A just wrote are still in L2 when B reads them (with D = 1 the B items
// wait for A(t+1), issued just before them; D = 4..8 leaves no such stalls). DRAM sees the input,
// the links and the output about once, plus the write-back of the intermediate.
// The intermediate is read through L2 only (ld.global.cg): it is written during
// the launch, so a copy held in an SM's L1 could be stale.
#include <algorithm>

#include "weo_internal.h"
#include "weo_dslash.cuh"

namespace weo {

// Intermediate loaders that bypass L1 (same layouts as SpF32 and Sp16).
struct SpF32L2 : SpF32 {
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const float2 *p = static_cast<const float2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float2 d = __ldcg(p + k * vh + i);
            v[k] = {R(d.x), R(d.y)};
        }
    }
};

template <class Tr>
struct Sp16L2 : Sp16<Tr> {
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const uint4 *p = static_cast<const uint4 *>(base);
        const float n = __ldcg(reinterpret_cast<const float *>(p + 3 * vh) + i);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const uint4 w = __ldcg(p + q * vh + i);
            const float2 a = Tr::to_f2(w.x), b = Tr::to_f2(w.y), c = Tr::to_f2(w.z), d = Tr::to_f2(w.w);
            v[4 * q + 0] = {R(a.x * n), R(a.y * n)};
            v[4 * q + 1] = {R(b.x * n), R(b.y * n)};
            v[4 * q + 2] = {R(c.x * n), R(c.y * n)};
            v[4 * q + 3] = {R(d.x * n), R(d.y * n)};
        }
    }
};

struct FusedParams {
    HopParams a;     // H_oe: in (even) -> mid (odd)
    HopParams b;     // mid -> out (even), out = in + a * H_eo mid
    int vs;          // sites of one parity in one t-slice
    int lt;
    int lookahead;   // slices the first hop runs ahead of the second (1 .. Lt-1)
    int chunks;      // CTA-sized chunks per slice
    int total;       // items in the queue
    unsigned int *ctrl;  // [0] sticky error (kept across launches), [1] ticket,
                         // [2] this launch's error, [3 .. 3+Lt) chunks of A(t) done
    unsigned int spin_limit;
    int inject;      // test of the failure path: A items never publish completion
};

__device__ __forceinline__ unsigned int fused_ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (thread 0) until ctrl[idx] >= target; false on timeout or a prior error.
__device__ __forceinline__ bool fused_wait(const FusedParams &f, int idx, unsigned int target)
{
    unsigned int n = 0;
    while (fused_ld_acquire(f.ctrl + idx) < target) {
        if (fused_ld_acquire(f.ctrl + 2) != 0u) return false;
        if (++n > f.spin_limit) {
            atomicExch(f.ctrl + 2, 1u);
            atomicOr(f.ctrl + 0, 1u);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// slice task k -> (phase B?, t): A(Lt-1), A(0) .. A(D-1), then A(t+D) and B(t)
// in turn while t+D <= Lt-2, then the remaining B(t) (D = lookahead >= 1)
__device__ __forceinline__ void fused_task(int L, int D, int k, bool &phase_b, int &t)
{
    if (k == 0) {
        phase_b = false;
        t = L - 1;
        return;
    }
    if (k <= D) {
        phase_b = false;
        t = k - 1;
        return;
    }
    const int kp = k - (D + 1), pairs = L - 1 - D;
    if (kp < 2 * pairs) {
        phase_b = kp & 1;
        t = phase_b ? (kp >> 1) : (kp >> 1) + D;
    } else {
        phase_b = true;
        t = pairs + (kp - 2 * pairs);
    }
}

template <class SMid, class SMidL2, class LkA, class LkB, bool Dag, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) fused_meo_kernel(const FusedParams f)
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
        fused_task(L, f.lookahead, k, pb, t);
        if (threadIdx.x == 0) {
            bool ok = true;
            if (pb) {
                const unsigned int full = (unsigned int)f.chunks;
                const int tm = t == 0 ? L - 1 : t - 1, tp = t + 1 == L ? 0 : t + 1;
                ok = fused_wait(f, 3 + tm, full) && fused_wait(f, 3 + t, full) && fused_wait(f, 3 + tp, full);
            }
            sh_ok = ok;
        }
        __syncthreads();
        if (!sh_ok) break;  // give up after a recorded error
        const int s = c * THREADS + (int)threadIdx.x;
        if (s < f.vs) {
            const int i = t * f.vs + s;
            if (pb) hop_site<SMidL2, SpF32, SpF32, LkB, Dag, true, 1>(f.b, i, 0);
            else hop_site<SpF32, SMid, SpF32, LkA, Dag, false, 1>(f.a, i, 0);
        }
        __syncthreads();
        if (threadIdx.x == 0 && !pb && !f.inject) {
            __threadfence();
            atomicAdd(f.ctrl + 3 + t, 1u);
        }
    }
}

template <class SMid, class SMidL2, class LkA, class LkB, bool Dag, int THREADS, int MINB>
static int launch_fused_v(FusedParams f, int sms, cudaStream_t s)
{
    int per_sm = 0;
    auto kern = fused_meo_kernel<SMid, SMidL2, LkA, LkB, Dag, THREADS, MINB>;
    f.chunks = (f.vs + THREADS - 1) / THREADS;
    f.total = 2 * f.lt * f.chunks;
    WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0));
    if (per_sm < 1) return set_error(WEO_ERR_CUDA, "fused kernel cannot be resident");
    kern<<<sms * per_sm, THREADS, 0, s>>>(f);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

// 128 threads with six CTAs per SM (85 registers) or 256 threads with three:
// both measured faster than the 64-register cap of the two-launch kernels,
// which makes this kernel (both hops' code in one body) spill heavily.
template <class SMid, class SMidL2, class LkA, class LkB, bool Dag>
static int launch_fused_t(FusedParams f, int threads, cudaStream_t s)
{
    int dev = 0, sms = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (threads == 256) return launch_fused_v<SMid, SMidL2, LkA, LkB, Dag, 256, 3>(f, sms, s);
    return launch_fused_v<SMid, SMidL2, LkA, LkB, Dag, 128, 6>(f, sms, s);
}

// The first hop reads the links with L2 retention (the second hop of the same
// slice reads them again a few slices later), the second with evict-first.
template <class SMid, class SMidL2, template <class> class LkOf>
static int launch_fused_d(const FusedParams &f, bool dag, int threads, cudaStream_t s)
{
    using LkA = LkOf<LdL2>;
    using LkB = LkOf<LdStream>;
    return dag ? launch_fused_t<SMid, SMidL2, LkA, LkB, true>(f, threads, s)
               : launch_fused_t<SMid, SMidL2, LkA, LkB, false>(f, threads, s);
}

template <class Ld> using LkH16_18_ = Lk16_18<H16Traits, Ld>;
template <class Ld> using LkH16_12_ = Lk16_12<H16Traits, Ld>;
template <class Ld> using LkB16_18_ = Lk16_18<B16Traits, Ld>;
template <class Ld> using LkB16_12_ = Lk16_12<B16Traits, Ld>;

// M_eo (or M_eo^dag) of one right-hand side with FP32 spinors through the
// fused kernel, links from `g` (FP32 with an FP32 intermediate, or FP16 /
// BF16 with a 16-bit intermediate as in the two-launch path). `mid` holds the
// odd intermediate (96 or 52 bytes per odd site).
int meo_fused(wilson_eo_s *h, const PackedGauge &g, void *mid, void *out, const void *in, bool dag,
              cudaStream_t s, bool inject_timeout)
{
    if (g.prec == WEO_F64) return set_error(WEO_ERR_UNSUPPORTED, "the fused M_eo has FP32 arithmetic only");
    const int L = h->dims[3];
    WEO_TRY(fused_prepare(h, s));
    const size_t nctrl = (size_t)(3 + L);
    // reset the ticket, this launch's error and the completion counters
    WEO_CUDA(cudaMemsetAsync(static_cast<unsigned int *>(h->fused_ctrl.ptr) + 1, 0,
                             (nctrl - 1) * sizeof(unsigned int), s));
    FusedParams f;
    HopParams p = geom_params(h);
    p.nrhs = 1;
    p.gauge = static_cast<const char *>(g.buf.ptr);
    p.gauge_pb = g.pb;
    const long long ext = h->vh * 96;
    const long long mid_ext = h->vh * (g.prec == WEO_F32 ? 96 : spinor_site_bytes(SK_H16));
    p.reverse = 0;
    p.out_parity = 1;
    p.in = in;
    p.in_stride = ext;
    p.out = mid;
    p.out_stride = mid_ext;
    p.x = nullptr;
    p.x_stride = 0;
    p.a = 0.0;
    f.a = p;
    p.out_parity = 0;
    p.in = mid;
    p.in_stride = mid_ext;
    p.out = out;
    p.out_stride = ext;
    p.x = in;
    p.x_stride = ext;
    p.a = -h->kappa * h->kappa;
    f.b = p;
    f.vs = (h->dims[0] / 2) * h->dims[1] * h->dims[2];
    f.lt = L;
    f.lookahead = std::max(1, std::min(h->fused_lookahead, L - 1));
    f.chunks = f.total = 0;
    f.ctrl = static_cast<unsigned int *>(h->fused_ctrl.ptr);
    f.spin_limit = 1u << 24;  // at least ~1 s of polling (64 ns sleeps) before giving up
    f.inject = inject_timeout ? 1 : 0;
    if (inject_timeout) f.spin_limit = 1u << 12;  // give up after ~0.3 ms
    const int threads = h->fused_threads == 256 ? 256 : 128;
    const bool c = g.fmt == WEO_LINK12;
    int tok = prof_begin(h, kernel_label("fused", g.prec, g.fmt, dag, true).c_str(), s);
    int st;
    switch (g.prec) {
    case WEO_F32:
        st = c ? launch_fused_d<SpF32, SpF32L2, LkF32_12T>(f, dag, threads, s)
               : launch_fused_d<SpF32, SpF32L2, LkF32_18T>(f, dag, threads, s);
        break;
    case WEO_F16:
        st = c ? launch_fused_d<SpH16, Sp16L2<H16Traits>, LkH16_12_>(f, dag, threads, s)
               : launch_fused_d<SpH16, Sp16L2<H16Traits>, LkH16_18_>(f, dag, threads, s);
        break;
    default:
        st = c ? launch_fused_d<SpB16, Sp16L2<B16Traits>, LkB16_12_>(f, dag, threads, s)
               : launch_fused_d<SpB16, Sp16L2<B16Traits>, LkB16_18_>(f, dag, threads, s);
        break;
    }
    prof_end(h, tok, s);
    return st;
}

// Control words (outside any stream capture).
int fused_prepare(wilson_eo_s *h, cudaStream_t s)
{
    const size_t nctrl = (size_t)(3 + h->dims[3]);
    if (!h->fused_ctrl.ptr || h->fused_ctrl.bytes < nctrl * sizeof(unsigned int)) {
        WEO_TRY(h->fused_ctrl.ensure(nctrl * sizeof(unsigned int)));
        WEO_CUDA(cudaMemsetAsync(h->fused_ctrl.ptr, 0, nctrl * sizeof(unsigned int), s));
    }
    return WEO_OK;
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
