// Solvers for M_eo^dag M_eo x = b (the normal equations of Eq. 4's even system;
// the paper's Sec. 2 notes that the solver's speed is set by the matrix
// multiplication), for one or several right-hand sides at once.
//
//  * plain FP64 conjugate gradient: every vector, operator and reduction in FP64;
//  * mixed precision: CG iterated with an FP32 or 16-bit-storage operator and
//    FP32 vectors, with reliable updates (Clark et al., "Solving lattice QCD
//    systems of equations using mixed precision solvers on GPUs", 2010): when
//    the iterated residual has dropped by `delta` since the last update, the
//    low-precision solution increment is added to the FP64 solution, and the
//    residual is recomputed from scratch in FP64 as b - A x with the FP64
//    operator. The search direction is kept. Convergence is declared on that
//    FP64 true residual only.
//
// Several right-hand sides run as independent CGs in lockstep: every operator
// application covers all of them (the multi-RHS hop kernels read each link once
// for a block of right-hand sides), every BLAS-1 kernel and reduction is a 2-D
// grid over (elements, right-hand side), and each right-hand side has its own
// scalars, convergence flag and restarts.
//
// All scalars (rho, alpha, beta) live on the device: the last block of each
// reduction finishes it and derives the next scalar, so an iteration is a fixed
// sequence of kernel launches with no host round trip. Iterations run in chunks
// captured once as a CUDA graph and replayed; the host reads the residual norms
// only between chunks. Reductions are deterministic (fixed grid, partial sums
// added in block order).
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <chrono>
#include <vector>

#include "weo_internal.h"

namespace weo {

constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;
constexpr int kMaxBreakdowns = 64;  // direction restarts before a solve gives up
constexpr int kMaxRhs = 64;
// a true residual this many times above the smallest one seen means the
// low-precision iteration is diverging from the FP64 system: give up
constexpr double kDivergence = 1e4;

struct SolveScalars {
    double rr;       // |r|^2 of the iterated residual
    double pAp;      // Re <p, A p>
    double alpha;
    double beta;
    double red;      // result of the last plain reduction
    int nonfinite;   // set when a reduction or a scalar is NaN / Inf or pAp <= 0
    int active;      // 0 once this right-hand side has converged
    unsigned int counter;
    unsigned int pad;
    double partial[kRedBlocks];
};
constexpr size_t kHead = offsetof(SolveScalars, counter);

struct SolverState {
    Buffer scal;                     // nrhs x SolveScalars on the device
    SolveScalars *host = nullptr;    // pinned mirror of the heads (kMaxRhs entries)
    Buffer x64, b64, r64, e64, t64, odd64;     // FP64 work vectors
    Buffer xs, rs, p, Ap, t32, oddlo;          // low-precision work vectors
    Buffer p64, Ap64;                          // plain FP64 CG
    Buffer xff, eff, tff, oddff;               // float-float true residuals
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [mixed]
    int graph_chunk[2] = {0, 0};
    int graph_nrhs[2] = {0, 0};
    double delta = 0.1;
    int chunk = 8;
    int use_graphs = 1;
    int nrhs = 1;                    // right-hand sides of the current solve
    int ff_residual = 1;             // mixed mode: reliable updates with the float-float operator
    // mixed mode, direction after a reliable update: 0 keep, 1 restart, 2 restart
    // when the inner operator stores BF16 (measured: with 2^-9 link rounding the
    // kept directions diverge at 48^3 x 96, kappa = 0.135, restarted ones converge)
    int restart_on_update = 2;
    // statistics of the last solve
    int iterations = 0, reliable_updates = 0, hi_applies = 0, ff_applies = 0;
    double seconds = 0.0;
};

// ---------------------------------------------------------------- kernels --
// Every kernel is a 2-D grid: blockIdx.y selects the right-hand side, whose
// vectors start at offset rhs * n and whose scalars are sc[rhs].

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (int)threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

// Store this block's partial; the last block sums all partials in block order.
// Returns true in every thread of the last block; *total is valid in thread 0.
__device__ __forceinline__ bool finish_reduction(SolveScalars *sc, double block_val, double *total)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        sc->partial[blockIdx.x] = block_val;
        __threadfence();
        const unsigned int ticket = atomicAdd(&sc->counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x)
        v += reinterpret_cast<volatile double *>(sc->partial)[k];
    v = block_sum(v);
    if (threadIdx.x == 0) {
        *total = v;
        sc->counter = 0;
    }
    return true;
}

template <typename T2>
__device__ __forceinline__ double re_dot(T2 a, T2 b) { return double(a.x) * b.x + double(a.y) * b.y; }

#define FOR_ELEMENTS(k) \
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)

// FP32 vectors are read as float4 (two complex numbers; n = 12 V/2 is even and
// every right-hand side starts on a 16-byte boundary). Squares are summed in
// FP32 over the handful of values one thread has in flight and only those
// group sums are accumulated in FP64: per-element FP64 arithmetic would run at
// the FP64 rate, a small fraction of the FP32 one, and would bound these
// otherwise memory-bound kernels.
__device__ __forceinline__ float sq4(float4 q) { return q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w; }

__device__ __forceinline__ long long grid_stride() { return (long long)gridDim.x * blockDim.x; }
__device__ __forceinline__ long long grid_index() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }

// sum of |a_k|^2 over n complex values, this thread's share
template <typename T2>
__device__ __forceinline__ double sum_sq(const T2 *a, long long n)
{
    double v = 0.0;
    if constexpr (std::is_same<T2, float2>::value) {
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const long long n4 = n >> 1, st = grid_stride();
        long long k = grid_index();
        for (; k + 3 * st < n4; k += 4 * st) {
            const float4 q0 = a4[k], q1 = a4[k + st], q2 = a4[k + 2 * st], q3 = a4[k + 3 * st];
            v += double((sq4(q0) + sq4(q1)) + (sq4(q2) + sq4(q3)));
        }
        for (; k < n4; k += st) v += double(sq4(a4[k]));
    } else {
        FOR_ELEMENTS(k) v += re_dot(a[k], a[k]);
    }
    return v;
}

// mode 0: red = |a|^2 (every right-hand side);  mode 1: rr = |a|^2 (active
// ones);  mode 2: pAp = |a|^2 and alpha = rr / pAp (active, finite ones).
// The solver calls mode 2 with a = M p: for A = M^dag M, <p, A p> = |M p|^2,
// which reads one vector instead of two and cannot come out negative when the
// low-precision M and M^dag are not exact adjoints of each other.
template <typename T2>
__global__ void __launch_bounds__(kRedThreads) k_norm2(const T2 *a, long long n, SolveScalars *scs,
                                                       int mode)
{
    SolveScalars *sc = scs + blockIdx.y;
    if (mode >= 1 && !sc->active) return;
    if (mode == 2 && sc->nonfinite) return;
    double v = block_sum(sum_sq(a + blockIdx.y * n, n));
    double tot;
    if (finish_reduction(sc, v, &tot) && threadIdx.x == 0) {
        if (mode == 0) {
            sc->red = tot;
        } else if (mode == 1) {
            sc->rr = tot;
            if (!isfinite(tot)) sc->nonfinite = 1;
        } else {
            sc->pAp = tot;
            const double alpha = sc->rr / tot;
            if (!isfinite(tot) || !(tot > 0.0) || !isfinite(alpha)) sc->nonfinite = 1;
            else sc->alpha = alpha;
        }
    }
}

__device__ __forceinline__ void axpy4(float4 &y, float a, float4 x)
{
    y.x += a * x.x;
    y.y += a * x.y;
    y.z += a * x.z;
    y.w += a * x.w;
}

// r -= alpha Ap ; rr_new = |r|^2 ; beta = rr_new / rr ; rr = rr_new
// (x += alpha p is done by k_cg_dir, which reads p anyway)
template <typename T2>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(T2 *r, const T2 *Ap, long long n,
                                                           SolveScalars *scs)
{
    SolveScalars *sc = scs + blockIdx.y;
    if (!sc->active || sc->nonfinite) return;
    using T = decltype(T2().x);
    const long long o = blockIdx.y * n;
    r += o;
    Ap += o;
    const T alpha = T(sc->alpha);
    double v = 0.0;
    if constexpr (std::is_same<T2, float2>::value) {
        float4 *r4 = reinterpret_cast<float4 *>(r);
        const float4 *a4 = reinterpret_cast<const float4 *>(Ap);
        const long long n4 = n >> 1, st = grid_stride();
        long long k = grid_index();
        for (; k + 3 * st < n4; k += 4 * st) {
            float4 r0 = r4[k], r1 = r4[k + st], r2 = r4[k + 2 * st], r3 = r4[k + 3 * st];
            axpy4(r0, -alpha, a4[k]);
            axpy4(r1, -alpha, a4[k + st]);
            axpy4(r2, -alpha, a4[k + 2 * st]);
            axpy4(r3, -alpha, a4[k + 3 * st]);
            r4[k] = r0;
            r4[k + st] = r1;
            r4[k + 2 * st] = r2;
            r4[k + 3 * st] = r3;
            v += double((sq4(r0) + sq4(r1)) + (sq4(r2) + sq4(r3)));
        }
        for (; k < n4; k += st) {
            float4 r0 = r4[k];
            axpy4(r0, -alpha, a4[k]);
            r4[k] = r0;
            v += double(sq4(r0));
        }
    } else {
        FOR_ELEMENTS(k) {
            T2 rv = r[k];
            const T2 av = Ap[k];
            rv.x -= alpha * av.x;
            rv.y -= alpha * av.y;
            r[k] = rv;
            v += re_dot(rv, rv);
        }
    }
    v = block_sum(v);
    double tot;
    if (finish_reduction(sc, v, &tot) && threadIdx.x == 0) {
        if (!isfinite(tot) || !isfinite(tot / sc->rr)) {
            sc->nonfinite = 1;
        } else {
            sc->beta = tot / sc->rr;
            sc->rr = tot;
        }
    }
}

// x += alpha p ; p = r + beta p
template <typename T2>
__global__ void __launch_bounds__(kRedThreads) k_cg_dir(T2 *x, T2 *p, const T2 *r, long long n,
                                                        const SolveScalars *scs)
{
    const SolveScalars *sc = scs + blockIdx.y;
    if (!sc->active || sc->nonfinite) return;
    using T = decltype(T2().x);
    const long long o = blockIdx.y * n;
    x += o;
    p += o;
    r += o;
    const T alpha = T(sc->alpha), beta = T(sc->beta);
    if constexpr (std::is_same<T2, float2>::value) {
        float4 *x4 = reinterpret_cast<float4 *>(x), *p4 = reinterpret_cast<float4 *>(p);
        const float4 *r4 = reinterpret_cast<const float4 *>(r);
        const long long n4 = n >> 1, st = grid_stride();
        long long k = grid_index();
        for (; k + st < n4; k += 2 * st) {
            const float4 q0 = p4[k], q1 = p4[k + st];
            float4 x0 = x4[k], x1 = x4[k + st], y0 = r4[k], y1 = r4[k + st];
            axpy4(x0, alpha, q0);
            axpy4(x1, alpha, q1);
            axpy4(y0, beta, q0);
            axpy4(y1, beta, q1);
            x4[k] = x0;
            x4[k + st] = x1;
            p4[k] = y0;
            p4[k + st] = y1;
        }
        if (k < n4) {
            const float4 q0 = p4[k];
            float4 x0 = x4[k], y0 = r4[k];
            axpy4(x0, alpha, q0);
            axpy4(y0, beta, q0);
            x4[k] = x0;
            p4[k] = y0;
        }
    } else {
        FOR_ELEMENTS(k) {
            const T2 pv = p[k], rv = r[k];
            T2 xv = x[k];
            xv.x += alpha * pv.x;
            xv.y += alpha * pv.y;
            x[k] = xv;
            T2 q;
            q.x = rv.x + beta * pv.x;
            q.y = rv.y + beta * pv.y;
            p[k] = q;
        }
    }
}

// r = b - t ; red = |r|^2 (every right-hand side)
__global__ void __launch_bounds__(kRedThreads) k_residual(double2 *r, const double2 *b,
                                                          const double2 *t, long long n,
                                                          SolveScalars *scs)
{
    SolveScalars *sc = scs + blockIdx.y;
    const long long o = blockIdx.y * n;
    r += o;
    b += o;
    t += o;
    double v = 0.0;
    FOR_ELEMENTS(k) {
        double2 rv = make_double2(b[k].x - t[k].x, b[k].y - t[k].y);
        r[k] = rv;
        v += rv.x * rv.x + rv.y * rv.y;
    }
    v = block_sum(v);
    double tot;
    if (finish_reduction(sc, v, &tot) && threadIdx.x == 0) sc->red = tot;
}

// r = b - t with t in float-float (SpFF: 12 planes of high parts, then 12 of
// low parts per right-hand side) ; red = |r|^2 (every right-hand side)
__global__ void __launch_bounds__(kRedThreads) k_residual_ff(double2 *r, const double2 *b,
                                                             const float2 *t, long long n,
                                                             SolveScalars *scs)
{
    SolveScalars *sc = scs + blockIdx.y;
    const long long o = blockIdx.y * n;
    r += o;
    b += o;
    t += 2 * o;
    double v = 0.0;
    FOR_ELEMENTS(k) {
        const float2 hi = t[k], lo = t[n + k];
        const double2 bv = b[k];
        const double2 rv = make_double2((bv.x - double(hi.x)) - double(lo.x), (bv.y - double(hi.y)) - double(lo.y));
        r[k] = rv;
        v += rv.x * rv.x + rv.y * rv.y;
    }
    v = block_sum(v);
    double tot;
    if (finish_reduction(sc, v, &tot) && threadIdx.x == 0) sc->red = tot;
}

// d = s over all right-hand sides (n_total elements)
template <typename D2, typename S2>
__global__ void k_convert(D2 *d, const S2 *s, long long n)
{
    FOR_ELEMENTS(k) {
        const S2 v = s[k];
        D2 o;
        o.x = v.x;
        o.y = v.y;
        d[k] = o;
    }
}

// x64 += xs ; xs = 0 (n_total elements)
__global__ void k_accumulate(double2 *x, float2 *xs, long long n)
{
    FOR_ELEMENTS(k) {
        const float2 v = xs[k];
        double2 a = x[k];
        a.x += v.x;
        a.y += v.y;
        x[k] = a;
        xs[k] = make_float2(0.f, 0.f);
    }
}

static unsigned red_grid(long long n)
{
    long long b = (n + kRedThreads - 1) / kRedThreads;
    return (unsigned)(b < kRedBlocks ? (b < 1 ? 1 : b) : kRedBlocks);
}

static unsigned flat_grid(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)std::min<long long>(std::max<long long>(b, 1), 65535LL * 8);
}

// ------------------------------------------------------------------ state --

void solver_destroy(wilson_eo_s *h)
{
    SolverState *S = h->solver;
    if (!S) return;
    for (auto &g : S->graph)
        if (g) cudaGraphExecDestroy(g);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->host) cudaFreeHost(S->host);
    Buffer *bufs[] = {&S->scal, &S->x64, &S->b64, &S->r64, &S->e64, &S->t64, &S->odd64,
                      &S->xs, &S->rs, &S->p, &S->Ap, &S->t32, &S->oddlo, &S->p64, &S->Ap64,
                      &S->xff, &S->eff, &S->tff, &S->oddff};
    for (Buffer *b : bufs) b->release();
    delete S;
    h->solver = nullptr;
}

static int solver_state(wilson_eo_s *h, SolverState **out)
{
    if (!h->solver) {
        SolverState *S = new SolverState();
        h->solver = S;
        cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
        e = cudaMallocHost(&S->host, sizeof(SolveScalars) * kMaxRhs);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMallocHost", __FILE__, __LINE__);
        WEO_TRY(S->scal.ensure(sizeof(SolveScalars) * kMaxRhs));
        WEO_CUDA(cudaMemsetAsync(S->scal.ptr, 0, sizeof(SolveScalars) * kMaxRhs, S->stream));
    }
    *out = h->solver;
    return WEO_OK;
}

static SolveScalars *dev_scal(SolverState *S) { return static_cast<SolveScalars *>(S->scal.ptr); }

// heads of every right-hand side's scalars into S->host (blocking)
static int read_scalars(SolverState *S)
{
    WEO_CUDA(cudaMemcpy2DAsync(S->host, sizeof(SolveScalars), S->scal.ptr, sizeof(SolveScalars), kHead,
                               S->nrhs, cudaMemcpyDeviceToHost, S->stream));
    WEO_CUDA(cudaStreamSynchronize(S->stream));
    return WEO_OK;
}

static int set_flag(SolverState *S, int rhs, size_t offset, int value)
{
    // a tiny host-to-device write of one int field of sc[rhs]
    char *dst = static_cast<char *>(S->scal.ptr) + rhs * sizeof(SolveScalars) + offset;
    static const int vals[2] = {0, 1};
    WEO_CUDA(cudaMemcpyAsync(dst, &vals[value ? 1 : 0], sizeof(int), cudaMemcpyHostToDevice, S->stream));
    return WEO_OK;
}

// After a chunk of fused-operator iterations: did a bounded wait give up?
static int check_fused(wilson_eo_s *h, SolverState *S)
{
    if (h->algo != 1) return WEO_OK;
    unsigned int err = 0;
    WEO_TRY(fused_take_error(h, S->stream, &err));
    if (err) return set_error(WEO_ERR_TIMEOUT, "a bounded wait in the fused M_eo kernel gave up during the solve");
    return WEO_OK;
}

// FP64 packed gauge for true residuals (the handle's own if it is FP64)
static int hi_gauge(wilson_eo_s *h, const PackedGauge **g, cudaStream_t s)
{
    if (h->prec == WEO_F64) {
        *g = &h->gauge;
        return WEO_OK;
    }
    if (!h->gauge_f64.valid)
        WEO_TRY(pack_gauge(h, h->gauge_f64, WEO_F64, WEO_LINK18, h->canon_gauge.ptr, h->canon_is_f64, s));
    *g = &h->gauge_f64;
    return WEO_OK;
}

// low-precision operator for the mixed solver: FP32 for an FP64 handle
static int lo_gauge(wilson_eo_s *h, const PackedGauge **g, cudaStream_t s)
{
    if (h->prec != WEO_F64) {
        *g = &h->gauge;
        return WEO_OK;
    }
    if (!h->gauge_lo.valid)
        WEO_TRY(pack_gauge(h, h->gauge_lo, WEO_F32, h->fmt, h->canon_gauge.ptr, h->canon_is_f64, s));
    *g = &h->gauge_lo;
    return WEO_OK;
}

// A v = M^dag (M v) with gauge g for all right-hand sides
static int normal_op(wilson_eo_s *h, SolverState *S, const PackedGauge &g, Buffer &odd, void *e,
                     void *out, const void *v, cudaStream_t s)
{
    WEO_TRY(meo_with(h, g, odd, e, v, S->nrhs, false, s));
    return meo_with(h, g, odd, out, e, S->nrhs, true, s);
}

// One CG iteration of every right-hand side. mixed: low-precision vectors
// (float2) with operator g; otherwise FP64 vectors.
static int cg_iteration(wilson_eo_s *h, SolverState *S, const PackedGauge &g, bool mixed,
                        cudaStream_t s)
{
    const long long n = 12 * h->vh;
    const dim3 grid(red_grid(n), S->nrhs);
    SolveScalars *sc = dev_scal(S);
    if (mixed) {
        WEO_TRY(normal_op(h, S, g, S->oddlo, S->t32.ptr, S->Ap.ptr, S->p.ptr, s));
        k_norm2<float2><<<grid, kRedThreads, 0, s>>>((const float2 *)S->t32.ptr, n, sc, 2);
        k_cg_update<float2><<<grid, kRedThreads, 0, s>>>((float2 *)S->rs.ptr, (const float2 *)S->Ap.ptr, n, sc);
        k_cg_dir<float2><<<grid, kRedThreads, 0, s>>>((float2 *)S->xs.ptr, (float2 *)S->p.ptr,
                                                       (const float2 *)S->rs.ptr, n, sc);
    } else {
        WEO_TRY(normal_op(h, S, g, S->odd64, S->e64.ptr, S->Ap64.ptr, S->p64.ptr, s));
        k_norm2<double2><<<grid, kRedThreads, 0, s>>>((const double2 *)S->e64.ptr, n, sc, 2);
        k_cg_update<double2><<<grid, kRedThreads, 0, s>>>((double2 *)S->r64.ptr, (const double2 *)S->Ap64.ptr, n, sc);
        k_cg_dir<double2><<<grid, kRedThreads, 0, s>>>((double2 *)S->x64.ptr, (double2 *)S->p64.ptr,
                                                        (const double2 *)S->r64.ptr, n, sc);
    }
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

// Run `k` iterations, from a captured graph when enabled.
static int cg_chunk(wilson_eo_s *h, SolverState *S, const PackedGauge &g, bool mixed, int k)
{
    cudaStream_t s = S->stream;
    if (!S->use_graphs) {
        for (int i = 0; i < k; ++i) WEO_TRY(cg_iteration(h, S, g, mixed, s));
        return WEO_OK;
    }
    const int gi = mixed ? 1 : 0;
    if (!S->graph[gi] || S->graph_chunk[gi] != k || S->graph_nrhs[gi] != S->nrhs) {
        if (S->graph[gi]) {
            cudaGraphExecDestroy(S->graph[gi]);
            S->graph[gi] = nullptr;
        }
        // profiling events are not recorded into the graph
        Profiler *saved = h->prof;
        h->prof = nullptr;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            h->prof = saved;
            return fail_cuda(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        }
        int st = WEO_OK;
        for (int i = 0; i < k && st == WEO_OK; ++i) st = cg_iteration(h, S, g, mixed, s);
        e = cudaStreamEndCapture(s, &graph);
        h->prof = saved;
        if (st != WEO_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&S->graph[gi], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            S->graph[gi] = nullptr;
            return fail_cuda(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        S->graph_chunk[gi] = k;
        S->graph_nrhs[gi] = S->nrhs;
    }
    WEO_CUDA(cudaGraphLaunch(S->graph[gi], s));
    return WEO_OK;
}

// r64 = b64 - A x64 with the FP64 operator for every right-hand side;
// |r|^2 of each lands in S->host[rhs].red
static int true_residual(wilson_eo_s *h, SolverState *S, const PackedGauge &ghi)
{
    cudaStream_t s = S->stream;
    const long long n = 12 * h->vh;
    WEO_TRY(normal_op(h, S, ghi, S->odd64, S->e64.ptr, S->t64.ptr, S->x64.ptr, s));
    k_residual<<<dim3(red_grid(n), S->nrhs), kRedThreads, 0, s>>>(
        (double2 *)S->r64.ptr, (const double2 *)S->b64.ptr, (const double2 *)S->t64.ptr, n, dev_scal(S));
    WEO_CUDA(cudaGetLastError());
    S->hi_applies += 1;
    return read_scalars(S);
}

// The same with the float-float operator (about 48 significant bits from FP32
// arithmetic, several times the FP64 pipe's rate on GB300): x64 is split into
// float-float, A x is formed in float-float, and r = b - A x in FP64.
static int true_residual_ff(wilson_eo_s *h, SolverState *S)
{
    cudaStream_t s = S->stream;
    const long long n = 12 * h->vh;
    const size_t bytes = (size_t)h->vh * 192 * S->nrhs;
    const PackedGauge *gff = nullptr;
    WEO_TRY(ff_gauge(h, &gff, s));
    WEO_TRY(S->xff.ensure(bytes));
    WEO_TRY(S->eff.ensure(bytes));
    WEO_TRY(S->tff.ensure(bytes));
    WEO_TRY(ff_from_f64(S->xff.ptr, S->x64.ptr, h->vh, S->nrhs, s));
    WEO_TRY(normal_op(h, S, *gff, S->oddff, S->eff.ptr, S->tff.ptr, S->xff.ptr, s));
    k_residual_ff<<<dim3(red_grid(n), S->nrhs), kRedThreads, 0, s>>>(
        (double2 *)S->r64.ptr, (const double2 *)S->b64.ptr, (const float2 *)S->tff.ptr, n, dev_scal(S));
    WEO_CUDA(cudaGetLastError());
    S->ff_applies += 1;
    return read_scalars(S);
}

// True residual of a reliable update: float-float when enabled, and then, if
// any active system looks converged, once more with the native FP64 operator,
// so that convergence is only ever declared on an FP64 true residual.
static int update_residual(wilson_eo_s *h, SolverState *S, const PackedGauge &ghi, bool ff,
                           const std::vector<int> &active, const std::vector<double> &target)
{
    if (!ff) return true_residual(h, S, ghi);
    WEO_TRY(true_residual_ff(h, S));
    bool converged = false;
    for (int r = 0; r < S->nrhs; ++r)
        if (active[r] && S->host[r].red <= target[r]) converged = true;
    return converged ? true_residual(h, S, ghi) : WEO_OK;
}

static int solve_impl(wilson_eo_s *h, double tol, int maxiter, int mixed, int *iters_out,
                      double *relres_out)
{
    SolverState *S = h->solver;
    cudaStream_t s = S->stream;
    const int R = S->nrhs;
    const long long n = 12 * h->vh, nt = n * R;
    const size_t b64 = (size_t)nt * 16, b32 = (size_t)nt * 8, v64 = (size_t)n * 16, v32 = (size_t)n * 8;
    const dim3 grid(red_grid(n), R);
    SolveScalars *sc = dev_scal(S);
    const PackedGauge *ghi = nullptr, *glo = nullptr;
    WEO_TRY(hi_gauge(h, &ghi, s));
    WEO_TRY(S->r64.ensure(b64));
    WEO_TRY(S->e64.ensure(b64));
    WEO_TRY(S->t64.ensure(b64));
    // reset every right-hand side's scalars and mark them active
    WEO_CUDA(cudaMemsetAsync(sc, 0, sizeof(SolveScalars) * R, s));
    for (int r = 0; r < R; ++r) WEO_TRY(set_flag(S, r, offsetof(SolveScalars, active), 1));
    S->iterations = S->reliable_updates = S->hi_applies = S->ff_applies = 0;
    const bool ff = mixed && S->ff_residual;
    std::vector<int> active(R, 1), iters(R, 0);
    std::vector<double> target(R), rr_true(R), r_max(R), rr_min(R);

    // |b|^2 of every right-hand side
    k_norm2<double2><<<grid, kRedThreads, 0, s>>>((const double2 *)S->b64.ptr, n, sc, 0);
    WEO_CUDA(cudaGetLastError());
    WEO_TRY(read_scalars(S));
    std::vector<double> bb(R);
    for (int r = 0; r < R; ++r) {
        bb[r] = S->host[r].red;
        if (!isfinite(bb[r])) return set_error(WEO_ERR_NONFINITE, "non-finite right-hand side");
        target[r] = tol * tol * bb[r];
    }

    // b = 0: x = 0 is exact
    for (int r = 0; r < R; ++r)
        if (bb[r] == 0.0)
            WEO_CUDA(cudaMemsetAsync(static_cast<char *>(S->x64.ptr) + r * v64, 0, v64, s));
    // a zero initial guess needs no operator application: r = b
    k_norm2<double2><<<grid, kRedThreads, 0, s>>>((const double2 *)S->x64.ptr, n, sc, 0);
    WEO_CUDA(cudaGetLastError());
    WEO_TRY(read_scalars(S));
    bool zero_guess = true;
    for (int r = 0; r < R; ++r)
        if (S->host[r].red != 0.0) zero_guess = false;
    if (zero_guess) {
        WEO_CUDA(cudaMemcpyAsync(S->r64.ptr, S->b64.ptr, b64, cudaMemcpyDeviceToDevice, s));
        for (int r = 0; r < R; ++r) S->host[r].red = bb[r];
    } else {
        WEO_TRY(update_residual(h, S, *ghi, ff, active, target));
    }
    int n_active = R;
    auto retire = [&](int r) -> int {  // right-hand side r has converged
        active[r] = 0;
        iters[r] = S->iterations;
        --n_active;
        return set_flag(S, r, offsetof(SolveScalars, active), 0);
    };
    for (int r = 0; r < R; ++r) {
        rr_true[r] = S->host[r].red;
        if (!isfinite(rr_true[r])) return set_error(WEO_ERR_NONFINITE, "non-finite initial residual");
        r_max[r] = sqrt(rr_true[r]);
        rr_min[r] = rr_true[r];
        if (bb[r] == 0.0 || rr_true[r] <= target[r]) WEO_TRY(retire(r));
    }
    int breakdowns = 0;

    if (!mixed) {
        WEO_TRY(S->p64.ensure(b64));
        WEO_TRY(S->Ap64.ensure(b64));
        WEO_CUDA(cudaMemcpyAsync(S->p64.ptr, S->r64.ptr, b64, cudaMemcpyDeviceToDevice, s));
        k_norm2<double2><<<grid, kRedThreads, 0, s>>>((const double2 *)S->r64.ptr, n, sc, 1);
        WEO_CUDA(cudaGetLastError());
        while (n_active > 0 && S->iterations < maxiter) {
            const int k = std::min(S->chunk, maxiter - S->iterations);
            WEO_TRY(cg_chunk(h, S, *ghi, false, k));
            S->iterations += k;
            WEO_TRY(read_scalars(S));
            std::vector<int> restart(R, 0);
            bool any = false;
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                if (S->host[r].nonfinite) {
                    // <p, A p> <= 0 or a non-finite scalar: that system stopped
                    // at its last good iterate; restart it from the true residual
                    if (++breakdowns > kMaxBreakdowns)
                        return set_error(WEO_ERR_NONFINITE, "repeated breakdown (non-finite or non-positive <p,Ap>) in FP64 CG");
                    WEO_TRY(set_flag(S, r, offsetof(SolveScalars, nonfinite), 0));
                    restart[r] = 1;
                    any = true;
                } else if (S->host[r].rr <= target[r]) {
                    any = true;  // confirm on the recomputed residual
                }
            }
            if (!any) continue;
            WEO_TRY(true_residual(h, S, *ghi));
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                rr_true[r] = S->host[r].red;
                if (!isfinite(rr_true[r])) return set_error(WEO_ERR_NONFINITE, "non-finite true residual");
                if (rr_true[r] <= target[r]) {
                    WEO_TRY(retire(r));
                } else if (restart[r] || S->host[r].rr <= target[r]) {
                    WEO_CUDA(cudaMemcpyAsync(static_cast<char *>(S->p64.ptr) + r * v64,
                                             static_cast<const char *>(S->r64.ptr) + r * v64, v64,
                                             cudaMemcpyDeviceToDevice, s));
                }
            }
            // iterated residual := recomputed one for the systems still running
            k_norm2<double2><<<grid, kRedThreads, 0, s>>>((const double2 *)S->r64.ptr, n, sc, 1);
            WEO_CUDA(cudaGetLastError());
        }
    } else {
        WEO_TRY(lo_gauge(h, &glo, s));
        WEO_TRY(staged_prepare(h, *glo, s));  // before any capture
        WEO_TRY(fstaged_prepare(h, *glo, s));
        const bool restart_all = S->restart_on_update == 1 ||
                                 (S->restart_on_update == 2 && glo->prec == WEO_BF16);
        WEO_TRY(S->xs.ensure(b32));
        WEO_TRY(S->rs.ensure(b32));
        WEO_TRY(S->p.ensure(b32));
        WEO_TRY(S->Ap.ensure(b32));
        WEO_TRY(S->t32.ensure(b32));
        WEO_CUDA(cudaMemsetAsync(S->xs.ptr, 0, b32, s));
        k_convert<float2, double2><<<flat_grid(nt), 256, 0, s>>>((float2 *)S->rs.ptr, (const double2 *)S->r64.ptr, nt);
        WEO_CUDA(cudaMemcpyAsync(S->p.ptr, S->rs.ptr, b32, cudaMemcpyDeviceToDevice, s));
        k_norm2<float2><<<grid, kRedThreads, 0, s>>>((const float2 *)S->rs.ptr, n, sc, 1);
        WEO_CUDA(cudaGetLastError());
        while (n_active > 0 && S->iterations < maxiter) {
            const int k = std::min(S->chunk, maxiter - S->iterations);
            WEO_TRY(cg_chunk(h, S, *glo, true, k));
            S->iterations += k;
            WEO_TRY(read_scalars(S));
            WEO_TRY(check_fused(h, S));
            std::vector<int> restart(R, 0);
            bool update = S->iterations >= maxiter;
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                if (S->host[r].nonfinite) {
                    // breakdown of the low-precision iteration (its operator is
                    // only approximately Hermitian positive): reliable update and
                    // restart that system's direction
                    if (++breakdowns > kMaxBreakdowns)
                        return set_error(WEO_ERR_NONFINITE, "repeated breakdown (non-finite or non-positive <p,Ap>) in the low-precision CG");
                    WEO_TRY(set_flag(S, r, offsetof(SolveScalars, nonfinite), 0));
                    restart[r] = 1;
                    update = true;
                }
                const double rr = S->host[r].rr;
                if (sqrt(rr) < S->delta * r_max[r] || rr <= target[r]) update = true;
                // an iterated residual far above the last true one: check the
                // true residual now rather than after the iteration has run away
                if (rr > kDivergence * kDivergence * rr_min[r]) update = true;
            }
            if (!update) continue;
            // reliable update of every system: fold the increments into x and
            // recompute the residuals in FP64
            k_accumulate<<<flat_grid(nt), 256, 0, s>>>((double2 *)S->x64.ptr, (float2 *)S->xs.ptr, nt);
            WEO_CUDA(cudaGetLastError());
            WEO_TRY(update_residual(h, S, *ghi, ff, active, target));
            S->reliable_updates += 1;
            bool diverging = false;
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                rr_true[r] = S->host[r].red;
                if (!isfinite(rr_true[r])) return set_error(WEO_ERR_NONFINITE, "non-finite true residual");
                if (rr_true[r] <= target[r]) WEO_TRY(retire(r));
                else r_max[r] = sqrt(rr_true[r]);
                rr_min[r] = std::min(rr_min[r], rr_true[r]);
                if (rr_true[r] > kDivergence * kDivergence * rr_min[r]) diverging = true;
            }
            if (diverging) {
                for (int r = 0; r < R; ++r)
                    if (active[r]) iters[r] = S->iterations;
                if (iters_out)
                    for (int r = 0; r < R; ++r) iters_out[r] = active[r] ? S->iterations : iters[r];
                if (relres_out)
                    for (int r = 0; r < R; ++r) relres_out[r] = bb[r] > 0.0 ? sqrt(rr_true[r] / bb[r]) : 0.0;
                return set_error(WEO_ERR_NOT_CONVERGED,
                                 "the low-precision iteration diverges from the FP64 system (true residual "
                                 "grew 1e4-fold); its operator is too far from the FP64 one");
            }
            if (n_active == 0) break;
            k_convert<float2, double2><<<flat_grid(nt), 256, 0, s>>>((float2 *)S->rs.ptr, (const double2 *)S->r64.ptr, nt);
            for (int r = 0; r < R; ++r)
                if (active[r] && (restart[r] || restart_all))
                    WEO_CUDA(cudaMemcpyAsync(static_cast<char *>(S->p.ptr) + r * v32,
                                             static_cast<const char *>(S->rs.ptr) + r * v32, v32,
                                             cudaMemcpyDeviceToDevice, s));
            k_norm2<float2><<<grid, kRedThreads, 0, s>>>((const float2 *)S->rs.ptr, n, sc, 1);
            WEO_CUDA(cudaGetLastError());
        }
    }
    int status = WEO_OK;
    if (n_active > 0) {
        // report the residuals of the returned iterates
        WEO_TRY(true_residual(h, S, *ghi));
        for (int r = 0; r < R; ++r)
            if (active[r]) {
                rr_true[r] = S->host[r].red;
                iters[r] = S->iterations;
            }
        status = set_error(WEO_ERR_NOT_CONVERGED, "maxiter reached before every true residual met tol");
    }
    for (int r = 0; r < R; ++r) {
        if (iters_out) iters_out[r] = iters[r];
        if (relres_out) relres_out[r] = bb[r] > 0.0 ? sqrt(rr_true[r] / bb[r]) : 0.0;
    }
    return status;
}

int solver_configure(wilson_eo_s *h, double delta, int chunk, int use_graphs)
{
    SolverState *S = nullptr;
    WEO_TRY(solver_state(h, &S));
    if (delta > 0.0 && delta < 1.0) S->delta = delta;
    if (chunk >= 1) S->chunk = chunk;
    if (use_graphs >= 0) S->use_graphs = use_graphs ? 1 : 0;
    for (auto &g : S->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return WEO_OK;
}

int solve_device(wilson_eo_s *h, void *x_e, const void *b_e, bool x_host, bool b_host, int nrhs,
                 double tol, int maxiter, int mixed, int *iters_out, double *relres_out,
                 cudaStream_t user)
{
    if (nrhs < 1 || nrhs > kMaxRhs) return set_error(WEO_ERR_ARG, "nrhs must be in 1..64");
    SolverState *S = nullptr;
    WEO_TRY(solver_state(h, &S));
    S->nrhs = nrhs;
    const size_t b64 = (size_t)12 * h->vh * 16 * nrhs;
    WEO_TRY(S->x64.ensure(b64));
    WEO_TRY(S->b64.ensure(b64));
    // every buffer an iteration touches exists before a graph is captured
    WEO_TRY(S->oddlo.ensure((size_t)h->vh * 96 * nrhs));
    WEO_TRY(S->odd64.ensure(b64));
    if (h->algo == 1 || h->algo == 2) WEO_TRY(fused_prepare(h, S->stream));
    // order after the caller's prior work, then run on the solver's own stream
    WEO_CUDA(cudaStreamSynchronize(user));
    cudaStream_t s = S->stream;
    WEO_CUDA(cudaMemcpyAsync(S->x64.ptr, x_e, b64,
                             x_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    WEO_CUDA(cudaMemcpyAsync(S->b64.ptr, b_e, b64,
                             b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    auto t0 = std::chrono::steady_clock::now();
    int st = solve_impl(h, tol, maxiter, mixed, iters_out, relres_out);
    if (st == WEO_OK || st == WEO_ERR_NOT_CONVERGED) {
        cudaError_t e = cudaMemcpyAsync(x_e, S->x64.ptr, b64,
                                        x_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

int solver_stats(wilson_eo_s *h, int *iterations, int *reliable_updates, int *hi_applies,
                 int *ff_applies, double *seconds)
{
    SolverState *S = h->solver;
    if (iterations) *iterations = S ? S->iterations : 0;
    if (reliable_updates) *reliable_updates = S ? S->reliable_updates : 0;
    if (hi_applies) *hi_applies = S ? S->hi_applies : 0;
    if (ff_applies) *ff_applies = S ? S->ff_applies : 0;
    if (seconds) *seconds = S ? S->seconds : 0.0;
    return WEO_OK;
}

int solver_restart_mode(wilson_eo_s *h, int restart)
{
    if (restart < 0 || restart > 2) return set_error(WEO_ERR_ARG, "restart must be 0, 1 or 2");
    SolverState *S = nullptr;
    WEO_TRY(solver_state(h, &S));
    S->restart_on_update = restart;
    return WEO_OK;
}

int solver_residual_mode(wilson_eo_s *h, int mode)
{
    if (mode != 0 && mode != 1) return set_error(WEO_ERR_ARG, "mode must be 0 (FP64) or 1 (float-float)");
    SolverState *S = nullptr;
    WEO_TRY(solver_state(h, &S));
    S->ff_residual = mode;
    return WEO_OK;
}

}  // namespace weo

// ------------------------------------------------- full system (Eqs. 3-5) --
namespace weo {

// out = x + a * H_{po} in with gauge g (precision g.prec, spinors of that precision)
static int hop_axpy(wilson_eo_s *h, const PackedGauge &g, int out_parity, void *out,
                    const void *in, const void *x, double a, cudaStream_t s)
{
    HopParams p = geom_params(h);
    p.nrhs = 1;
    p.gauge = static_cast<const char *>(g.buf.ptr);
    p.gauge_pb = g.pb;
    const long long ext = h->vh * (g.prec == WEO_F64 ? 192 : 96);
    p.in_stride = p.out_stride = p.x_stride = ext;
    p.out_parity = out_parity;
    p.in = in;
    p.out = out;
    p.x = x;
    p.a = a;
    return handle_hop(h, g.prec, g.fmt, IO_SAME, false, true, p, s);
}

// rhs_e = eta_e - D_eo eta_o = eta_e + kappa H_eo eta_o   (right side of Eq. 4)
int prepare_source_device(wilson_eo_s *h, void *rhs_e, const void *eta_e, const void *eta_o,
                          cudaStream_t s)
{
    return hop_axpy(h, h->gauge, 0, rhs_e, eta_o, eta_e, h->kappa, s);
}

// xi_o = eta_o - D_oe xi_e = eta_o + kappa H_oe xi_e   (Eq. 5, D_oo = 1)
int reconstruct_device(wilson_eo_s *h, void *xi_o, const void *eta_o, const void *xi_e,
                       cudaStream_t s)
{
    return hop_axpy(h, h->gauge, 1, xi_o, xi_e, eta_o, h->kappa, s);
}

// D_W xi = eta through Eqs. 3-5, all FP64 except the mixed solver's inner CG.
// Device or host complex128 arrays (flags say which).
int solve_full_device(wilson_eo_s *h, void *xi_e, void *xi_o, const void *eta_e,
                      const void *eta_o, const bool host[4], double tol, int maxiter, int mixed,
                      int *iters_out, double *relres_out, cudaStream_t user)
{
    SolverState *S = nullptr;
    WEO_TRY(solver_state(h, &S));
    cudaStream_t s = S->stream;
    const size_t b64 = (size_t)12 * h->vh * 16;
    WEO_CUDA(cudaStreamSynchronize(user));
    const PackedGauge *ghi = nullptr;
    WEO_TRY(hi_gauge(h, &ghi, s));
    Buffer ee, eo, rhs;
    int st = ee.ensure(b64);
    if (st == WEO_OK) st = eo.ensure(b64);
    if (st == WEO_OK) st = rhs.ensure(b64);
    auto cleanup = [&]() { ee.release(); eo.release(); rhs.release(); };
    if (st != WEO_OK) { cleanup(); return st; }
    cudaMemcpyKind k2 = host[2] ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaMemcpyKind k3 = host[3] ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(ee.ptr, eta_e, b64, k2, s) != cudaSuccess ||
        cudaMemcpyAsync(eo.ptr, eta_o, b64, k3, s) != cudaSuccess) {
        cleanup();
        return fail_cuda(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__);
    }
    // rhs = eta_e + kappa H_eo eta_o ; b = M^dag rhs (into ee, which is free now)
    st = hop_axpy(h, *ghi, 0, rhs.ptr, eo.ptr, ee.ptr, h->kappa, s);
    if (st == WEO_OK) st = S->odd64.ensure(b64);
    if (st == WEO_OK) st = meo_with(h, *ghi, S->odd64, ee.ptr, rhs.ptr, 1, true, s);
    if (st != WEO_OK) { cleanup(); return st; }
    // even solve on device copies (x starts from the caller's xi_e guess)
    if (cudaMemcpyAsync(rhs.ptr, xi_e, b64, host[0] ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cleanup();
        return fail_cuda(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__);
    }
    st = solve_device(h, rhs.ptr, ee.ptr, false, false, 1, tol, maxiter, mixed, iters_out, relres_out, s);
    if (st != WEO_OK && st != WEO_ERR_NOT_CONVERGED) { cleanup(); return st; }
    const int solve_status = st;
    // xi_o = eta_o + kappa H_oe xi_e  (into ee)
    st = hop_axpy(h, *ghi, 1, ee.ptr, rhs.ptr, eo.ptr, h->kappa, s);
    if (st == WEO_OK && cudaMemcpyAsync(xi_e, rhs.ptr, b64, host[0] ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = fail_cuda(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__);
    if (st == WEO_OK && cudaMemcpyAsync(xi_o, ee.ptr, b64, host[1] ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = fail_cuda(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__);
    if (st == WEO_OK && cudaStreamSynchronize(s) != cudaSuccess)
        st = fail_cuda(cudaGetLastError(), "cudaStreamSynchronize", __FILE__, __LINE__);
    cleanup();
    return st == WEO_OK ? solve_status : st;
}

}  // namespace weo
