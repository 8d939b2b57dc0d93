// Link gradient and pseudofermion force of the even-odd Wilson matrix.
//
// For L = Re<g, M_eo phi> (g, phi even), with t = H_oe phi and w = H_eo^dag g
// (both odd), differentiating the two terms of Eq. 1 at each link gives the
// Euclidean gradient G_mu(x) = dL/dRe U + i dL/dIm U:
//   x even: G = -kappa^2 ( sum_spin [(1-gamma)g(x)] (x) conj(t(x+mu))
//                        + sum_spin phi(x) (x) conj([(1+gamma)w(x+mu)]) )
//   x odd : G = -kappa^2 ( sum_spin t(x) (x) conj([(1+gamma)g(x+mu)])
//                        + sum_spin [(1-gamma)w(x)] (x) conj(phi(x+mu)) )
// Since (1 -+ gamma)/2 is an orthogonal projector, each spin sum equals
// sum_{r=0,1} h_r(p) (x) conj(h_r(q)) with both vectors projected onto the same
// 2-spinor (the projection of the hopping kernel), halving the work.
// The force of S = |M_eo phi|^2 (g = 2 M_eo phi) is F = TA(G U^dag),
// TA(W) = (W - W^dag)/2 - tr(W - W^dag)/6: the traceless anti-Hermitian matrix
// with dS/d eps = Re tr(X^dag F) under U -> exp(eps X) U.
#include <type_traits>

#include "weo_internal.h"

namespace weo {

struct GradParams {
    int lxh, ly, lz, lt, vh;
    const void *g, *phi;   // even
    const void *t, *w;     // odd
    const char *gauge;     // packed links (for the force)
    long long gauge_pb;
    void *out;             // canonical [mu][lex][3][3] complex (T)
    double scale;          // -kappa^2
    int force;             // 0: gradient, 1: TA(G U^dag)
};

constexpr int kGradThreads = 128;

// The projection of the hopping kernel written as h = psi_up + S q, with q
// fixed by mu (chiral basis): the sign S may then differ between threads.
template <int MU, typename T>
__device__ __forceinline__ void proj_rt(const cx<T> v[12], T S, cx<T> h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> p2 = v[6 + c], p3 = v[9 + c];
        cx<T> q0, q1;
        if (MU == 0) {
            q0 = cmuli(p3);
            q1 = cmuli(p2);
        } else if (MU == 1) {
            q0 = p3;
            q1 = cneg(p2);
        } else if (MU == 2) {
            q0 = cmuli(p2);
            q1 = cneg(cmuli(p3));
        } else {
            q0 = cneg(p2);
            q1 = cneg(p3);
        }
        h[0][c] = {fma(S, q0.r, v[c].r), fma(S, q0.i, v[c].i)};
        h[1][c] = {fma(S, q1.r, v[3 + c].r), fma(S, q1.i, v[3 + c].i)};
    }
}

// G[a][b] += sum_r hp[r][a] conj(hq[r][b])
template <typename T>
__device__ __forceinline__ void outer_acc(cx<T> G[3][3], const cx<T> hp[2][3], const cx<T> hq[2][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            G[a][b] = cfmaconj(hq[0][b], hp[0][a], G[a][b]);
            G[a][b] = cfmaconj(hq[1][b], hp[1][a], G[a][b]);
        }
}

// The 3x3 result for link (mu, x) of a thread's site: the gradient G, or the
// force TA(G U^dag), as 18 reals in m.
template <class Sp, class Lk, int MU>
__device__ __forceinline__ void grad_link(const GradParams &p, int par, long long i, long long nb,
                                          const cx<typename Sp::real> own0[12],
                                          const cx<typename Sp::real> own1[12],
                                          typename Sp::real m[18])
{
    using T = typename Sp::real;
    // even x: G = (1-g)g(x) (x) (1-g)t(x+mu) + (1+g)phi(x) (x) (1+g)w(x+mu);
    // odd x:  G = (1+g)t(x) (x) (1+g)g(x+mu) + (1-g)w(x) (x) (1-g)phi(x+mu)
    const T S1 = par ? T(-1) : T(1);
    cx<T> n0[12], n1[12], ha[2][3], hb[2][3];
    Sp::load(par ? p.g : p.t, p.vh, nb, n0);
    Sp::load(par ? p.phi : p.w, p.vh, nb, n1);
    cx<T> G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[a][b] = {T(0), T(0)};
    proj_rt<MU>(own0, S1, ha);
    proj_rt<MU>(n0, S1, hb);
    outer_acc(G, ha, hb);
    proj_rt<MU>(own1, -S1, ha);
    proj_rt<MU>(n1, -S1, hb);
    outer_acc(G, ha, hb);
    const T sc = T(p.scale);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[a][b] = cscale(G[a][b], sc);
    if (p.force) {
        cx<T> U[3][3];
        Lk::load(p.gauge + (2 * MU + par) * p.gauge_pb, p.vh, i, U);
        cx<T> W[3][3];  // G U^dag
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                cx<T> z = {T(0), T(0)};
#pragma unroll
                for (int k = 0; k < 3; ++k) z = cfmaconj(U[b][k], G[a][k], z);
                W[a][b] = z;
            }
        // TA(W): anti-Hermitian part minus its trace / 3
        const T trim = (W[0][0].i + W[1][1].i + W[2][2].i) / T(3);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                m[2 * (3 * a + b)] = (W[a][b].r - W[b][a].r) * T(0.5);
                m[2 * (3 * a + b) + 1] = (W[a][b].i + W[b][a].i) * T(0.5) - (a == b ? trim : T(0));
            }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                m[2 * (3 * a + b)] = G[a][b].r;
                m[2 * (3 * a + b) + 1] = G[a][b].i;
            }
    }
}

// Stage the block's matrices for one direction in shared memory and write them
// out as one contiguous, coalesced range of the canonical [mu][lex] array.
template <typename T>
__device__ __forceinline__ void write_links(const GradParams &p, int mu, long long lex0, int nvalid,
                                            const T m[18], T *sh)
{
#pragma unroll
    for (int k = 0; k < 18; ++k) sh[threadIdx.x * 18 + k] = m[k];
    __syncthreads();
    const long long V = 2LL * p.vh;
    T *dst = static_cast<T *>(p.out) + 18 * (mu * V + lex0);
    if (nvalid == kGradThreads && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        // 16-byte vectors: 18 * kGradThreads reals per block (the block's range
        // starts 16-byte aligned whenever the output array does)
        using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int kPer = 16 / sizeof(T);
        const V4 *src4 = reinterpret_cast<const V4 *>(sh);
        V4 *dst4 = reinterpret_cast<V4 *>(dst);
        for (int k = threadIdx.x; k < 18 * kGradThreads / kPer; k += kGradThreads) dst4[k] = src4[k];
    } else {
        for (int k = threadIdx.x; k < 18 * nvalid; k += kGradThreads) dst[k] = sh[k];
    }
    __syncthreads();
}

// One thread per lattice site (lexicographic, both parities): it computes the
// four links based there; each block writes its links per direction as one
// contiguous range.
template <class Sp, class Lk>
__global__ void __launch_bounds__(kGradThreads) link_grad_kernel(const GradParams p)
{
    using T = typename Sp::real;
    __shared__ __align__(16) T sh[18 * kGradThreads];
    const long long lx = 2LL * p.lxh, V = 2LL * p.vh;
    const long long lex0 = (long long)blockIdx.x * kGradThreads;
    const long long lex = lex0 + threadIdx.x;
    const int nvalid = (int)(V - lex0 < kGradThreads ? V - lex0 : kGradThreads);
    const bool valid = lex < V;
    long long r = valid ? lex : 0;
    const int x = (int)(r % lx);
    r /= lx;
    const int y = (int)(r % p.ly);
    r /= p.ly;
    const int z = (int)(r % p.lz);
    const int t = (int)(r / p.lz);
    const int par = (x + y + z + t) & 1;
    const long long i = (valid ? lex : 0) >> 1;
    // compact indices of x + mu (the other parity)
    const long long base = ((long long)(t * p.lz + z) * p.ly + y) * lx;
    const long long n_x = (base + (x + 1 == lx ? 0 : x + 1)) >> 1;
    const long long n_y = (((long long)(t * p.lz + z) * p.ly + (y + 1 == p.ly ? 0 : y + 1)) * lx + x) >> 1;
    const long long n_z = (((long long)(t * p.lz + (z + 1 == p.lz ? 0 : z + 1)) * p.ly + y) * lx + x) >> 1;
    const long long n_t = (((long long)((t + 1 == p.lt ? 0 : t + 1) * p.lz + z) * p.ly + y) * lx + x) >> 1;
    cx<T> own0[12], own1[12];
    // own fields: g, phi on even sites; t, w on odd sites
    Sp::load(par ? p.t : p.g, p.vh, i, own0);
    Sp::load(par ? p.w : p.phi, p.vh, i, own1);
    T m[18];
    grad_link<Sp, Lk, 0>(p, par, i, n_x, own0, own1, m);
    write_links(p, 0, lex0, nvalid, m, sh);
    grad_link<Sp, Lk, 1>(p, par, i, n_y, own0, own1, m);
    write_links(p, 1, lex0, nvalid, m, sh);
    grad_link<Sp, Lk, 2>(p, par, i, n_z, own0, own1, m);
    write_links(p, 2, lex0, nvalid, m, sh);
    grad_link<Sp, Lk, 3>(p, par, i, n_t, own0, own1, m);
    write_links(p, 3, lex0, nvalid, m, sh);
}

template <class Sp, class Lk>
static int launch_grad(const GradParams &p, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((2LL * p.vh + kGradThreads - 1) / kGradThreads);
    link_grad_kernel<Sp, Lk><<<blocks, kGradThreads, 0, s>>>(p);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

// Gradient (force = 0) or force (force = 1) with g and phi on the device.
// Uses h->tmp2 and h->tmp3 for t and w (odd).
int link_grad_device(wilson_eo_s *h, void *out, const void *g, const void *phi, int force,
                     cudaStream_t s, const void *t_known)
{
    const long long ext = h->vh * (h->prec == WEO_F64 ? 192 : 96);
    WEO_TRY(h->tmp2.ensure((size_t)ext));
    WEO_TRY(h->tmp3.ensure((size_t)ext));
    HopParams hp = geom_params(h);
    hp.nrhs = 1;
    hp.gauge = static_cast<const char *>(h->gauge.buf.ptr);
    hp.gauge_pb = h->gauge.pb;
    hp.in_stride = hp.out_stride = ext;
    // t = H_oe phi (unless the caller has it: the intermediate of M_eo phi)
    hp.out_parity = 1;
    if (!t_known) {
        hp.in = phi;
        hp.out = h->tmp2.ptr;
        WEO_TRY(handle_hop(h, h->prec, h->fmt, IO_SAME, false, false, hp, s));
    }
    // w = H_eo^dag g: the adjoint hop onto odd sites
    hp.in = g;
    hp.out = h->tmp3.ptr;
    WEO_TRY(handle_hop(h, h->prec, h->fmt, IO_SAME, true, false, hp, s));
    GradParams p;
    p.lxh = h->dims[0] / 2;
    p.ly = h->dims[1];
    p.lz = h->dims[2];
    p.lt = h->dims[3];
    p.vh = (int)h->vh;
    p.g = g;
    p.phi = phi;
    p.t = t_known ? t_known : h->tmp2.ptr;
    p.w = h->tmp3.ptr;
    p.gauge = static_cast<const char *>(h->gauge.buf.ptr);
    p.gauge_pb = h->gauge.pb;
    p.out = out;
    p.scale = -h->kappa * h->kappa;
    p.force = force;
    int tok = prof_begin(h, force ? "force" : "link_grad", s);
    int st;
    if (h->prec == WEO_F64)
        st = h->fmt == WEO_LINK12 ? launch_grad<SpF64, LkF64_12>(p, s) : launch_grad<SpF64, LkF64_18>(p, s);
    else
        st = h->fmt == WEO_LINK12 ? launch_grad<SpF32, LkF32_12>(p, s) : launch_grad<SpF32, LkF32_18>(p, s);
    prof_end(h, tok, s);
    return st;
}

// Scale an external spinor in place: v *= c (used for g = 2 chi).
template <typename T2, typename T>
__global__ void scale_kernel(T2 *v, long long n, T c)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) {
        T2 a = v[k];
        a.x *= c;
        a.y *= c;
        v[k] = a;
    }
}

int scale_spinor(wilson_eo_s *h, void *v, int nrhs, double c, cudaStream_t s)
{
    const long long n = 12LL * h->vh * nrhs;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (h->prec == WEO_F64)
        scale_kernel<double2, double><<<blocks, 256, 0, s>>>(static_cast<double2 *>(v), n, c);
    else
        scale_kernel<float2, float><<<blocks, 256, 0, s>>>(static_cast<float2 *>(v), n, (float)c);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

}  // namespace weo
