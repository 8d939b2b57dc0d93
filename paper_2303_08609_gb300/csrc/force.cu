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
#include "weo_internal.h"

namespace weo {

struct GradParams {
    int lxh, ly, lz, lt, vh;
    int parity;            // parity of the link base sites x handled by this launch
    const void *g, *phi;   // even
    const void *t, *w;     // odd
    const char *gauge;     // packed links (for the force)
    long long gauge_pb;
    void *out;             // canonical [mu][lex][3][3] complex (T)
    double scale;          // -kappa^2
    int force;             // 0: gradient, 1: TA(G U^dag)
};

template <int MU, int S, typename T>
__device__ __forceinline__ void proj_all(const cx<T> v[12], cx<T> h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) project<MU, S>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
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

template <class Sp, class Lk, int MU>
__device__ __forceinline__ void grad_dir(const GradParams &p, long long i, long long nb,
                                         const cx<typename Sp::real> own0[12],
                                         const cx<typename Sp::real> own1[12], long long lex)
{
    using T = typename Sp::real;
    cx<T> n0[12], n1[12], ha[2][3], hb[2][3];
    cx<T> G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[a][b] = {T(0), T(0)};
    if (p.parity == 0) {
        // own0 = g(x), own1 = phi(x); neighbours t(x+mu), w(x+mu)
        Sp::load(p.t, p.vh, nb, n0);
        Sp::load(p.w, p.vh, nb, n1);
        proj_all<MU, 1>(own0, ha);   // (1 - gamma) g(x)
        proj_all<MU, 1>(n0, hb);     // same projector on t(x+mu)
        outer_acc(G, ha, hb);
        proj_all<MU, -1>(own1, ha);  // (1 + gamma) on phi(x)
        proj_all<MU, -1>(n1, hb);    // (1 + gamma) w(x+mu)
        outer_acc(G, ha, hb);
    } else {
        // own0 = t(x), own1 = w(x); neighbours g(x+mu), phi(x+mu)
        Sp::load(p.g, p.vh, nb, n0);
        Sp::load(p.phi, p.vh, nb, n1);
        proj_all<MU, -1>(own0, ha);  // (1 + gamma) on t(x)
        proj_all<MU, -1>(n0, hb);    // (1 + gamma) g(x+mu)
        outer_acc(G, ha, hb);
        proj_all<MU, 1>(own1, ha);   // (1 - gamma) w(x)
        proj_all<MU, 1>(n1, hb);     // (1 - gamma) on phi(x+mu)
        outer_acc(G, ha, hb);
    }
    const T sc = T(p.scale);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[a][b] = cscale(G[a][b], sc);
    const long long V = 2LL * p.vh;
    T *out = static_cast<T *>(p.out) + 18 * (MU * V + lex);
    if (p.force) {
        cx<T> U[3][3];
        Lk::load(p.gauge + (2 * MU + p.parity) * p.gauge_pb, p.vh, i, U);
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
                T re = (W[a][b].r - W[b][a].r) * T(0.5);
                T im = (W[a][b].i + W[b][a].i) * T(0.5) - (a == b ? trim : T(0));
                out[2 * (3 * a + b)] = re;
                out[2 * (3 * a + b) + 1] = im;
            }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                out[2 * (3 * a + b)] = G[a][b].r;
                out[2 * (3 * a + b) + 1] = G[a][b].i;
            }
    }
}

// One thread per site of parity p.parity; it writes the four links based there.
template <class Sp, class Lk>
__global__ void __launch_bounds__(128) link_grad_kernel(const GradParams p)
{
    using T = typename Sp::real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.vh) return;
    int rem = i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.parity) & 1;
    const int x = 2 * xh + par;
    const long long lx = 2LL * p.lxh;
    const long long lex = ((long long)(t * p.lz + z) * p.ly + y) * lx + x;
    const int sy = p.lxh, sz = p.lxh * p.ly, st = p.lxh * p.ly * p.lz;
    const int xp = par ? (xh + 1 == p.lxh ? 0 : xh + 1) : xh;
    const long long n_x = i - xh + xp;
    const long long n_y = i + (y + 1 == p.ly ? -(p.ly - 1) * sy : sy);
    const long long n_z = i + (z + 1 == p.lz ? -(p.lz - 1) * sz : sz);
    const long long n_t = i + (t + 1 == p.lt ? -(long long)(p.lt - 1) * st : st);
    cx<T> own0[12], own1[12];
    if (p.parity == 0) {
        Sp::load(p.g, p.vh, i, own0);
        Sp::load(p.phi, p.vh, i, own1);
    } else {
        Sp::load(p.t, p.vh, i, own0);
        Sp::load(p.w, p.vh, i, own1);
    }
    grad_dir<Sp, Lk, 0>(p, i, n_x, own0, own1, lex);
    grad_dir<Sp, Lk, 1>(p, i, n_y, own0, own1, lex);
    grad_dir<Sp, Lk, 2>(p, i, n_z, own0, own1, lex);
    grad_dir<Sp, Lk, 3>(p, i, n_t, own0, own1, lex);
}

template <class Sp, class Lk>
static int launch_grad(const GradParams &p0, cudaStream_t s)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((p0.vh + threads - 1) / threads);
    for (int par = 0; par < 2; ++par) {
        GradParams p = p0;
        p.parity = par;
        link_grad_kernel<Sp, Lk><<<blocks, threads, 0, s>>>(p);
        WEO_CUDA(cudaGetLastError());
    }
    return WEO_OK;
}

// Gradient (force = 0) or force (force = 1) with g and phi on the device.
// Uses h->tmp2 and h->tmp3 for t and w (odd).
int link_grad_device(wilson_eo_s *h, void *out, const void *g, const void *phi, int force,
                     cudaStream_t s)
{
    const long long ext = h->vh * (h->prec == WEO_F64 ? 192 : 96);
    WEO_TRY(h->tmp2.ensure((size_t)ext));
    WEO_TRY(h->tmp3.ensure((size_t)ext));
    HopParams hp = geom_params(h);
    hp.nrhs = 1;
    hp.gauge = static_cast<const char *>(h->gauge.buf.ptr);
    hp.gauge_pb = h->gauge.pb;
    hp.in_stride = hp.out_stride = ext;
    // t = H_oe phi
    hp.out_parity = 1;
    hp.in = phi;
    hp.out = h->tmp2.ptr;
    WEO_TRY(handle_hop(h, h->prec, h->fmt, IO_SAME, false, false, hp, s));
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
    p.parity = 0;
    p.g = g;
    p.phi = phi;
    p.t = h->tmp2.ptr;
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
