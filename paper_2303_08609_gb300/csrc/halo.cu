// Domain-decomposed hopping term with forced exchange (Secs. 3.5-3.6).
//
// The lattice is split along t into P sub-domains ("ranks") of Lt/P slices.
// Every t-hop that crosses a sub-domain boundary -- including the periodic
// wrap, so P = 1 exchanges with itself, as the paper's benchmark forces
// communication in all directions -- travels through face buffers:
//   EO1 (pack): for the slice just above each boundary, the 2-spinor projected
//        with the forward projector (no link: the receiver owns U_t(x)); for
//        the slice just below, the 2-spinor projected with the backward
//        projector and multiplied by U_t^dag already (the sender owns that
//        link), as the paper pre-multiplies upward exports;
//   exchange: one device copy per face and rank (the stand-in for MPI/NCCL
//        messages; on one GPU the "send" and "receive" buffers are distinct);
//   bulk: every output site, all hops that stay inside the sub-domain;
//   EO2 (finish): boundary sites add the received halo contributions.
// Sites across a t boundary share the slice-local compact index s, so a face
// is simply the Vs = Lx Ly Lz / 2 sites of one slice of one parity.
#include <string.h>

#include "weo_internal.h"

namespace weo {

struct HaloParams {
    HopParams p;     // geometry, fields, gauge (hop mode)
    int ranks;       // P
    int lt_local;    // Lt / P
    int vs;          // sites of one parity per t-slice
    void *send_fwd, *send_bwd, *recv_fwd, *recv_bwd;  // [P][12 reals ... ] 2-spinors
};

// 2-spinor face element: [rank][k = 0..5][s] complex (planar in s)
template <typename T2>
__device__ __forceinline__ T2 *face_ptr(void *base, int vs, int rank, int k, int s)
{
    return static_cast<T2 *>(base) + ((long long)rank * 6 + k) * vs + s;
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// EO1: faces of every rank. Thread = (rank, s).
template <class Sp, class Lk, bool Dag>
__global__ void halo_pack_kernel(const HaloParams hp)
{
    using T = typename Sp::real;
    using T2 = typename Vec2<T>::type;
    constexpr int S0 = Dag ? -1 : 1;
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= (long long)hp.ranks * hp.vs) return;
    const int r = (int)(g / hp.vs), s = (int)(g % hp.vs);
    const HopParams &p = hp.p;
    const int in_par = p.out_parity ^ 1;
    cx<T> v[12], h[2][3];
    // bottom slice of rank r: needed (forward hop) by the top slice of rank r-1
    {
        const int t = r * hp.lt_local;
        const long long j = (long long)t * hp.vs + s;
        Sp::load(p.in, p.vh, j, v);
#pragma unroll
        for (int c = 0; c < 3; ++c) project<3, S0>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            T2 o;
            o.x = h[k / 3][k % 3].r;
            o.y = h[k / 3][k % 3].i;
            *face_ptr<T2>(hp.send_fwd, hp.vs, r, k, s) = o;
        }
    }
    // top slice of rank r: needed (backward hop) by the bottom slice of rank r+1,
    // projected with the backward projector and multiplied by U_t(y)^dag here
    {
        const int t = (r + 1) * hp.lt_local - 1;
        const long long j = (long long)t * hp.vs + s;
        Sp::load(p.in, p.vh, j, v);
#pragma unroll
        for (int c = 0; c < 3; ++c) project<3, -S0>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
        cx<T> U[3][3];
        Lk::load(p.gauge + (2 * 3 + in_par) * p.gauge_pb, p.vh, j, U);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<T> z = {T(0), T(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) z = cfmaconj(U[b][a], h[sp][b], z);
                T2 o;
                o.x = z.r;
                o.y = z.i;
                *face_ptr<T2>(hp.send_bwd, hp.vs, r, 3 * sp + a, s) = o;
            }
    }
}

// bulk: all output sites; t-hops that leave the sub-domain are skipped.
template <class Sp, class Lk, bool Dag>
__global__ void __launch_bounds__(128) halo_bulk_kernel(const HaloParams hp)
{
    using T = typename Sp::real;
    constexpr int S0 = Dag ? -1 : 1;
    const HopParams &p = hp.p;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.vh) return;
    int rem = i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.out_parity) & 1;
    const int in_par = p.out_parity ^ 1;
    const int sy = p.lxh, sz = p.lxh * p.ly, st = hp.vs;
    const int row = i - xh;
    const int xp = par ? (xh + 1 == p.lxh ? 0 : xh + 1) : xh;
    const int xm = par ? xh : (xh == 0 ? p.lxh - 1 : xh - 1);
    const long long n_xp = row + xp, n_xm = row + xm;
    const long long n_yp = i + (y + 1 == p.ly ? -(p.ly - 1) * sy : sy);
    const long long n_ym = i + (y == 0 ? (p.ly - 1) * sy : -sy);
    const long long n_zp = i + (z + 1 == p.lz ? -(p.lz - 1) * sz : sz);
    const long long n_zm = i + (z == 0 ? (p.lz - 1) * sz : -sz);
    const int tl = t % hp.lt_local;
    cx<T> acc[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0][k] = {T(0), T(0)};
    const int op = p.out_parity;
    hop_dir<Sp, Lk, 0, true, S0, 1>(acc, p, n_xp, i, op, 0);
    hop_dir<Sp, Lk, 0, false, S0, 1>(acc, p, n_xm, n_xm, in_par, 0);
    hop_dir<Sp, Lk, 1, true, S0, 1>(acc, p, n_yp, i, op, 0);
    hop_dir<Sp, Lk, 1, false, S0, 1>(acc, p, n_ym, n_ym, in_par, 0);
    hop_dir<Sp, Lk, 2, true, S0, 1>(acc, p, n_zp, i, op, 0);
    hop_dir<Sp, Lk, 2, false, S0, 1>(acc, p, n_zm, n_zm, in_par, 0);
    if (tl + 1 < hp.lt_local) hop_dir<Sp, Lk, 3, true, S0, 1>(acc, p, i + st, i, op, 0);
    if (tl > 0) hop_dir<Sp, Lk, 3, false, S0, 1>(acc, p, i - st, i - st, in_par, 0);
    Sp::store(p.out, p.vh, i, acc[0]);
}

// Add one received face to acc at output site i (face 0: forward t-hop from
// the halo with the local link U_t(x); face 1: backward t-hop, halo already
// multiplied by U^dag).
template <class Sp, class Lk, bool Dag>
__device__ __forceinline__ void add_face(const HaloParams &hp, int face, int r, int s, long long i,
                                         cx<typename Sp::real> acc[12])
{
    using T = typename Sp::real;
    using T2 = typename Vec2<T>::type;
    constexpr int S0 = Dag ? -1 : 1;
    const HopParams &p = hp.p;
    cx<T> h[2][3], w[2][3];
    if (face == 0) {
        const T2 *src = face_ptr<T2>(hp.recv_fwd, hp.vs, r, 0, s);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T2 d = src[(long long)k * hp.vs];
            h[k / 3][k % 3] = {d.x, d.y};
        }
        cx<T> U[3][3];
        Lk::load(p.gauge + (2 * 3 + p.out_parity) * p.gauge_pb, p.vh, i, U);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<T> z = {T(0), T(0)};
#pragma unroll
                for (int b = 0; b < 3; ++b) z = cfma(U[a][b], h[sp][b], z);
                w[sp][a] = z;
            }
#pragma unroll
        for (int c = 0; c < 3; ++c) reconstruct<3, S0>(acc[c], acc[3 + c], acc[6 + c], acc[9 + c], w[0][c], w[1][c]);
    } else {
        const T2 *src = face_ptr<T2>(hp.recv_bwd, hp.vs, r, 0, s);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T2 d = src[(long long)k * hp.vs];
            w[k / 3][k % 3] = {d.x, d.y};
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) reconstruct<3, -S0>(acc[c], acc[3 + c], acc[6 + c], acc[9 + c], w[0][c], w[1][c]);
    }
}

// EO2: boundary slices add the received halo contributions. Thread = (rank, s).
// Each output site is read and written once (with one slice per rank the
// top and bottom slices coincide and both faces are added in registers).
template <class Sp, class Lk, bool Dag>
__global__ void halo_finish_kernel(const HaloParams hp)
{
    using T = typename Sp::real;
    const HopParams &p = hp.p;
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= (long long)hp.ranks * hp.vs) return;
    const int r = (int)(g / hp.vs), s = (int)(g % hp.vs);
    const int t_top = (r + 1) * hp.lt_local - 1, t_bot = r * hp.lt_local;
    cx<T> acc[12];
    const long long it = (long long)t_top * hp.vs + s;
    Sp::load(p.out, p.vh, it, acc);
    add_face<Sp, Lk, Dag>(hp, 0, r, s, it, acc);
    if (t_bot == t_top) {
        add_face<Sp, Lk, Dag>(hp, 1, r, s, it, acc);
        Sp::store(p.out, p.vh, it, acc);
        return;
    }
    Sp::store(p.out, p.vh, it, acc);
    const long long ib = (long long)t_bot * hp.vs + s;
    Sp::load(p.out, p.vh, ib, acc);
    add_face<Sp, Lk, Dag>(hp, 1, r, s, ib, acc);
    Sp::store(p.out, p.vh, ib, acc);
}

template <class Sp, class Lk, bool Dag>
static int run_split(wilson_eo_s *h, const HaloParams &hp, size_t face_bytes, cudaStream_t s)
{
    const long long nface = (long long)hp.ranks * hp.vs;
    const unsigned fb = (unsigned)((nface + 127) / 128);
    halo_pack_kernel<Sp, Lk, Dag><<<fb, 128, 0, s>>>(hp);
    WEO_CUDA(cudaGetLastError());
    // exchange: rank r receives the forward face of rank r+1 and the backward
    // face of rank r-1 (periodic; with one rank, from itself)
    const size_t per_rank = face_bytes / hp.ranks;
    for (int r = 0; r < hp.ranks; ++r) {
        const int up = (r + 1) % hp.ranks, dn = (r - 1 + hp.ranks) % hp.ranks;
        WEO_CUDA(cudaMemcpyAsync(static_cast<char *>(hp.recv_fwd) + r * per_rank,
                                 static_cast<const char *>(hp.send_fwd) + up * per_rank, per_rank,
                                 cudaMemcpyDeviceToDevice, s));
        WEO_CUDA(cudaMemcpyAsync(static_cast<char *>(hp.recv_bwd) + r * per_rank,
                                 static_cast<const char *>(hp.send_bwd) + dn * per_rank, per_rank,
                                 cudaMemcpyDeviceToDevice, s));
    }
    halo_bulk_kernel<Sp, Lk, Dag><<<(unsigned)((hp.p.vh + 127) / 128), 128, 0, s>>>(hp);
    WEO_CUDA(cudaGetLastError());
    halo_finish_kernel<Sp, Lk, Dag><<<fb, 128, 0, s>>>(hp);
    WEO_CUDA(cudaGetLastError());
    (void)h;
    return WEO_OK;
}

template <class Sp, class Lk>
static int run_split_d(wilson_eo_s *h, const HaloParams &hp, size_t fb, bool dag, cudaStream_t s)
{
    return dag ? run_split<Sp, Lk, true>(h, hp, fb, s) : run_split<Sp, Lk, false>(h, hp, fb, s);
}

int hop_split_device(wilson_eo_s *h, int ranks, int out_parity, bool dag, void *out,
                     const void *in, cudaStream_t s)
{
    if (h->prec != WEO_F64 && h->prec != WEO_F32)
        return set_error(WEO_ERR_UNSUPPORTED, "the split hop needs an FP64 or FP32 handle");
    const int lt = h->dims[3];
    if (ranks < 1 || lt % ranks) return set_error(WEO_ERR_ARG, "ranks must divide Lt");
    HaloParams hp;
    memset(&hp, 0, sizeof(hp));
    hp.p = geom_params(h);
    hp.p.nrhs = 1;
    hp.p.gauge = static_cast<const char *>(h->gauge.buf.ptr);
    hp.p.gauge_pb = h->gauge.pb;
    hp.p.out_parity = out_parity;
    hp.p.in = in;
    hp.p.out = out;
    const long long ext = h->vh * (h->prec == WEO_F64 ? 192 : 96);
    hp.p.in_stride = hp.p.out_stride = ext;
    hp.ranks = ranks;
    hp.lt_local = lt / ranks;
    hp.vs = (h->dims[0] / 2) * h->dims[1] * h->dims[2];
    const size_t face_bytes = (size_t)ranks * 6 * hp.vs * (h->prec == WEO_F64 ? 16 : 8);
    WEO_TRY(h->halo.ensure(4 * face_bytes));
    char *b = static_cast<char *>(h->halo.ptr);
    hp.send_fwd = b;
    hp.send_bwd = b + face_bytes;
    hp.recv_fwd = b + 2 * face_bytes;
    hp.recv_bwd = b + 3 * face_bytes;
    const bool c = h->fmt == WEO_LINK12;
    int tok = prof_begin(h, "hop_split", s);
    int st;
    if (h->prec == WEO_F64)
        st = c ? run_split_d<SpF64, LkF64_12>(h, hp, face_bytes, dag, s) : run_split_d<SpF64, LkF64_18>(h, hp, face_bytes, dag, s);
    else
        st = c ? run_split_d<SpF32, LkF32_12>(h, hp, face_bytes, dag, s) : run_split_d<SpF32, LkF32_18>(h, hp, face_bytes, dag, s);
    prof_end(h, tok, s);
    return st;
}

}  // namespace weo
