// Hopping kernel of the even-odd Wilson matrix, one output site per thread.
//
// Computes, for every site x of parity `out_parity` (Eq. 1 without -kappa):
//   (H psi)(x) = sum_mu [ (1 - s gamma_mu) U_mu(x) psi(x+mu) + (1 + s gamma_mu) U_mu^dag(x-mu) psi(x-mu) ]
// with s = +1, or s = -1 for the adjoint (H^dag swaps the projectors, which is
// the gamma_5-hermiticity of Eq. 1). Mode Axpy writes out = x + a * (H psi),
// which with a = -kappa^2 completes M_eo = 1 - kappa^2 H_eo H_oe (Eq. 4).
//
// Per direction the 4-spinor is projected onto a 2-spinor (the structure of
// (1 -+ gamma_mu) in the chiral basis), multiplied by the link, and the two
// lower spin components are rebuilt from the upper ones (Sec. 2, Fig. 2).
// Chiral basis: gamma_mu = [[0, A_mu], [A_mu^dag, 0]] with A_x = -i sigma_1,
// A_y = -i sigma_2, A_z = -i sigma_3, A_t = 1. For the projector (1 - S gamma):
//   h = psi_up - S A psi_dn ;  chi = W h ;  out_up += chi ; out_dn += -S A^dag chi.
//
// Neighbour indexing on the x-compacted parity arrays (Sec. 3.3-3.4): with
// x = 2 xh + p and p = (y+z+t+out_parity) & 1, the x+1 neighbour has compact
// index xh + p and the x-1 neighbour xh - (1-p), both periodic in Lx/2; the
// other directions are plain strides Lx/2, Lx Ly/2, Lx Ly Lz/2 with wrap.
// This index arithmetic replaces the SIMD select/permute shuffles the paper
// needs for its x and y shifts (Figs. 5-6).
#pragma once

#include <type_traits>

#include "weo_fields.cuh"

namespace weo {

struct HopParams {
    int lxh, ly, lz, lt;   // Lx/2 and the other extents
    int vh;                // V/2
    int out_parity;
    int nrhs;
    const void *in;        // input spinor (opposite parity), rhs stride in bytes
    long long in_stride;
    void *out;             // output spinor (out_parity)
    long long out_stride;
    const void *x;         // axpy addend (out_parity), may be null in hop mode
    long long x_stride;
    const char *gauge;     // packed links: field (mu, parity) at gauge + (2 mu + parity) * gauge_pb
    long long gauge_pb;
    double a;              // axpy coefficient
    int reverse;           // walk the sites from the top (blocks in reverse order)
    int blocked;           // CTAs take 2x2x2 blocks of rows in (y, z, t) (blockDim = 8 Lx/2)
};

// h = psi_up - S A_mu psi_dn for one colour
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cx<R> p0, const cx<R> p1, const cx<R> p2,
                                        const cx<R> p3, cx<R> &h0, cx<R> &h1)
{
    if (MU == 0) {  // A = -i sigma_1: A psi_dn = (-i p3, -i p2)
        h0 = S > 0 ? cadd(p0, cmuli(p3)) : csub(p0, cmuli(p3));
        h1 = S > 0 ? cadd(p1, cmuli(p2)) : csub(p1, cmuli(p2));
    } else if (MU == 1) {  // A = -i sigma_2 = [[0,-1],[1,0]]: A psi_dn = (-p3, p2)
        h0 = S > 0 ? cadd(p0, p3) : csub(p0, p3);
        h1 = S > 0 ? csub(p1, p2) : cadd(p1, p2);
    } else if (MU == 2) {  // A = -i sigma_3: A psi_dn = (-i p2, i p3)
        h0 = S > 0 ? cadd(p0, cmuli(p2)) : csub(p0, cmuli(p2));
        h1 = S > 0 ? csub(p1, cmuli(p3)) : cadd(p1, cmuli(p3));
    } else {  // A = 1
        h0 = S > 0 ? csub(p0, p2) : cadd(p0, p2);
        h1 = S > 0 ? csub(p1, p3) : cadd(p1, p3);
    }
}

// out_up += chi ; out_dn += -S A^dag chi, for one colour
template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct(cx<R> &o0, cx<R> &o1, cx<R> &o2, cx<R> &o3,
                                            const cx<R> c0, const cx<R> c1)
{
    o0 = cadd(o0, c0);
    o1 = cadd(o1, c1);
    if (MU == 0) {  // A^dag chi = (i c1, i c0)
        o2 = S > 0 ? csub(o2, cmuli(c1)) : cadd(o2, cmuli(c1));
        o3 = S > 0 ? csub(o3, cmuli(c0)) : cadd(o3, cmuli(c0));
    } else if (MU == 1) {  // A^dag chi = (c1, -c0)
        o2 = S > 0 ? csub(o2, c1) : cadd(o2, c1);
        o3 = S > 0 ? cadd(o3, c0) : csub(o3, c0);
    } else if (MU == 2) {  // A^dag chi = (i c0, -i c1)
        o2 = S > 0 ? csub(o2, cmuli(c0)) : cadd(o2, cmuli(c0));
        o3 = S > 0 ? cadd(o3, cmuli(c1)) : csub(o3, cmuli(c1));
    } else {  // A^dag chi = (c0, c1)
        o2 = S > 0 ? csub(o2, c0) : cadd(o2, c0);
        o3 = S > 0 ? csub(o3, c1) : cadd(o3, c1);
    }
}

// One hopping direction for R right-hand sides. FWD: link U_mu(x), projector
// (1 - S0 gamma); backward: link U_mu(x-mu)^dag, projector (1 + S0 gamma).
template <class SIn, class Lk, int MU, bool FWD, int S0, int R, typename T>
__device__ __forceinline__ void hop_dir(cx<T> (&acc)[R][12], const HopParams &p, long long nb,
                                        long long link_idx, int link_par, int rhs0)
{
    constexpr int S = FWD ? S0 : -S0;
    cx<T> U[3][3];
    Lk::load(p.gauge + (2 * MU + link_par) * p.gauge_pb, p.vh, link_idx, U);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (R > 1 && rhs0 + r >= p.nrhs) break;
        cx<T> v[12];
        SIn::load(static_cast<const char *>(p.in) + (rhs0 + r) * p.in_stride, p.vh, nb, v);
        // spin-colour index k = 3*spin + colour
        cx<T> h[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) project<MU, S>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
        cx<T> w[2][3];
        if constexpr (std::is_same<T, ff>::value) {
            // float-float: the six real products of each row are exact and
            // independent; they are summed pairwise (short dependency chains)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    ff re[6], im[6];
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const cx<ff> u = FWD ? U[a][b] : U[b][a];
                        const cx<ff> v = h[s][b];
                        const ff ui = FWD ? u.i : -u.i;  // conj(u) for the backward hop
                        re[2 * b] = ff_prod(u.r, v.r);
                        re[2 * b + 1] = ff_prod(-ui, v.i);
                        im[2 * b] = ff_prod(u.r, v.i);
                        im[2 * b + 1] = ff_prod(ui, v.r);
                    }
                    w[s][a] = {((re[0] + re[1]) + (re[2] + re[3])) + (re[4] + re[5]),
                               ((im[0] + im[1]) + (im[2] + im[3])) + (im[4] + im[5])};
                }
        } else {
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cx<T> z = {T(0), T(0)};
#pragma unroll
                    for (int b = 0; b < 3; ++b) z = FWD ? cfma(U[a][b], h[s][b], z) : cfmaconj(U[b][a], h[s][b], z);
                    w[s][a] = z;
                }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            reconstruct<MU, S>(acc[r][c], acc[r][3 + c], acc[r][6 + c], acc[r][9 + c], w[0][c], w[1][c]);
    }
}

// All hops of output site i (parity p.out_parity) for right-hand sides
// rhs0 .. rhs0+R-1, then the optional axpy and the store.
template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int R>
__device__ __forceinline__ void hop_site(const HopParams &p, const int i, const int rhs0)
{
    using T = typename SOut::real;  // FP64 only when the output is FP64
    constexpr int S0 = Dag ? -1 : 1;

    int rem = i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.out_parity) & 1;
    const int in_par = p.out_parity ^ 1;

    const int sy = p.lxh, sz = p.lxh * p.ly, st = p.lxh * p.ly * p.lz;
    const int row = i - xh;
    const int xp = par ? (xh + 1 == p.lxh ? 0 : xh + 1) : xh;
    const int xm = par ? xh : (xh == 0 ? p.lxh - 1 : xh - 1);
    const long long n_xp = row + xp, n_xm = row + xm;
    const long long n_yp = i + (y + 1 == p.ly ? -(p.ly - 1) * sy : sy);
    const long long n_ym = i + (y == 0 ? (p.ly - 1) * sy : -sy);
    const long long n_zp = i + (z + 1 == p.lz ? -(p.lz - 1) * sz : sz);
    const long long n_zm = i + (z == 0 ? (p.lz - 1) * sz : -sz);
    const long long n_tp = i + (t + 1 == p.lt ? -(long long)(p.lt - 1) * st : st);
    const long long n_tm = i + (t == 0 ? (long long)(p.lt - 1) * st : -st);

    cx<T> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = {T(0), T(0)};

    const int op = p.out_parity;
    hop_dir<SIn, Lk, 0, true, S0, R>(acc, p, n_xp, i, op, rhs0);
    hop_dir<SIn, Lk, 0, false, S0, R>(acc, p, n_xm, n_xm, in_par, rhs0);
    hop_dir<SIn, Lk, 1, true, S0, R>(acc, p, n_yp, i, op, rhs0);
    hop_dir<SIn, Lk, 1, false, S0, R>(acc, p, n_ym, n_ym, in_par, rhs0);
    hop_dir<SIn, Lk, 2, true, S0, R>(acc, p, n_zp, i, op, rhs0);
    hop_dir<SIn, Lk, 2, false, S0, R>(acc, p, n_zm, n_zm, in_par, rhs0);
    hop_dir<SIn, Lk, 3, true, S0, R>(acc, p, n_tp, i, op, rhs0);
    hop_dir<SIn, Lk, 3, false, S0, R>(acc, p, n_tm, n_tm, in_par, rhs0);

#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (R > 1 && rhs0 + r >= p.nrhs) break;
        if (Axpy) {
            cx<T> xv[12];
            SX::load(static_cast<const char *>(p.x) + (rhs0 + r) * p.x_stride, p.vh, i, xv);
            const T a = T(p.a);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[r][k].r = fma(a, acc[r][k].r, xv[k].r);
                acc[r][k].i = fma(a, acc[r][k].i, xv[k].i);
            }
        }
        SOut::store(static_cast<char *>(p.out) + (rhs0 + r) * p.out_stride, p.vh, i, acc[r]);
    }
}

// Block order of the hop kernels: a 1-D grid of (site block, right-hand-side
// block) pairs with the right-hand-side block varying fastest, so the CTAs of
// one site block -- which read the same links -- run side by side and every
// link comes from HBM once per hop, the other right-hand-side blocks finding it
// in L2. With p.reverse the site blocks are taken from the top down, so a hop
// that follows another one first reads the part of its input that was written
// last (and is still in L2). nrb = right-hand-side blocks.
__device__ __forceinline__ void block_coords(const HopParams &p, int nrb, int &site_block, int &rhs_block)
{
    const int nsb = (int)gridDim.x / nrb;
    rhs_block = (int)blockIdx.x % nrb;
    const int sb = (int)blockIdx.x / nrb;
    site_block = p.reverse ? nsb - 1 - sb : sb;
}

// Output site of thread t in site block b. Default: consecutive compact
// indices (a CTA covers whole rows of one (z, t) plane). Blocked: a CTA of
// 8 Lx/2 threads covers the rows (y0 + dy, z0 + dz, t0 + dt), dy, dz, dt in
// {0, 1}, so half of its y, z and t neighbour rows are its own input rows
// and reach it through L1 instead of L2 (all extents are even, so the blocks
// tile the lattice exactly).
__device__ __forceinline__ int site_of(const HopParams &p, int b, int t)
{
    if (!p.blocked) return b * (int)blockDim.x + t;
    const int hy = p.ly >> 1, hz = p.lz >> 1;
    const int y0 = 2 * (b % hy), z0 = 2 * ((b / hy) % hz), t0 = 2 * (b / (hy * hz));
    const int row = t / p.lxh, xh = t - row * p.lxh;
    return (((t0 + (row >> 2)) * p.lz + z0 + ((row >> 1) & 1)) * p.ly + y0 + (row & 1)) * p.lxh + xh;
}

// One output site per thread.
template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int R>
__global__ void __launch_bounds__(256) hop_kernel(const HopParams p)
{
    int b, rb;
    block_coords(p, (p.nrhs + R - 1) / R, b, rb);
    const int i = site_of(p, b, threadIdx.x);
    if (i >= p.vh) return;
    hop_site<SIn, SOut, SX, Lk, Dag, Axpy, R>(p, i, rb * R);
}

// The same kernel with the register allocation capped at 64 (four CTAs of 256
// threads per SM, 50 % occupancy): for FP32-arithmetic hops with one
// right-hand side per thread and 18-real FP32 or 16-bit links this measured
// faster on GB300 than the uncapped 78-80 registers, despite a few spilled
// values.
template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int R>
__global__ void __launch_bounds__(256, 4) hop_kernel_occ(const HopParams p)
{
    int b, rb;
    block_coords(p, (p.nrhs + R - 1) / R, b, rb);
    const int i = site_of(p, b, threadIdx.x);
    if (i >= p.vh) return;
    hop_site<SIn, SOut, SX, Lk, Dag, Axpy, R>(p, i, rb * R);
}

// Right-hand sides on neighbouring lanes: NL consecutive threads take one site
// and NL different right-hand sides. Their link loads read the same addresses,
// so each warp fetches a link once for NL right-hand sides, while every thread
// keeps the register footprint of a single right-hand side.
template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int NL>
__global__ void __launch_bounds__(256, 4) hop_kernel_lanes(const HopParams p)
{
    int b, rb;
    block_coords(p, (p.nrhs + NL - 1) / NL, b, rb);
    const int i = b * (int)(blockDim.x / NL) + (int)threadIdx.x / NL;
    const int r = rb * NL + (int)threadIdx.x % NL;
    if (i >= p.vh || r >= p.nrhs) return;
    hop_site<SIn, SOut, SX, Lk, Dag, Axpy, 1>(p, i, r);
}

// ------------------------------------------------ links shared per tile --
// Several right-hand sides with each tile's links loaded once: a CTA of 256
// threads owns a tile of T = 256 / NRL consecutive output sites. It first
// copies the eight links of every tile site -- U_mu(x) and U_mu(x - mu) for the
// backward hop -- into shared memory (converted to FP32 complex, [8][9][T],
// 576 T bytes), then its NRL groups of T threads take the right-hand sides
// rhs0 = 0 .. NRL-1 and step by NRL, one (site, right-hand side) per thread --
// or RP right-hand sides per thread sharing each link read from shared memory
// -- with the spinors read from global memory as in hop_kernel. A link leaves
// global memory once per tile instead of once per right-hand-side block.

// compact indices of the 8 neighbours of site i (order: +x, -x, +y, -y, +z,
// -z, +t, -t), as in hop_site
__device__ __forceinline__ void site_neighbours(const HopParams &p, int i, int nb[8])
{
    int rem = i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.out_parity) & 1;
    const int sy = p.lxh, sz = p.lxh * p.ly, st = p.lxh * p.ly * p.lz;
    const int row = i - xh;
    nb[0] = row + (par ? (xh + 1 == p.lxh ? 0 : xh + 1) : xh);
    nb[1] = row + (par ? xh : (xh == 0 ? p.lxh - 1 : xh - 1));
    nb[2] = i + (y + 1 == p.ly ? -(p.ly - 1) * sy : sy);
    nb[3] = i + (y == 0 ? (p.ly - 1) * sy : -sy);
    nb[4] = i + (z + 1 == p.lz ? -(p.lz - 1) * sz : sz);
    nb[5] = i + (z == 0 ? (p.lz - 1) * sz : -sz);
    nb[6] = i + (t + 1 == p.lt ? -(p.lt - 1) * st : st);
    nb[7] = i + (t == 0 ? (p.lt - 1) * st : -st);
}

// one hopping direction with the link from shared memory (9 complex at
// stride T from lk)
// (RP right-hand sides rhs, rhs + step, ... share the link's registers)
template <class SIn, int MU, bool FWD, int S0, int RP>
__device__ __forceinline__ void hop_dir_shared(cx<float> (&acc)[RP][12], const HopParams &p, int nb,
                                               const float2 *lk, int T, int rhs, int step)
{
    constexpr int S = FWD ? S0 : -S0;
    cx<float> U[3][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 u = lk[k * T];
        U[k / 3][k % 3] = {u.x, u.y};
    }
#pragma unroll
    for (int r = 0; r < RP; ++r) {
        if (RP > 1 && rhs + r * step >= p.nrhs) break;
        cx<float> v[12];
        SIn::load(static_cast<const char *>(p.in) + (rhs + r * step) * p.in_stride, p.vh, nb, v);
        cx<float> h[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) project<MU, S>(v[c], v[3 + c], v[6 + c], v[9 + c], h[0][c], h[1][c]);
        cx<float> w[2][3];
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<float> z = {0.f, 0.f};
#pragma unroll
                for (int b = 0; b < 3; ++b) z = FWD ? cfma(U[a][b], h[sp][b], z) : cfmaconj(U[b][a], h[sp][b], z);
                w[sp][a] = z;
            }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            reconstruct<MU, S>(acc[r][c], acc[r][3 + c], acc[r][6 + c], acc[r][9 + c], w[0][c], w[1][c]);
    }
}

template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int NRL, int RP = 1>
__global__ void __launch_bounds__(256, RP == 1 ? 3 : 2) hop_kernel_tile_links(const HopParams p)
{
    constexpr int T = 256 / NRL;
    extern __shared__ __align__(16) float2 lk_sm[];  // [8 directions][9 complex][T]
    const int ntiles = (int)gridDim.x;
    const int tile = p.reverse ? ntiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
    const int i0 = tile * T;
    const int in_par = p.out_parity ^ 1;
    // the tile's links: direction d = 2 mu + b, U_mu(x) (b = 0) or U_mu(x - mu) (b = 1)
    for (int e = threadIdx.x; e < 8 * T; e += 256) {
        const int d = e / T, s = e - d * T;
        const int i = i0 + s;
        if (i >= p.vh) continue;
        const int mu = d >> 1;
        int idx = i;
        if (d & 1) {
            int nb[8];
            site_neighbours(p, i, nb);
            idx = nb[d];
        }
        cx<float> U[3][3];
        Lk::load(p.gauge + (2 * mu + ((d & 1) ? in_par : p.out_parity)) * p.gauge_pb, p.vh, idx, U);
#pragma unroll
        for (int k = 0; k < 9; ++k) lk_sm[(d * 9 + k) * T + s] = make_float2(U[k / 3][k % 3].r, U[k / 3][k % 3].i);
    }
    __syncthreads();
    const int s = (int)threadIdx.x % T, rl = (int)threadIdx.x / T;
    const int i = i0 + s;
    if (i >= p.vh) return;
    constexpr int S0 = Dag ? -1 : 1;
    const float2 *lk = lk_sm + s;
    // each thread takes right-hand sides r, r + NRL, ..., RP of them per pass
    for (int r = rl; r < p.nrhs; r += NRL * RP) {
        int nb[8];
        site_neighbours(p, i, nb);
        cx<float> acc[RP][12];
#pragma unroll
        for (int q = 0; q < RP; ++q)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[q][k] = {0.f, 0.f};
        hop_dir_shared<SIn, 0, true, S0, RP>(acc, p, nb[0], lk + 0 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 0, false, S0, RP>(acc, p, nb[1], lk + 1 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 1, true, S0, RP>(acc, p, nb[2], lk + 2 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 1, false, S0, RP>(acc, p, nb[3], lk + 3 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 2, true, S0, RP>(acc, p, nb[4], lk + 4 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 2, false, S0, RP>(acc, p, nb[5], lk + 5 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 3, true, S0, RP>(acc, p, nb[6], lk + 6 * 9 * T, T, r, NRL);
        hop_dir_shared<SIn, 3, false, S0, RP>(acc, p, nb[7], lk + 7 * 9 * T, T, r, NRL);
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            const int rq = r + q * NRL;
            if (RP > 1 && rq >= p.nrhs) break;
            if (Axpy) {
                cx<float> xv[12];
                SX::load(static_cast<const char *>(p.x) + rq * p.x_stride, p.vh, i, xv);
                const float a = float(p.a);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    acc[q][k].r = fmaf(a, acc[q][k].r, xv[k].r);
                    acc[q][k].i = fmaf(a, acc[q][k].i, xv[k].i);
                }
            }
            SOut::store(static_cast<char *>(p.out) + rq * p.out_stride, p.vh, i, acc[q]);
        }
    }
}

}  // namespace weo
