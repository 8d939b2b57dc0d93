// Hopping kernel with its operands staged in shared memory by TMA: the same
// sum as hop_kernel (Eq. 1 for one parity, Sec. 3.3's H_oe / H_eo pass), one
// right-hand side, templated on the formats it reads and writes:
//   In   FP32 planar spinors (loaded as tensor boxes), or 16-bit spinors with a
//        per-site norm in row blocks (loaded as plain bulk copies);
//   Out  FP32 planar spinors, or 16-bit row blocks;
//   Lk   the link format of the per-tile link blocks (FP32 or 16-bit, 18 or 12
//        reals per link).
//
// The output sites are cut into tiles of R lattice rows: T = R * Lx/2
// consecutive compact indices inside one (z, t) plane. Everything the hopping
// sum of a tile reads is then a few contiguous blocks:
//   input spinor (parity 1-p): the tile rows of the same plane (+-x, and +-y
//     inside the tile), the rows y0-1 and y0+R (periodic in y), and the tile
//     rows of the planes z+1, z-1, t+1, t-1 (periodic): seven regions;
//   links: the eight links of every output site -- U_mu(x) and U_mu(x-mu) --
//     repacked once per gauge field into one block per tile (direction-major,
//     each direction in the link format's planar layout with plane stride T),
//     so a tile's links are a single cp.async.bulk copy. This doubles the
//     links' footprint (each link is stored for both sites it joins), not
//     their traffic: a hop still reads each stored link once;
//   the FP32 axpy addend at the tile: one box.
// One producer thread issues them into a ring of two to five stages, each with
// an mbarrier that counts the bytes landed. Each stage is owned by one group
// of consumer teams, which compute from shared memory only, so the bytes in
// flight no longer depend on the registers each thread holds. A team is two
// warps on 32 sites of the tile: one takes the x and y directions, the other
// the z and t directions, whose partial sums it hands over in shared memory; a
// tile of more than 32 sites has two teams. Owning its stage, each group waits
// on each barrier for the phase after the one it saw last, which the parity
// form of mbarrier.try_wait requires.
//
// Every wait is bounded (a time limit on the global timer): on expiry the
// kernel records an error word that wilson_eo_check reports, stops, and the
// producer waits, again bounded, for its own copies still in flight.
#pragma once

#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "weo_internal.h"

namespace weo {
namespace staged {

constexpr int kMaxTeams = 8;  // consumer teams of two warps
constexpr int kMaxTile = 64;  // sites per tile (tensor box limit of 256 floats)
constexpr int kMaxStages = 5;
constexpr int kSmemLimit = 227 * 1024;

// plain loads: operands already in shared memory
struct LdPlain {
    template <typename T>
    __device__ static __forceinline__ T ld(const T *p) { return *p; }
};

// ------------------------------------------------------- spinor formats --
// A region holds `rows` lattice rows of Lx/2 = hx sites; (r, xh) is a site.

// FP32 planar: [12][n] complex (n = rows * hx), loaded as a tensor box.
struct InF32 {
    static constexpr int kSite = 96;
    static constexpr bool kBoxes = true;
    __device__ static __forceinline__ void load(const char *reg, int n, int hx, int r, int xh,
                                                cx<float> v[12])
    {
        const float2 *p = reinterpret_cast<const float2 *>(reg) + r * hx + xh;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float2 q = p[k * n];
            v[k] = {q.x, q.y};
        }
    }
};

// 16-bit with a per-site FP32 norm, in row blocks: row = [3][hx] uint4 (four
// complex each) then [hx] float norms (52 hx bytes); a region is `rows`
// consecutive row blocks, copied as one contiguous range.
template <class Tr>
struct In16 {
    static constexpr int kSite = 52;
    static constexpr bool kBoxes = false;
    __device__ static __forceinline__ void load(const char *reg, int n, int hx, int r, int xh,
                                                cx<float> v[12])
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(reg + (size_t)r * 52 * hx);
        const float nrm = reinterpret_cast<const float *>(p + 3 * hx)[xh];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const uint4 w = p[q * hx + xh];
            const float2 a = Tr::to_f2(w.x), b = Tr::to_f2(w.y), c = Tr::to_f2(w.z),
                         d = Tr::to_f2(w.w);
            v[4 * q + 0] = {a.x * nrm, a.y * nrm};
            v[4 * q + 1] = {b.x * nrm, b.y * nrm};
            v[4 * q + 2] = {c.x * nrm, c.y * nrm};
            v[4 * q + 3] = {d.x * nrm, d.y * nrm};
        }
    }
};

// output at compact index i
struct OutF32 {
    __device__ static __forceinline__ void store(void *out, long long vh, int hx, long long i,
                                                 const cx<float> v[12])
    {
        float2 *o = static_cast<float2 *>(out) + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k * vh] = make_float2(v[k].r, v[k].i);
    }
};

template <class Tr>
struct Out16 {
    __device__ static __forceinline__ void store(void *out, long long vh, int hx, long long i,
                                                 const cx<float> v[12])
    {
        const long long row = i / hx;
        Sp16<Tr>::store(static_cast<char *>(out) + row * 52 * hx, hx, (long long)(i - row * hx), v);
    }
};

// ------------------------------------------------------ stage layout --
struct StageLayout {
    int sp[7];  // spinor regions: tile rows, row y0-1, row y0+R, planes z+1, z-1, t+1, t-1
    int lk;     // the tile's link block
    int x;      // FP32 axpy addend
    int part;   // z/t partial sums (the z+1 region for FP32 input)
    int bytes;  // one stage
    int tx;     // bytes the loads of one tile deliver
};

inline int round128(int b) { return (b + 127) & ~127; }

inline size_t stage_smem(const StageLayout &L, int stages)
{
    return (size_t)stages * L.bytes + (2 * stages + kMaxTeams) * sizeof(uint64_t);
}

// layout of one stage; site_bytes: input spinor bytes per site; link_bytes:
// one link in the block format
inline void make_layout(int hx, int rows, int site_bytes, int link_bytes, bool axpy, StageLayout &L)
{
    const int T = hx * rows;
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off += round128(bytes);
        return o;
    };
    L.sp[0] = take(site_bytes * T);
    L.sp[1] = take(site_bytes * hx);
    L.sp[2] = take(site_bytes * hx);
    for (int k = 3; k < 7; ++k) L.sp[k] = take(site_bytes * T);
    L.lk = take(8 * link_bytes * T);
    L.x = axpy ? take(96 * T) : 0;
    L.part = site_bytes >= 96 ? L.sp[3] : take(96 * T);
    L.bytes = off;
    L.tx = site_bytes * (5 * T + 2 * hx) + 8 * link_bytes * T + (axpy ? 96 * T : 0);
}

// teams per tile of T sites
inline int teams_per_tile(int T) { return T > 32 ? 2 : 1; }

// ring depth: the requested one if it fits in shared memory and in the team
// limit, else the most that fit up to `cap` (0 if none)
inline int pick_depth(const StageLayout &L, int T, int want, int cap)
{
    const int tpt = teams_per_tile(T);
    auto ok = [&](int d) {
        return d >= 2 && d <= kMaxStages && d * tpt <= kMaxTeams && stage_smem(L, d) <= kSmemLimit;
    };
    if (want) return ok(want) ? want : 0;
    for (int d = cap; d >= 2; --d)
        if (ok(d)) return d;
    return 0;
}

struct Params {
    CUtensorMap sp_tile, sp_row, x_tile;
    const char *in;     // input spinor (row blocks when In is 16-bit)
    const char *links;  // link blocks of this output parity
    void *out;
    StageLayout L;
    int lxh, ly, lz, lt, rows, tile, ntiles, out_parity, reverse, tpt, link_block;
    long long vh;
    float a;
    unsigned int *err;
    unsigned long long limit_ns;
    int inject;  // failure-path test: the producer never loads the CTA's first tile
};

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of `bar` with the given parity to complete, at most
// limit_ns nanoseconds; false (and the error word set) on expiry
static __device__ __noinline__ bool mbar_wait(uint64_t *bar, unsigned parity, const Params &P)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > P.limit_ns) {
            atomicOr(P.err, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                          uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *m)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// ---------------------------------------------------------------- tiles --
struct TileGeo {
    int y0, z, t;
    long long i0;  // first compact index of the tile
};

__device__ __forceinline__ TileGeo tile_geo(const Params &P, int j)
{
    if (P.reverse) j = P.ntiles - 1 - j;
    TileGeo g;
    const int row0 = j * P.rows;
    const int plane = row0 / P.ly;
    g.y0 = row0 - plane * P.ly;
    g.z = plane % P.lz;
    g.t = plane / P.lz;
    g.i0 = (long long)row0 * P.lxh;
    return g;
}

// global row index of row y of plane (z, t)
__device__ __forceinline__ int row_index(const Params &P, int z, int t, int y)
{
    return (t * P.lz + z) * P.ly + y;
}

// issue the loads of tile j into the stage at `base`
template <class In, bool Axpy>
__device__ __forceinline__ void issue_tile(const Params &P, int j, char *base, uint64_t *full,
                                           uint64_t pol)
{
    const TileGeo g = tile_geo(P, j);
    const StageLayout &L = P.L;
    const int ly = P.ly, lz = P.lz, lt = P.lt, hx = P.lxh;
    const int ym = g.y0 == 0 ? ly - 1 : g.y0 - 1;
    const int yp = g.y0 + P.rows == ly ? 0 : g.y0 + P.rows;
    const int zp = g.z + 1 == lz ? 0 : g.z + 1, zm = g.z == 0 ? lz - 1 : g.z - 1;
    const int tp = g.t + 1 == lt ? 0 : g.t + 1, tm = g.t == 0 ? lt - 1 : g.t - 1;
    // first rows of the seven spinor regions
    const int rws[7] = {row_index(P, g.z, g.t, g.y0), row_index(P, g.z, g.t, ym),
                        row_index(P, g.z, g.t, yp),   row_index(P, zp, g.t, g.y0),
                        row_index(P, zm, g.t, g.y0),  row_index(P, g.z, tp, g.y0),
                        row_index(P, g.z, tm, g.y0)};
    const long long jt = g.i0 / P.tile;  // tile index in memory order
    mbar_expect_tx(full, (unsigned)L.tx);
    // the links are read once per launch: evict first
    bulk_hint(base + L.lk, P.links + jt * P.link_block, (unsigned)P.link_block, full, pol);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int nrow = (k == 1 || k == 2) ? 1 : P.rows;
        if (In::kBoxes)  // coordinate in floats, 2 per complex
            tma_2d(base + L.sp[k], nrow == 1 ? &P.sp_row : &P.sp_tile, 2 * rws[k] * hx, 0, full);
        else
            bulk(base + L.sp[k], P.in + (long long)rws[k] * In::kSite * hx,
                 (unsigned)(In::kSite * hx * nrow), full);
    }
    if (Axpy) tma_2d(base + L.x, &P.x_tile, 2 * (int)g.i0, 0, full);
}

// one hopping direction from shared memory: the spinor at (r, xh) of a region
// of n sites, the link of site s of the direction block `lk` (plane stride T)
template <class In, class Lk, int MU, bool FWD, int S0>
__device__ __forceinline__ void staged_dir(cx<float> (&acc)[12], const char *reg, int n, int hx,
                                           int r, int xh, const char *lk, int T, int s)
{
    constexpr int S = FWD ? S0 : -S0;
    cx<float> U[3][3];
    Lk::template load<float>(lk, T, s, U);
    cx<float> v[12];
    In::load(reg, n, hx, r, xh, v);
    cx<float> h[2][3];
#pragma unroll
    for (int col = 0; col < 3; ++col)
        project<MU, S>(v[col], v[3 + col], v[6 + col], v[9 + col], h[0][col], h[1][col]);
    cx<float> w[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<float> zz = {0.f, 0.f};
#pragma unroll
            for (int col = 0; col < 3; ++col)
                zz = FWD ? cfma(U[a][col], h[sp][col], zz) : cfmaconj(U[col][a], h[sp][col], zz);
            w[sp][a] = zz;
        }
#pragma unroll
    for (int col = 0; col < 3; ++col)
        reconstruct<MU, S>(acc[col], acc[3 + col], acc[6 + col], acc[9 + col], w[0][col], w[1][col]);
}

// at most two teams per stage, and the producer warp
template <class In, class Out, class Lk, bool Dag, bool Axpy, int NS>
__global__ void __launch_bounds__(32 * (4 * NS + 1), 1) hop_staged_kernel(const __grid_constant__ Params P)
{
    extern __shared__ __align__(128) char smem[];
    const StageLayout &L = P.L;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NS * L.bytes);
    uint64_t *empty = full + NS;
    uint64_t *ready = empty + NS;  // per team: z/t partial sums written
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int ntile_cta =
        P.ntiles > (int)blockIdx.x ? (P.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, (unsigned)P.tpt);  // the x/y warps of the tile's teams
        }
        for (int t = 0; t < NS * P.tpt; ++t) mbar_init(ready + t, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 2 * NS * P.tpt) {  // producer
        if (lane != 0) return;
        if (In::kBoxes) {
            prefetch_map(&P.sp_tile);
            prefetch_map(&P.sp_row);
        }
        if (Axpy) prefetch_map(&P.x_tile);
        const uint64_t pol = policy_evict_first();
        int issued = 0;
        for (int k = 0; k < ntile_cta; ++k) {
            const int s = k % NS, n = k / NS;
            if (n >= 1 && !mbar_wait(empty + s, (unsigned)((n - 1) & 1), P)) break;
            if (P.inject && k == 0) continue;  // nothing loaded, nothing in flight
            issue_tile<In, Axpy>(P, (int)blockIdx.x + k * (int)gridDim.x, smem + s * L.bytes,
                                 full + s, pol);
            issued = k + 1;
        }
        // the last loads of each stage must have landed before the CTA exits
        for (int k = issued - 1; k >= 0 && k >= issued - NS; --k) {
            if (P.inject && k == 0) continue;
            mbar_wait(full + k % NS, (unsigned)((k / NS) & 1), P);
        }
        return;
    }

    // consumers: team = two warps (x/y and z/t) on 32 sites of a tile; group g
    // = tpt teams owning stage g and the CTA's tiles k = g, g + NS, ...
    const int team = warp >> 1, q = warp & 1;
    const int g = team / P.tpt;
    const int s = (team - g * P.tpt) * 32 + lane;  // site within the tile
    const bool active = s < P.tile;
    const int hx = P.lxh, T = P.tile;
    const int r = s / hx, xh = s - r * hx;
    constexpr int S0 = Dag ? -1 : 1;
    char *base = smem + g * L.bytes;
    const char *lk = base + L.lk;
    constexpr int LB = Lk::kBytesPerSite;  // one direction's block: LB * T bytes
    float2 *part = reinterpret_cast<float2 *>(base + L.part);  // [12][T] z/t partial sums
    for (int k = g; k < ntile_cta; k += NS) {
        const unsigned m = (unsigned)(k / NS);  // use of this stage
        if (!mbar_wait(full + g, m & 1u, P)) return;
        const TileGeo tg = tile_geo(P, (int)blockIdx.x + k * (int)gridDim.x);
        cx<float> acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {0.f, 0.f};
        if (q == 0) {
            if (active) {
                const int par = (tg.y0 + r + tg.z + tg.t + P.out_parity) & 1;
                const int xp = par ? (xh + 1 == hx ? 0 : xh + 1) : xh;
                const int xm = par ? xh : (xh == 0 ? hx - 1 : xh - 1);
                const char *c0 = base + L.sp[0];
                staged_dir<In, Lk, 0, true, S0>(acc, c0, T, hx, r, xp, lk, T, s);
                staged_dir<In, Lk, 0, false, S0>(acc, c0, T, hx, r, xm, lk + LB * T, T, s);
                if (r + 1 < P.rows)
                    staged_dir<In, Lk, 1, true, S0>(acc, c0, T, hx, r + 1, xh, lk + 2 * LB * T, T, s);
                else
                    staged_dir<In, Lk, 1, true, S0>(acc, base + L.sp[2], hx, hx, 0, xh,
                                                    lk + 2 * LB * T, T, s);
                if (r > 0)
                    staged_dir<In, Lk, 1, false, S0>(acc, c0, T, hx, r - 1, xh, lk + 3 * LB * T, T, s);
                else
                    staged_dir<In, Lk, 1, false, S0>(acc, base + L.sp[1], hx, hx, 0, xh,
                                                     lk + 3 * LB * T, T, s);
            }
            if (!mbar_wait(ready + team, m & 1u, P)) return;
            if (active) {
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const float2 v = part[c * T + s];
                    acc[c].r += v.x;
                    acc[c].i += v.y;
                }
                if (Axpy) {
                    const float2 *xv = reinterpret_cast<const float2 *>(base + L.x);
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        const float2 v = xv[c * T + s];
                        acc[c] = {fmaf(P.a, acc[c].r, v.x), fmaf(P.a, acc[c].i, v.y)};
                    }
                }
                Out::store(P.out, P.vh, hx, tg.i0 + s, acc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + g);
        } else {
            if (active) {
                staged_dir<In, Lk, 2, true, S0>(acc, base + L.sp[3], T, hx, r, xh, lk + 4 * LB * T, T, s);
                staged_dir<In, Lk, 2, false, S0>(acc, base + L.sp[4], T, hx, r, xh, lk + 5 * LB * T, T, s);
                staged_dir<In, Lk, 3, true, S0>(acc, base + L.sp[5], T, hx, r, xh, lk + 6 * LB * T, T, s);
                staged_dir<In, Lk, 3, false, S0>(acc, base + L.sp[6], T, hx, r, xh, lk + 7 * LB * T, T, s);
                // each lane writes only its own site's slots (for FP32 input,
                // the z+1 slots it has read itself)
#pragma unroll
                for (int c = 0; c < 12; ++c) part[c * T + s] = make_float2(acc[c].r, acc[c].i);
            }
            // a later TMA load into this stage may write over the partial sums
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(ready + team);
        }
    }
}

// ----------------------------------------------------------- link blocks --
// Link block of output parity p for tiles of T sites: output site i (tile i / T,
// s = i % T), direction d = 2 mu + b holds U_mu(x) (b = 0) or U_mu(x - mu)
// (b = 1) in the block format's planar layout at block(i / T) + d * LB * T,
// plane stride T. Src: the packed field's format; Blk: the block format.
template <class Src, class Blk>
__global__ void pack_link_blocks_kernel(const HopParams p, int T, char *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.vh) return;
    int rem = (int)i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.out_parity) & 1;
    const long long sy = p.lxh, sz = (long long)p.lxh * p.ly, st = sz * p.lz;
    const long long row = i - xh;
    const long long nb[4] = {row + (par ? xh : (xh == 0 ? p.lxh - 1 : xh - 1)),
                             i + (y == 0 ? (p.ly - 1) * sy : -sy),
                             i + (z == 0 ? (p.lz - 1) * sz : -sz),
                             i + (t == 0 ? (p.lt - 1) * st : -st)};
    constexpr int LB = Blk::kBytesPerSite;
    char *blk = out + (i / T) * 8 * LB * T;
    const long long s = i % T;
    for (int mu = 0; mu < 4; ++mu)
        for (int b = 0; b < 2; ++b) {
            cx<double> U[3][3];
            const char *f = p.gauge + (2 * mu + (b ? p.out_parity ^ 1 : p.out_parity)) * p.gauge_pb;
            Src::template load<double>(f, p.vh, b ? nb[mu] : i, U);
            Blk::store(blk + (2 * mu + b) * LB * T, T, s, U);
        }
}

template <class Src, class Blk>
int pack_link_blocks(const HopParams &p0, int T, char *out, cudaStream_t s)
{
    HopParams p = p0;
    const long long per_parity = 8ll * Blk::kBytesPerSite * p.vh;
    for (int par = 0; par < 2; ++par) {
        p.out_parity = par;
        pack_link_blocks_kernel<Src, Blk><<<(unsigned)((p.vh + 255) / 256), 256, 0, s>>>(
            p, T, out + par * per_parity);
        WEO_CUDA(cudaGetLastError());
    }
    return WEO_OK;
}

// ------------------------------------------------------------ launching --
// Tensor maps: FP32 planar spinor, 12 planes of 2 vh floats.
bool encode_spinor_map(CUtensorMap *m, const void *ptr, long long vh, int box_sites);

// A staged hop. blocks: link blocks of both output parities; depth 0 picks
// the most stages (up to 3) that fit.
template <class In, class Out, class Lk, bool Dag, bool Axpy, int NS>
int launch_one(const Params &P, int grid, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(hop_staged_kernel<In, Out, Lk, Dag, Axpy, NS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    });
    WEO_CUDA(attr);
    const int threads = 32 * (2 * NS * P.tpt + 1);  // NS x tpt teams and the producer
    hop_staged_kernel<In, Out, Lk, Dag, Axpy, NS><<<grid, threads, stage_smem(P.L, NS), s>>>(P);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <class In, class Out, class Lk, bool Axpy, int... Depths>
int launch_depths(bool dag, int depth, const Params &P, int grid, cudaStream_t s)
{
    int st = WEO_ERR_UNSUPPORTED;
    bool done = false;
    auto one = [&](auto d) {
        constexpr int D = decltype(d)::value;
        if (done || depth != D) return;
        done = true;
        st = dag ? launch_one<In, Out, Lk, true, Axpy, D>(P, grid, s)
                 : launch_one<In, Out, Lk, false, Axpy, D>(P, grid, s);
    };
    (one(std::integral_constant<int, Depths>{}), ...);
    return done ? st : set_error(WEO_ERR_UNSUPPORTED, "staged hop: ring depth not compiled");
}

// Fill the parameters and launch. Returns WEO_ERR_UNSUPPORTED when the layout
// does not fit or the depth is not compiled for this format.
template <class In, class Out, class Lk, bool Axpy, int... Depths>
int launch_staged(wilson_eo_s *h, bool dag, const HopParams &p, const char *blocks, int rows,
                  int want_depth, int depth_cap, cudaStream_t s, bool inject)
{
    constexpr bool axpy = Axpy;
    Params P;
    std::memset(&P, 0, sizeof(P));
    const int hx = p.lxh, T = rows * hx;
    make_layout(hx, rows, In::kSite, Lk::kBytesPerSite, axpy, P.L);
    const int depth = pick_depth(P.L, T, want_depth, depth_cap);
    if (!depth) return set_error(WEO_ERR_UNSUPPORTED, "staged hop: ring does not fit");
    bool ok = true;
    if (In::kBoxes)
        ok = encode_spinor_map(&P.sp_tile, p.in, p.vh, T) && encode_spinor_map(&P.sp_row, p.in, p.vh, hx);
    if (ok && axpy) ok = encode_spinor_map(&P.x_tile, p.x, p.vh, T);
    if (!ok) return set_error(WEO_ERR_CUDA, "staged hop: tensor map encoding failed");
    P.in = static_cast<const char *>(p.in);
    P.link_block = 8 * Lk::kBytesPerSite * T;
    P.links = blocks + (long long)p.out_parity * 8 * Lk::kBytesPerSite * p.vh;
    P.out = p.out;
    P.lxh = hx;
    P.ly = p.ly;
    P.lz = p.lz;
    P.lt = p.lt;
    P.rows = rows;
    P.tile = T;
    P.tpt = teams_per_tile(T);
    P.ntiles = (int)(p.vh / T);
    P.out_parity = p.out_parity;
    P.reverse = p.reverse;
    P.vh = p.vh;
    P.a = (float)p.a;
    P.err = static_cast<unsigned int *>(h->fused_ctrl.ptr);
    P.limit_ns = inject ? 2000000ull : 1000000000ull;
    P.inject = inject ? 1 : 0;
    int sms = 0;
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = P.ntiles < sms ? P.ntiles : sms;
    return launch_depths<In, Out, Lk, Axpy, Depths...>(dag, depth, P, grid, s);
}

// 16-bit operators: the first hop reads FP32 planar spinors and writes the
// 16-bit intermediate in row blocks; the second reads the row blocks and
// writes FP32 planar spinors with the axpy of Eq. 4.
template <class Tr>
int launch_16(wilson_eo_s *h, int io, bool c12, bool dag, const HopParams &p, const char *blocks,
              int rows, int want, int cap, cudaStream_t s, bool inject)
{
    using L18 = Lk16_18<Tr, LdPlain>;
    using L12 = Lk16_12<Tr, LdPlain>;
    if (io == IO_TO16)
        return c12 ? launch_staged<InF32, Out16<Tr>, L12, false, 3, 4>(h, dag, p, blocks, rows, want, cap, s, inject)
                   : launch_staged<InF32, Out16<Tr>, L18, false, 3, 4>(h, dag, p, blocks, rows, want, cap, s, inject);
    return c12 ? launch_staged<In16<Tr>, OutF32, L12, true, 3, 4>(h, dag, p, blocks, rows, want, cap, s, inject)
               : launch_staged<In16<Tr>, OutF32, L18, true, 3, 4>(h, dag, p, blocks, rows, want, cap, s, inject);
}

template <class Tr>
int pack_16(const HopParams &p, bool c12, int T, char *out, cudaStream_t s)
{
    return c12 ? pack_link_blocks<Lk16_12<Tr>, Lk16_12<Tr, LdPlain>>(p, T, out, s)
               : pack_link_blocks<Lk16_18<Tr>, Lk16_18<Tr, LdPlain>>(p, T, out, s);
}

}  // namespace staged
}  // namespace weo
