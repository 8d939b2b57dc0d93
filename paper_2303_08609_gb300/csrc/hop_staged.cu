// Hopping kernel with its operands staged in shared memory by TMA: the same
// sum as hop_kernel (Eq. 1 for one parity, Sec. 3.3's H_oe / H_eo pass), FP32
// spinors and 18-real FP32 links, one right-hand side.
//
// The output sites are cut into tiles of R lattice rows: R * Lx/2 consecutive
// compact indices inside one (z, t) plane. Everything the hopping sum of a tile
// reads is then a few contiguous blocks:
//   input spinor (parity 1-p): the tile rows of the same plane (+-x, and +-y
//     inside the tile), the rows y0-1 and y0+R (periodic in y), and the tile
//     rows of the planes z+1, z-1, t+1, t-1 (periodic): seven boxes of the
//     planar array, loaded with cp.async.bulk.tensor;
//   links: the eight links of every output site -- U_mu(x), and U_mu(x-mu)
//     whose adjoint the backward hop applies -- repacked once per gauge field into one block per
//     tile (direction-major, planar inside), so a tile's links are a single
//     cp.async.bulk copy. This doubles the links' footprint (each link is
//     stored for both sites it joins), not their traffic: a hop still reads
//     each stored link once;
//   the axpy addend at the tile: one box.
// One producer thread issues them into a ring of two to five stages, each with
// an mbarrier that counts the bytes landed. Each stage is owned by one group
// of consumer teams, which compute from shared memory only, so the bytes in
// flight no longer depend on the registers each thread holds. A team is two
// warps on 32 sites of the tile: one takes the x and y directions, the other
// the z and t directions, whose partial sums are handed over in shared memory
// (in the slots of the z+1 spinor rows they no longer need); a tile of more
// than 32 sites has two teams.
//
// Every wait is bounded (a time limit on the global timer): on expiry the
// kernel records an error word that wilson_eo_check reports, stops, and the
// producer waits, again bounded, for its own copies still in flight.
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "weo_internal.h"
#include "weo_tma.cuh"

namespace weo {

namespace {

constexpr int kTeams = 6;                        // at most six consumer teams of two warps
constexpr int kConsumerWarps = 2 * kTeams;
constexpr int kStagedThreads = 32 * (kConsumerWarps + 1);
constexpr int kMaxTile = 64;                       // sites per tile (box limits)
constexpr int kMaxStages = 5;
constexpr int kSmemLimit = 227 * 1024;

// shared-memory regions of one stage, byte offsets
struct StageLayout {
    int sp[7];  // spinor: tile rows, row y0-1, row y0+R, planes z+1, z-1, t+1, t-1
    int lk;     // the tile's link block: 8 directions x (4 float4 + 1 float2 planes)
    int x;      // axpy addend
    int bytes;  // size of one stage
    int tx;     // bytes the loads of one tile deliver
};

struct StagedParams {
    CUtensorMap sp_tile, sp_row, x_tile;
    const char *links;  // link blocks of this output parity, 576 T bytes per tile
    StageLayout L;
    int lxh, ly, lz, lt, rows, tile, ntiles, out_parity, reverse;
    int tpt;     // teams per tile (32 sites each): 1 or 2
    long long vh;
    float a;
    float2 *out;
    unsigned int *err;
    unsigned long long limit_ns;
    int inject;  // failure-path test: the producer never loads the CTA's first tile
    // several right-hand sides (hop_staged_mrhs_kernel): the spinor maps are
    // 3D (rhs outermost); output r at out + r * out_stride (complex)
    int nrhs;
    long long out_stride;
};

// shared memory of the multi-RHS kernel: two link slots (a tile's links stay
// while all its right-hand sides pass) and a ring of spinor stages
struct MrhsLayout {
    int lk[2];   // link blocks of two tiles
    int base;    // first spinor stage
    StageLayout S;  // one spinor stage (S.lk unused)
};

int round128(int b) { return (b + 127) & ~127; }

// bytes of `stages` stages plus their mbarriers
size_t staged_smem(const StageLayout &L, int stages)
{
    return (size_t)stages * L.bytes + (2 * stages + kTeams) * sizeof(uint64_t);
}

bool make_layout(int lxh, int rows, bool axpy, StageLayout &L)
{
    const int T = lxh * rows;
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off += round128(bytes);
        return o;
    };
    L.sp[0] = take(96 * T);
    L.sp[1] = take(96 * lxh);
    L.sp[2] = take(96 * lxh);
    for (int k = 3; k < 7; ++k) L.sp[k] = take(96 * T);
    L.lk = take(576 * T);
    L.x = axpy ? take(96 * T) : 0;
    L.bytes = off;
    L.tx = 5 * 96 * T + 2 * 96 * lxh + 576 * T + (axpy ? 96 * T : 0);
    return staged_smem(L, 2) <= kSmemLimit;
}

// wait for the phase of `bar` with the given parity to complete, at most
// limit_ns nanoseconds; false (and the error word set) on expiry
__device__ __noinline__ bool mbar_wait(uint64_t *bar, unsigned parity, const StagedParams &P)
{
    return mbar_wait_bounded(bar, parity, P.limit_ns, P.err);
}

// ---------------------------------------------------------------- tiles --
struct TileGeo {
    int plane, y0, z, t;
    long long i0;  // first compact index of the tile
};

__device__ __forceinline__ TileGeo tile_geo(const StagedParams &P, int j)
{
    if (P.reverse) j = P.ntiles - 1 - j;
    TileGeo g;
    const int row0 = j * P.rows;
    g.plane = row0 / P.ly;
    g.y0 = row0 - g.plane * P.ly;
    g.z = g.plane % P.lz;
    g.t = g.plane / P.lz;
    g.i0 = (long long)row0 * P.lxh;
    return g;
}

// compact index of row y of plane (z, t)
__device__ __forceinline__ int row_start(const StagedParams &P, int z, int t, int y)
{
    return ((t * P.lz + z) * P.ly + y) * P.lxh;
}

// issue the loads of tile j into the stage at `base`
template <bool Axpy>
__device__ __forceinline__ void issue_tile(const StagedParams &P, int j, char *base, uint64_t *full,
                                           uint64_t pol)
{
    const TileGeo g = tile_geo(P, j);
    const StageLayout &L = P.L;
    const int ly = P.ly, lz = P.lz, lt = P.lt;
    const int ym = g.y0 == 0 ? ly - 1 : g.y0 - 1;
    const int yp = g.y0 + P.rows == ly ? 0 : g.y0 + P.rows;
    const int zp = g.z + 1 == lz ? 0 : g.z + 1, zm = g.z == 0 ? lz - 1 : g.z - 1;
    const int tp = g.t + 1 == lt ? 0 : g.t + 1, tm = g.t == 0 ? lt - 1 : g.t - 1;
    const int i0 = (int)g.i0;
    const int jt = (int)(g.i0 / P.tile);  // tile index in memory order
    mbar_expect_tx(full, (unsigned)L.tx);
    // the links are read once per launch: evict first
    bulk_hint(base + L.lk, P.links + (long long)jt * 576 * P.tile, (unsigned)(576 * P.tile), full, pol);
    // input spinor (parity 1-p); the coordinate is in floats, 2 per complex
    tma_2d(base + L.sp[0], &P.sp_tile, 2 * i0, 0, full);
    tma_2d(base + L.sp[1], &P.sp_row, 2 * row_start(P, g.z, g.t, ym), 0, full);
    tma_2d(base + L.sp[2], &P.sp_row, 2 * row_start(P, g.z, g.t, yp), 0, full);
    tma_2d(base + L.sp[3], &P.sp_tile, 2 * row_start(P, zp, g.t, g.y0), 0, full);
    tma_2d(base + L.sp[4], &P.sp_tile, 2 * row_start(P, zm, g.t, g.y0), 0, full);
    tma_2d(base + L.sp[5], &P.sp_tile, 2 * row_start(P, g.z, tp, g.y0), 0, full);
    tma_2d(base + L.sp[6], &P.sp_tile, 2 * row_start(P, g.z, tm, g.y0), 0, full);
    if (Axpy) tma_2d(base + L.x, &P.x_tile, 2 * i0, 0, full);
}

template <bool Dag, bool Axpy, int NS>
__global__ void __launch_bounds__(kStagedThreads, 1) hop_staged_kernel(const __grid_constant__ StagedParams P)
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
        for (int t = 0; t < kTeams; ++t) mbar_init(ready + t, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 2 * NS * P.tpt) {  // producer
        if (lane != 0) return;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.sp_tile)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.sp_row)) : "memory");
        if (Axpy)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.x_tile)) : "memory");
        const uint64_t pol = policy_evict_first();
        int issued = 0;
        for (int k = 0; k < ntile_cta; ++k) {
            const int s = k % NS, n = k / NS;
            if (n >= 1 && !mbar_wait(empty + s, (unsigned)((n - 1) & 1), P)) break;
            if (P.inject && k == 0) continue;  // nothing loaded, nothing in flight
            issue_tile<Axpy>(P, (int)blockIdx.x + k * (int)gridDim.x, smem + s * L.bytes,
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
    // = tpt teams owning stage g and the CTA's tiles k = g, g + NS, ... Each
    // barrier's waiter thus always waits for the phase after the one it saw last.
    const int team = warp >> 1, q = warp & 1;
    const int g = team / P.tpt;
    const int s = (team - g * P.tpt) * 32 + lane;  // site within the tile
    const bool active = s < P.tile;
    const int lxh = P.lxh, T = P.tile;
    const int r = s / lxh, xh = s - r * lxh;
    constexpr int S0 = Dag ? -1 : 1;
    const int st = g;
    char *base = smem + st * L.bytes;
    for (int k = g; k < ntile_cta; k += NS) {
        const unsigned m = (unsigned)(k / NS);  // use of this stage
        if (!mbar_wait(full + st, m & 1u, P)) return;
        const float2 *sp0 = reinterpret_cast<const float2 *>(base + L.sp[0]);
        float2 *part = reinterpret_cast<float2 *>(base + L.sp[3]);  // z/t partial sums
        const TileGeo tg = tile_geo(P, (int)blockIdx.x + k * (int)gridDim.x);
        cx<float> acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {0.f, 0.f};
        if (q == 0) {
            if (active) {
                const int y = tg.y0 + r;
                const int par = (y + tg.z + tg.t + P.out_parity) & 1;
                const int xp = par ? (xh + 1 == lxh ? 0 : xh + 1) : xh;
                const int xm = par ? xh : (xh == 0 ? lxh - 1 : xh - 1);
                const int rb = r * lxh;
                // direction d = 2 mu + (backward): links at lk + 72 T d, site s
                const float4 *l4 = reinterpret_cast<const float4 *>(base + L.lk);
                const float2 *l2 = reinterpret_cast<const float2 *>(base + L.lk + 64 * T);
                const int ld4 = 18 * T / 4, ld2 = 9 * T;  // one direction, in float4 / float2
                staged_dir<0, true, S0>(acc, sp0, T, rb + xp, l4, l2, T, s);
                staged_dir<0, false, S0>(acc, sp0, T, rb + xm, l4 + ld4, l2 + ld2, T, s);
                if (r + 1 < P.rows)
                    staged_dir<1, true, S0>(acc, sp0, T, rb + lxh + xh, l4 + 2 * ld4, l2 + 2 * ld2, T, s);
                else
                    staged_dir<1, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[2]),
                                            lxh, xh, l4 + 2 * ld4, l2 + 2 * ld2, T, s);
                if (r > 0)
                    staged_dir<1, false, S0>(acc, sp0, T, rb - lxh + xh, l4 + 3 * ld4, l2 + 3 * ld2, T, s);
                else
                    staged_dir<1, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[1]),
                                             lxh, xh, l4 + 3 * ld4, l2 + 3 * ld2, T, s);
            }
            if (!mbar_wait(ready + team, m & 1u, P)) return;
            if (active) {
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const float2 v = part[c * T + s];
                    acc[c].r += v.x;
                    acc[c].i += v.y;
                }
                float2 *out = P.out + tg.i0 + s;
                if (Axpy) {
                    const float2 *xv = reinterpret_cast<const float2 *>(base + L.x);
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        const float2 v = xv[c * T + s];
                        out[c * P.vh] = make_float2(fmaf(P.a, acc[c].r, v.x), fmaf(P.a, acc[c].i, v.y));
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 12; ++c) out[c * P.vh] = make_float2(acc[c].r, acc[c].i);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + st);
        } else {
            if (active) {
                const float4 *l4 = reinterpret_cast<const float4 *>(base + L.lk);
                const float2 *l2 = reinterpret_cast<const float2 *>(base + L.lk + 64 * T);
                const int ld4 = 18 * T / 4, ld2 = 9 * T;
                staged_dir<2, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[3]), T, s,
                                        l4 + 4 * ld4, l2 + 4 * ld2, T, s);
                staged_dir<2, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[4]), T, s,
                                         l4 + 5 * ld4, l2 + 5 * ld2, T, s);
                staged_dir<3, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[5]), T, s,
                                        l4 + 6 * ld4, l2 + 6 * ld2, T, s);
                staged_dir<3, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[6]), T, s,
                                         l4 + 7 * ld4, l2 + 7 * ld2, T, s);
                // each lane overwrites only the z+1 slots it read itself
#pragma unroll
                for (int c = 0; c < 12; ++c) part[c * T + s] = make_float2(acc[c].r, acc[c].i);
            }
            // the next TMA load into this stage writes over the partial sums
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(ready + team);
        }
    }
}

// Several right-hand sides: item k of a CTA is (tile m = k / nrhs, rhs r =
// k % nrhs). A tile's link block is loaded once, into slot m % 2, and serves
// all its right-hand sides; the spinor boxes of each item go through a ring of
// NS stages owned by NS consumer groups (item k -> group k % NS). With
// NS <= nrhs every group meets every tile, so each waiter again waits for the
// phase right after the one it saw last.
template <bool Dag, bool Axpy, int NS>
__global__ void __launch_bounds__(kStagedThreads, 1) hop_staged_mrhs_kernel(const __grid_constant__ StagedParams P,
                                                                           const __grid_constant__ MrhsLayout M)
{
    extern __shared__ __align__(128) char smem[];
    const StageLayout &L = M.S;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + M.base + NS * L.bytes);
    uint64_t *empty = full + NS;
    uint64_t *lfull = empty + NS;  // link slots
    uint64_t *lempty = lfull + 2;
    uint64_t *ready = lempty + 2;  // per team
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int ntile_cta =
        P.ntiles > (int)blockIdx.x ? (P.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nitems = ntile_cta * P.nrhs;
    const int T = P.tile;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, (unsigned)P.tpt);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(lfull + s, 1);
            mbar_init(lempty + s, (unsigned)(P.tpt * P.nrhs));  // every item of the tile
        }
        for (int t = 0; t < kTeams; ++t) mbar_init(ready + t, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 2 * NS * P.tpt) {  // producer
        if (lane != 0) return;
        const uint64_t pol = policy_evict_first();
        int issued = 0, tiles_issued = 0;
        bool ok = true;
        for (int k = 0; k < nitems && ok; ++k) {
            const int m = k / P.nrhs, r = k - m * P.nrhs;
            const TileGeo g = tile_geo(P, (int)blockIdx.x + m * (int)gridDim.x);
            if (r == 0) {  // the tile's links, once
                const int ls = m & 1, n = m >> 1;
                if (n >= 1 && !mbar_wait(lempty + ls, (unsigned)((n - 1) & 1), P)) break;
                mbar_expect_tx(lfull + ls, (unsigned)(576 * T));
                bulk_hint(smem + M.lk[ls], P.links + (g.i0 / T) * 576 * T, (unsigned)(576 * T),
                          lfull + ls, pol);
                tiles_issued = m + 1;
            }
            const int st = k % NS, u = k / NS;
            if (u >= 1 && !mbar_wait(empty + st, (unsigned)((u - 1) & 1), P)) break;
            char *base = smem + M.base + st * L.bytes;
            const int ly = P.ly, lz = P.lz, lt = P.lt;
            const int ym = g.y0 == 0 ? ly - 1 : g.y0 - 1;
            const int yp = g.y0 + P.rows == ly ? 0 : g.y0 + P.rows;
            const int zp = g.z + 1 == lz ? 0 : g.z + 1, zm = g.z == 0 ? lz - 1 : g.z - 1;
            const int tp = g.t + 1 == lt ? 0 : g.t + 1, tm = g.t == 0 ? lt - 1 : g.t - 1;
            mbar_expect_tx(full + st, (unsigned)L.tx);
            tma_3d(base + L.sp[0], &P.sp_tile, 2 * (int)g.i0, 0, r, full + st);
            tma_3d(base + L.sp[1], &P.sp_row, 2 * row_start(P, g.z, g.t, ym), 0, r, full + st);
            tma_3d(base + L.sp[2], &P.sp_row, 2 * row_start(P, g.z, g.t, yp), 0, r, full + st);
            tma_3d(base + L.sp[3], &P.sp_tile, 2 * row_start(P, zp, g.t, g.y0), 0, r, full + st);
            tma_3d(base + L.sp[4], &P.sp_tile, 2 * row_start(P, zm, g.t, g.y0), 0, r, full + st);
            tma_3d(base + L.sp[5], &P.sp_tile, 2 * row_start(P, g.z, tp, g.y0), 0, r, full + st);
            tma_3d(base + L.sp[6], &P.sp_tile, 2 * row_start(P, g.z, tm, g.y0), 0, r, full + st);
            if (Axpy) tma_3d(base + L.x, &P.x_tile, 2 * (int)g.i0, 0, r, full + st);
            issued = k + 1;
        }
        // the last loads of each stage and link slot must land before the CTA exits
        for (int k = issued - 1; k >= 0 && k >= issued - NS; --k)
            mbar_wait(full + k % NS, (unsigned)((k / NS) & 1), P);
        for (int m = tiles_issued - 1; m >= 0 && m >= tiles_issued - 2; --m)
            mbar_wait(lfull + (m & 1), (unsigned)((m >> 1) & 1), P);
        return;
    }

    const int team = warp >> 1, q = warp & 1;
    const int g = team / P.tpt;
    const int s = (team - g * P.tpt) * 32 + lane;
    const bool active = s < T;
    const int lxh = P.lxh;
    const int r0 = s / lxh, xh = s - r0 * lxh;
    constexpr int S0 = Dag ? -1 : 1;
    char *base = smem + M.base + g * L.bytes;
    const float2 *sp0 = reinterpret_cast<const float2 *>(base + L.sp[0]);
    float2 *part = reinterpret_cast<float2 *>(base + L.sp[3]);
    const int ld4 = 18 * T / 4, ld2 = 9 * T;
    for (int k = g; k < nitems; k += NS) {
        const int m = k / P.nrhs, rhs = k - m * P.nrhs;
        const unsigned u = (unsigned)(k / NS);
        if (!mbar_wait(lfull + (m & 1), (unsigned)((m >> 1) & 1), P)) return;
        if (!mbar_wait(full + g, u & 1u, P)) return;
        const char *lk = smem + M.lk[m & 1];
        const float4 *l4 = reinterpret_cast<const float4 *>(lk);
        const float2 *l2 = reinterpret_cast<const float2 *>(lk + 64 * T);
        const TileGeo tg = tile_geo(P, (int)blockIdx.x + m * (int)gridDim.x);
        cx<float> acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {0.f, 0.f};
        if (q == 0) {
            if (active) {
                const int par = (tg.y0 + r0 + tg.z + tg.t + P.out_parity) & 1;
                const int xp = par ? (xh + 1 == lxh ? 0 : xh + 1) : xh;
                const int xm = par ? xh : (xh == 0 ? lxh - 1 : xh - 1);
                const int rb = r0 * lxh;
                staged_dir<0, true, S0>(acc, sp0, T, rb + xp, l4, l2, T, s);
                staged_dir<0, false, S0>(acc, sp0, T, rb + xm, l4 + ld4, l2 + ld2, T, s);
                if (r0 + 1 < P.rows)
                    staged_dir<1, true, S0>(acc, sp0, T, rb + lxh + xh, l4 + 2 * ld4, l2 + 2 * ld2, T, s);
                else
                    staged_dir<1, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[2]),
                                            lxh, xh, l4 + 2 * ld4, l2 + 2 * ld2, T, s);
                if (r0 > 0)
                    staged_dir<1, false, S0>(acc, sp0, T, rb - lxh + xh, l4 + 3 * ld4, l2 + 3 * ld2, T, s);
                else
                    staged_dir<1, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[1]),
                                             lxh, xh, l4 + 3 * ld4, l2 + 3 * ld2, T, s);
            }
            if (!mbar_wait(ready + team, u & 1u, P)) return;
            if (active) {
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const float2 v = part[c * T + s];
                    acc[c].r += v.x;
                    acc[c].i += v.y;
                }
                float2 *out = P.out + rhs * P.out_stride + tg.i0 + s;
                if (Axpy) {
                    const float2 *xv = reinterpret_cast<const float2 *>(base + L.x);
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        const float2 v = xv[c * T + s];
                        out[c * P.vh] = make_float2(fmaf(P.a, acc[c].r, v.x), fmaf(P.a, acc[c].i, v.y));
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 12; ++c) out[c * P.vh] = make_float2(acc[c].r, acc[c].i);
                }
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(empty + g);
                mbar_arrive(lempty + (m & 1));
            }
        } else {
            if (active) {
                staged_dir<2, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[3]), T, s,
                                        l4 + 4 * ld4, l2 + 4 * ld2, T, s);
                staged_dir<2, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[4]), T, s,
                                         l4 + 5 * ld4, l2 + 5 * ld2, T, s);
                staged_dir<3, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[5]), T, s,
                                        l4 + 6 * ld4, l2 + 6 * ld2, T, s);
                staged_dir<3, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[6]), T, s,
                                         l4 + 7 * ld4, l2 + 7 * ld2, T, s);
#pragma unroll
                for (int c = 0; c < 12; ++c) part[c * T + s] = make_float2(acc[c].r, acc[c].i);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(ready + team);
        }
    }
}

// ----------------------------------------------------------- link blocks --
// Link block of output parity p for tile size T: for output site i (tile
// i / T, site s = i % T), direction d = 2 mu + b holds U_mu(x) (b = 0) or
// U_mu(x - mu) (b = 1) as 4 float4 planes then 1 float2 plane of T sites:
// block(i / T) + 72 T d + 16 T k + 16 s, block + 72 T d + 64 T + 8 s.
__global__ void pack_link_blocks_kernel(const HopParams p, int T, float *out)
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
    const long long tile = i / T, s = i % T;
    char *blk = reinterpret_cast<char *>(out) + tile * 576 * T;
    for (int mu = 0; mu < 4; ++mu)
        for (int b = 0; b < 2; ++b) {
            cx<double> U[3][3];
            const char *f = p.gauge + (2 * mu + (b ? p.out_parity ^ 1 : p.out_parity)) * p.gauge_pb;
            LkF32_18::load(f, p.vh, b ? nb[mu] : i, U);
            char *d = blk + 72ll * T * (2 * mu + b);
            float4 *q4 = reinterpret_cast<float4 *>(d) + s;
            q4[0] = make_float4(U[0][0].r, U[0][0].i, U[0][1].r, U[0][1].i);
            q4[T] = make_float4(U[0][2].r, U[0][2].i, U[1][0].r, U[1][0].i);
            q4[2 * T] = make_float4(U[1][1].r, U[1][1].i, U[1][2].r, U[1][2].i);
            q4[3 * T] = make_float4(U[2][0].r, U[2][0].i, U[2][1].r, U[2][1].i);
            reinterpret_cast<float2 *>(d + 64ll * T)[s] = make_float2(U[2][2].r, U[2][2].i);
        }
}

// rows of R per tile: R divides Ly, R >= 2, R * Lx/2 <= 64; the largest such
// R, or the requested one when it qualifies (0 if none does)
int staged_rows(int lxh, int ly, int want = 0)
{
    if (lxh % 2 != 0) return 0;  // rows must start on 16-byte boundaries
    auto ok = [&](int r) { return r >= 2 && ly % r == 0 && r * lxh <= kMaxTile; };
    if (want) return ok(want) ? want : 0;
    for (int r = kMaxTile / lxh; r >= 2; --r)
        if (ok(r)) return r;
    return 0;
}

// ring depth (= tiles computed at once, one group of teams per stage): the
// requested one if it fits in shared memory and in six teams, else the most
// that fit (at most 3)
int staged_depth(const StageLayout &L, int tile, int want)
{
    const int tpt = tile > 32 ? 2 : 1;
    auto ok = [&](int d) {
        return d >= 2 && d <= kMaxStages && d * tpt <= kTeams && staged_smem(L, d) <= kSmemLimit;
    };
    if (want) return ok(want) ? want : 0;
    for (int d = 3; d >= 2; --d)
        if (ok(d)) return d;
    return 0;
}

template <bool Dag, bool Axpy, int NS>
int launch_staged(const StagedParams &P, int grid, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(hop_staged_kernel<Dag, Axpy, NS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    });
    WEO_CUDA(attr);
    const int threads = 32 * (2 * NS * P.tpt + 1);  // NS x tpt teams and the producer
    hop_staged_kernel<Dag, Axpy, NS><<<grid, threads, staged_smem(P.L, NS), s>>>(P);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

// multi-RHS layout: two link slots, then `stages` spinor stages (no link
// region inside a stage); mbarriers after them
size_t mrhs_smem(const MrhsLayout &M, int stages)
{
    return (size_t)M.base + (size_t)stages * M.S.bytes + (2 * stages + 4 + kTeams) * sizeof(uint64_t);
}

void make_mrhs_layout(int lxh, int rows, bool axpy, MrhsLayout &M)
{
    const int T = lxh * rows;
    M.lk[0] = 0;
    M.lk[1] = round128(576 * T);
    M.base = 2 * round128(576 * T);
    StageLayout &L = M.S;
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off += round128(bytes);
        return o;
    };
    L.sp[0] = take(96 * T);
    L.sp[1] = take(96 * lxh);
    L.sp[2] = take(96 * lxh);
    for (int k = 3; k < 7; ++k) L.sp[k] = take(96 * T);
    L.lk = 0;
    L.x = axpy ? take(96 * T) : 0;
    L.bytes = off;
    L.tx = 5 * 96 * T + 2 * 96 * lxh + (axpy ? 96 * T : 0);
}

template <bool Dag, bool Axpy, int NS>
int launch_mrhs(const StagedParams &P, const MrhsLayout &M, int grid, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(hop_staged_mrhs_kernel<Dag, Axpy, NS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    });
    WEO_CUDA(attr);
    const int threads = 32 * (2 * NS * P.tpt + 1);
    hop_staged_mrhs_kernel<Dag, Axpy, NS><<<grid, threads, mrhs_smem(M, NS), s>>>(P, M);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <int NS>
int launch_depth(bool dag, bool axpy, const StagedParams &P, int grid, cudaStream_t s)
{
    if (dag) return axpy ? launch_staged<true, true, NS>(P, grid, s) : launch_staged<true, false, NS>(P, grid, s);
    return axpy ? launch_staged<false, true, NS>(P, grid, s) : launch_staged<false, false, NS>(P, grid, s);
}

}  // namespace

// -------------------------------------------------------- tensor maps --
EncodeFn tma_encoder()
{
    static std::once_flag once;
    static EncodeFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

// FP32 tensor of rank 2 or 3 (dims[0] contiguous; strides in bytes of dims 1..)
bool tma_encode(CUtensorMap *m, const void *ptr, int rank, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box)
{
    EncodeFn fn = tma_encoder();
    if (!fn) return false;
    const cuuint32_t one[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(ptr), dims,
              strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tile rows and ring depth a handle's staged hops use (0, 0 if not eligible)
void staged_shape(const wilson_eo_s *h, int *rows_out, int *depth_out)
{
    const int lxh = h->dims[0] / 2;
    StageLayout L;
    int rows = staged_rows(lxh, h->dims[1], h->staged_rows), depth = 0;
    // TMA coordinates are 32-bit: 2 floats per site in the spinor boxes
    if (rows >= 2 && make_layout(lxh, rows, true, L) && 2 * h->vh < (1ll << 31))
        depth = staged_depth(L, rows * lxh, h->staged_depth);
    if (!depth) rows = 0;
    *rows_out = rows;
    *depth_out = depth;
}

bool staged_eligible(const wilson_eo_s *h)
{
    int rows, depth;
    staged_shape(h, &rows, &depth);
    return depth > 0 && tma_encoder() != nullptr;
}

bool staged_arrays_ok(const HopParams &p, bool axpy)
{
    auto aligned = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    return aligned(p.in) && (!axpy || aligned(p.x));
}

// Link blocks of both output parities for the FP32 18-real field g, at the
// handle's tile size (allocates; not while `s` is being captured).
int staged_prepare(wilson_eo_s *h, const PackedGauge &g, cudaStream_t s)
{
    if (!h->cfg[WEO_F32].staged || g.prec != WEO_F32 || g.fmt != WEO_LINK18) return WEO_OK;
    int rows, depth;
    staged_shape(h, &rows, &depth);
    if (!depth) return WEO_OK;
    const int T = rows * (h->dims[0] / 2);
    if (h->staged_valid && h->staged_src == g.buf.ptr && h->staged_gen == g.gen && h->staged_tile == T)
        return WEO_OK;
    WEO_TRY(h->staged_links.ensure((size_t)2 * 576 * h->vh));
    HopParams p = geom_params(h);
    p.gauge = static_cast<const char *>(g.buf.ptr);
    p.gauge_pb = g.pb;
    for (int par = 0; par < 2; ++par) {
        p.out_parity = par;
        pack_link_blocks_kernel<<<(unsigned)((h->vh + 255) / 256), 256, 0, s>>>(
            p, T, reinterpret_cast<float *>(static_cast<char *>(h->staged_links.ptr) + par * 576 * h->vh));
        WEO_CUDA(cudaGetLastError());
    }
    h->staged_valid = true;
    h->staged_src = g.buf.ptr;
    h->staged_gen = g.gen;
    h->staged_tile = T;
    return WEO_OK;
}

// the link blocks for gauge pointer `gauge`, if current
static const char *staged_blocks(const wilson_eo_s *h, const char *gauge, int T)
{
    const PackedGauge *g = gauge == h->gauge.buf.ptr ? &h->gauge
                         : gauge == h->gauge_lo.buf.ptr ? &h->gauge_lo
                                                        : nullptr;
    if (!g || !h->staged_valid || h->staged_src != g->buf.ptr || h->staged_gen != g->gen ||
        h->staged_tile != T)
        return nullptr;
    return static_cast<const char *>(h->staged_links.ptr);
}

bool staged_ready(wilson_eo_s *h, const HopParams &p, cudaStream_t s)
{
    int rows, depth;
    staged_shape(h, &rows, &depth);
    if (!depth) return false;
    const int T = rows * p.lxh;
    if (staged_blocks(h, p.gauge, T)) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    const PackedGauge *g = p.gauge == h->gauge.buf.ptr ? &h->gauge
                         : p.gauge == h->gauge_lo.buf.ptr ? &h->gauge_lo
                                                          : nullptr;
    return g && staged_prepare(h, *g, s) == WEO_OK && staged_blocks(h, p.gauge, T) != nullptr;
}

int launch_hop_staged(wilson_eo_s *h, bool dag, bool axpy, const HopParams &p, cudaStream_t s,
                      bool inject)
{
    const int lxh = p.lxh;
    int rows, depth;
    staged_shape(h, &rows, &depth);
    const char *blocks = depth ? staged_blocks(h, p.gauge, rows * lxh) : nullptr;
    if (!blocks || !staged_arrays_ok(p, axpy) || !h->fused_ctrl.ptr)
        return set_error(WEO_ERR_UNSUPPORTED, "staged hop: lattice, link blocks or array alignment not ready");
    StagedParams P;
    std::memset(&P, 0, sizeof(P));
    make_layout(lxh, rows, axpy, P.L);
    const long long vh = p.vh;
    const int T = rows * lxh;
    const int nrhs = p.nrhs;
    // spinor: [rhs][12 planes][2 vh floats]; one right-hand side: 2D maps
    const cuuint64_t sd[3] = {(cuuint64_t)(2 * vh), 12, (cuuint64_t)nrhs};
    const cuuint64_t ss[2] = {(cuuint64_t)(8 * vh), (cuuint64_t)p.in_stride};
    const cuuint64_t sx[2] = {(cuuint64_t)(8 * vh), (cuuint64_t)p.x_stride};
    const cuuint32_t b_tile[3] = {(cuuint32_t)(2 * T), 12, 1}, b_row[3] = {(cuuint32_t)(2 * lxh), 12, 1};
    const int rank = nrhs > 1 ? 3 : 2;
    if (nrhs > 1 && ((p.in_stride & 15) || (axpy && (p.x_stride & 15)) || (p.out_stride & 7)))
        return set_error(WEO_ERR_UNSUPPORTED, "staged hop: right-hand-side strides not aligned");
    bool ok = tma_encode(&P.sp_tile, p.in, rank, sd, ss, b_tile) && tma_encode(&P.sp_row, p.in, rank, sd, ss, b_row);
    if (ok && axpy) ok = tma_encode(&P.x_tile, p.x, rank, sd, sx, b_tile);
    if (!ok) return set_error(WEO_ERR_CUDA, "staged hop: tensor map encoding failed");
    P.links = blocks + (long long)p.out_parity * 576 * vh;
    P.lxh = lxh;
    P.ly = p.ly;
    P.lz = p.lz;
    P.lt = p.lt;
    P.rows = rows;
    P.tile = T;
    P.tpt = T > 32 ? 2 : 1;
    P.ntiles = (int)(vh / T);
    P.out_parity = p.out_parity;
    P.reverse = p.reverse;
    P.vh = vh;
    P.a = (float)p.a;
    P.out = static_cast<float2 *>(p.out);
    P.err = static_cast<unsigned int *>(h->fused_ctrl.ptr);
    P.limit_ns = inject ? 2000000ull : 1000000000ull;
    P.inject = inject ? 1 : 0;
    int sms = 0;
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = P.ntiles < sms ? P.ntiles : sms;
    if (nrhs > 1) {
        // links once per tile for all right-hand sides; spinor ring of 2 or 3
        P.nrhs = nrhs;
        P.out_stride = p.out_stride / 8;
        MrhsLayout M;
        make_mrhs_layout(lxh, rows, axpy, M);
        int ns = nrhs < 3 ? nrhs : 3;
        while (ns > 2 && (mrhs_smem(M, ns) > kSmemLimit || ns * P.tpt > kTeams)) --ns;
        if (mrhs_smem(M, ns) > kSmemLimit || ns * P.tpt > kTeams)
            return set_error(WEO_ERR_UNSUPPORTED, "staged hop: multi-RHS ring does not fit");
        if (ns == 2)
            return dag ? (axpy ? launch_mrhs<true, true, 2>(P, M, grid, s) : launch_mrhs<true, false, 2>(P, M, grid, s))
                       : (axpy ? launch_mrhs<false, true, 2>(P, M, grid, s) : launch_mrhs<false, false, 2>(P, M, grid, s));
        return dag ? (axpy ? launch_mrhs<true, true, 3>(P, M, grid, s) : launch_mrhs<true, false, 3>(P, M, grid, s))
                   : (axpy ? launch_mrhs<false, true, 3>(P, M, grid, s) : launch_mrhs<false, false, 3>(P, M, grid, s));
    }
    switch (depth) {
    case 2: return launch_depth<2>(dag, axpy, P, grid, s);
    case 3: return launch_depth<3>(dag, axpy, P, grid, s);
    case 4: return launch_depth<4>(dag, axpy, P, grid, s);
    default: return launch_depth<5>(dag, axpy, P, grid, s);
    }
}

}  // namespace weo
