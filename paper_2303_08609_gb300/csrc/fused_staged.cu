// Fused M_eo through the TMA-staged pipeline: both hops of Eq. 4 in one
// persistent launch, FP32 spinors, 18-real FP32 links, one right-hand side.
//
// The lattice is cut into the tiles of the staged hop (R rows of one (z, t)
// plane, T = R Lx/2 sites of each parity). Work items are
//   A(tile): tmp = H_oe in onto the tile's odd sites, and
//   B(tile): out = in - kappa^2 H_eo tmp onto the tile's even sites,
// in the wavefront order of the fused kernel: slice tasks A(Lt-1), A(0) ..
// A(D-1), then A(t+D) and B(t) in turn, each task the tiles of one t-slice.
// The queue is dealt round robin to the CTAs (one per SM, all resident: the
// launch is cooperative), each taking its items in queue order. B(t) reads the
// intermediate at slices t-1, t and t+1, so the producer issues its loads only
// after A(t-1), A(t), A(t+1) have published completion (slices it has seen
// complete are remembered). Every wait is for items earlier in the queue, and
// every CTA works through its items in queue order, so the earliest unfinished
// item never waits and the launch always progresses (every wait is bounded all
// the same).
//
// Links: one pair block per tile holds the links owned by the tile's sites of
// both parities, each link stored once: fields (4 float4 planes + 1 float2
// plane each)
//     eYh | oZ oT oX oY eX eY eZ eT | oYh
// where oX = U_x at the tile's odd sites (T of them), eY = U_y at its even
// sites, and eYh / oYh = U_y at the Lx/2 sites of the row just below the tile
// (y0 - 1), which the tile's first row needs for its backward y hop. A copies
// eYh .. eY of its own block (forward links at odd sites, backward x / y links
// at even sites) plus eZ of the tile in plane z-1 and eT of the tile in plane
// t-1; B copies oX .. oYh plus oZ of tile (z-1) and oT of tile (t-1). Both hops
// read the same block bytes, so with B running a few slices after A the
// second read of a link comes from L2, and a link leaves HBM about once per
// M_eo.
// The blocks take 576 T + 144 Lx/2 bytes per tile: the packed field plus the
// halo rows (+6 % at 32^3 x 64).
//
// Per item the producer issues three bulk copies of link fields and seven
// spinor tensor boxes (tile rows, rows y0-1 and y0+R, planes z+-1, t+-1) into
// a ring of stages; the consumers are the staged hop's teams (one warp on the
// x and y directions, one on z and t, partial sums handed over in shared
// memory). A items store the odd intermediate with generic stores, fence them
// for the async proxy and count them per slice; the axpy addend of B items is
// read from global memory by the x/y warp while the partial sums arrive.
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "weo_internal.h"
#include "weo_tma.cuh"

namespace weo {

namespace {

constexpr int kFsTeams = 6;
constexpr int kFsMaxStages = 3;
constexpr int kFsSmemLimit = 227 * 1024;

// byte offsets of the fields of a pair block (and of the link region of a stage)
struct PairFields {
    int eYh, oZ, oT, oX, oY, eX, eY, eZ, eT, oYh, bytes;
};

__host__ __device__ inline PairFields pair_fields(int T, int lxh)
{
    PairFields f;
    f.eYh = 0;
    f.oZ = 72 * lxh;
    f.oT = f.oZ + 72 * T;
    f.oX = f.oT + 72 * T;
    f.oY = f.oX + 72 * T;
    f.eX = f.oY + 72 * T;
    f.eY = f.eX + 72 * T;
    f.eZ = f.eY + 72 * T;
    f.eT = f.eZ + 72 * T;
    f.oYh = f.eT + 72 * T;
    f.bytes = f.oYh + 72 * lxh;
    return f;
}

int round128f(int b) { return (b + 127) & ~127; }

struct FsLayout {
    int sp[7];   // spinor boxes: tile rows, row y0-1, row y0+R, planes z+1, z-1, t+1, t-1
    int lk;      // link region (pair-block layout)
    int bytes;   // one stage
    int tx_a, tx_b;  // bytes an A / B item's copies deliver
};

bool make_fs_layout(int lxh, int rows, FsLayout &L)
{
    const int T = lxh * rows;
    int off = 0;
    auto take = [&](int bytes) {
        const int o = off;
        off += round128f(bytes);
        return o;
    };
    L.sp[0] = take(96 * T);
    L.sp[1] = take(96 * lxh);
    L.sp[2] = take(96 * lxh);
    for (int k = 3; k < 7; ++k) L.sp[k] = take(96 * T);
    const PairFields f = pair_fields(T, lxh);
    L.lk = take(f.bytes);
    L.bytes = off;
    const int spin = 5 * 96 * T + 2 * 96 * lxh;
    L.tx_a = spin + (f.eY + 72 * T) + 2 * 72 * T;        // eYh .. eY, eZ', eT'
    L.tx_b = spin + (f.bytes - f.oX) + 2 * 72 * T;       // oX .. oYh, oZ', oT'
    return true;
}

size_t fs_smem(const FsLayout &L, int stages)
{
    return (size_t)stages * L.bytes + (2 * stages + kFsTeams) * sizeof(uint64_t) + kFsMaxStages * sizeof(int);
}

struct FsParams {
    CUtensorMap in_tile, in_row, mid_tile, mid_row;
    const char *blocks;  // pair blocks, f.bytes each, in tile order
    FsLayout L;
    int lxh, ly, lz, lt, rows, tile, tpt, tps, lookahead, total;
    long long vh;
    float a;
    const float2 *in;    // even input (axpy addend of B)
    float2 *mid;         // odd intermediate
    float2 *out;         // even output
    unsigned int *ctrl;  // [0] sticky error, [1] unused, [2] this launch's error, [3 ..) per-slice counts
    unsigned long long limit_ns;
    int inject;          // failure-path test: A items never publish completion
};

__device__ __forceinline__ unsigned fs_ld_acquire(const unsigned int *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fs_fail(const FsParams &P)
{
    atomicExch(P.ctrl + 2, 1u);
    atomicOr(P.ctrl + 0, 1u);
}

// wait until ctrl[idx] >= target (bounded); false after an error
__device__ bool fs_wait_count(const FsParams &P, int idx, unsigned target)
{
    if (fs_ld_acquire(P.ctrl + idx) >= target) return true;
    const unsigned long long t0 = global_ns();
    while (fs_ld_acquire(P.ctrl + idx) < target) {
        if (fs_ld_acquire(P.ctrl + 2) != 0u) return false;
        if (global_ns() - t0 > P.limit_ns) {
            fs_fail(P);
            return false;
        }
        __nanosleep(128);
    }
    return true;
}

__device__ __noinline__ bool fs_mbar_wait(uint64_t *bar, unsigned parity, const FsParams &P)
{
    if (mbar_wait_bounded(bar, parity, P.limit_ns, P.ctrl + 2)) return true;
    atomicOr(P.ctrl + 0, 1u);
    return false;
}

// slice task k -> (B?, t), the fused kernel's wavefront order (lookahead D >= 1)
__device__ __forceinline__ void fs_task(int L, int D, int k, bool &b, int &t)
{
    if (k == 0) {
        b = false;
        t = L - 1;
        return;
    }
    if (k <= D) {
        b = false;
        t = k - 1;
        return;
    }
    const int kp = k - (D + 1), pairs = L - 1 - D;
    if (kp < 2 * pairs) {
        b = kp & 1;
        t = b ? (kp >> 1) : (kp >> 1) + D;
    } else {
        b = true;
        t = pairs + (kp - 2 * pairs);
    }
}

struct FsItem {
    bool b;
    int t, z, y0, j, jzm, jtm;
    long long i0;
};

__device__ __forceinline__ FsItem fs_item(const FsParams &P, int q)
{
    FsItem it;
    const int k = q / P.tps, c = q - k * P.tps;
    fs_task(P.lt, P.lookahead, k, it.b, it.t);
    const int tiles_per_plane = P.ly / P.rows;
    it.z = c / tiles_per_plane;
    it.y0 = (c - it.z * tiles_per_plane) * P.rows;
    it.j = it.t * P.tps + c;
    const int zm = it.z == 0 ? P.lz - 1 : it.z - 1, tm = it.t == 0 ? P.lt - 1 : it.t - 1;
    it.jzm = it.t * P.tps + zm * tiles_per_plane + it.y0 / P.rows;
    it.jtm = tm * P.tps + c;
    it.i0 = (long long)it.j * P.tile;
    return it;
}

__device__ __forceinline__ int fs_row(const FsParams &P, int z, int t, int y)
{
    return ((t * P.lz + z) * P.ly + y) * P.lxh;
}

// issue the copies of item `it` into the stage at `base`
// pol_a: link copies of first-hop items (read again by the second hop of the
// same slices: normal L2 priority); pol_b: those of second-hop items (last
// use: evict first)
__device__ __forceinline__ void fs_issue(const FsParams &P, const FsItem &it, char *base, uint64_t *full,
                                         uint64_t pol_a, uint64_t pol_b)
{
    const FsLayout &L = P.L;
    const int T = P.tile;
    const PairFields f = pair_fields(T, P.lxh);
    const int ly = P.ly, lz = P.lz, lt = P.lt;
    const int ym = it.y0 == 0 ? ly - 1 : it.y0 - 1;
    const int yp = it.y0 + P.rows == ly ? 0 : it.y0 + P.rows;
    const int zp = it.z + 1 == lz ? 0 : it.z + 1, zm = it.z == 0 ? lz - 1 : it.z - 1;
    const int tp = it.t + 1 == lt ? 0 : it.t + 1, tm = it.t == 0 ? lt - 1 : it.t - 1;
    const char *blk = P.blocks + (long long)it.j * f.bytes;
    const char *bzm = P.blocks + (long long)it.jzm * f.bytes;
    const char *btm = P.blocks + (long long)it.jtm * f.bytes;
    char *lk = base + L.lk;
    mbar_expect_tx(full, (unsigned)(it.b ? L.tx_b : L.tx_a));
    if (!it.b) {
        bulk_hint(lk, blk, (unsigned)(f.eY + 72 * T), full, pol_a);
        bulk_hint(lk + f.eZ, bzm + f.eZ, (unsigned)(72 * T), full, pol_a);
        bulk_hint(lk + f.eT, btm + f.eT, (unsigned)(72 * T), full, pol_a);
    } else {
        bulk_hint(lk + f.oX, blk + f.oX, (unsigned)(f.bytes - f.oX), full, pol_b);
        bulk_hint(lk + f.oZ, bzm + f.oZ, (unsigned)(72 * T), full, pol_b);
        bulk_hint(lk + f.oT, btm + f.oT, (unsigned)(72 * T), full, pol_b);
    }
    const CUtensorMap *mt = it.b ? &P.mid_tile : &P.in_tile;
    const CUtensorMap *mr = it.b ? &P.mid_row : &P.in_row;
    const int i0 = (int)it.i0;
    tma_2d(base + L.sp[0], mt, 2 * i0, 0, full);
    tma_2d(base + L.sp[1], mr, 2 * fs_row(P, it.z, it.t, ym), 0, full);
    tma_2d(base + L.sp[2], mr, 2 * fs_row(P, it.z, it.t, yp), 0, full);
    tma_2d(base + L.sp[3], mt, 2 * fs_row(P, zp, it.t, it.y0), 0, full);
    tma_2d(base + L.sp[4], mt, 2 * fs_row(P, zm, it.t, it.y0), 0, full);
    tma_2d(base + L.sp[5], mt, 2 * fs_row(P, it.z, tp, it.y0), 0, full);
    tma_2d(base + L.sp[6], mt, 2 * fs_row(P, it.z, tm, it.y0), 0, full);
}

// planar link field at byte offset `off` of the stage's link region, n sites
struct Field {
    const float4 *l4;
    const float2 *l2;
};
__device__ __forceinline__ Field field(const char *lk, int off, int n)
{
    return {reinterpret_cast<const float4 *>(lk + off), reinterpret_cast<const float2 *>(lk + off + 64 * n)};
}

template <bool Dag, int NS>
__global__ void __launch_bounds__(32 * (2 * NS * 2 + 1), 1) fused_staged_kernel(const __grid_constant__ FsParams P)
{
    extern __shared__ __align__(128) char smem[];
    const FsLayout &L = P.L;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NS * L.bytes);
    uint64_t *empty = full + NS;
    uint64_t *ready = empty + NS;
    int *slot = reinterpret_cast<int *>(ready + kFsTeams);  // item of each stage (-1: stop)
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int T = P.tile, lxh = P.lxh;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, (unsigned)P.tpt);
        }
        for (int t = 0; t < kFsTeams; ++t) mbar_init(ready + t, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 2 * NS * P.tpt) {  // producer
        if (lane != 0) return;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.in_tile)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.in_row)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.mid_tile)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.mid_row)) : "memory");
        const uint64_t pol_a = policy_evict_normal(), pol_b = policy_evict_first();
        const unsigned need = (unsigned)(P.tps * P.tpt);  // team stores of one slice
        int known[4] = {-1, -1, -1, -1};  // slices seen complete (most recent four)
        int kn = 0;
        int k = 0;
        for (;; ++k) {
            const int s = k % NS, u = k / NS;
            if (u >= 1 && !fs_mbar_wait(empty + s, (unsigned)((u - 1) & 1), P)) break;
            // items in queue order, round robin over the co-resident CTAs
            const long long qq = (long long)blockIdx.x + (long long)k * gridDim.x;
            if (qq >= P.total) break;
            const int q = (int)qq;
            const FsItem it = fs_item(P, q);
            if (it.b) {
                const int tm = it.t == 0 ? P.lt - 1 : it.t - 1, tp = it.t + 1 == P.lt ? 0 : it.t + 1;
                const int need_t[3] = {tm, it.t, tp};
                bool ok = true, waited = false;
                for (int d = 0; d < 3 && ok; ++d) {
                    const int tt = need_t[d];
                    if (tt == known[0] || tt == known[1] || tt == known[2] || tt == known[3]) continue;
                    ok = fs_wait_count(P, 3 + tt, need);
                    waited = true;
                    if (ok) known[kn++ & 3] = tt;
                }
                if (!ok) break;
                // the intermediate was written by generic stores: order them before
                // the tensor copies that read it
                if (waited) asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            slot[s] = q;
            fs_issue(P, it, smem + s * L.bytes, full + s, pol_a, pol_b);
        }
        // stop every consumer group: the next NS stages carry no item. After an
        // error a stage may still be busy; its group gives up by its own bounded
        // waits, so the stop marks are only delivered to stages found free.
        for (int n = 0; n < NS; ++n, ++k) {
            const int s = k % NS, u = k / NS;
            if (u >= 1 && !fs_mbar_wait(empty + s, (unsigned)((u - 1) & 1), P)) continue;
            slot[s] = -1;
            mbar_arrive(full + s);
        }
        return;
    }

    // consumers: group g owns stage g; team = two warps on 32 sites of a tile
    const int team = warp >> 1, q = warp & 1;
    const int g = team / P.tpt;
    const int s = (team - g * P.tpt) * 32 + lane;
    const bool active = s < T;
    const int r = s / lxh, xh = s - r * lxh;
    const int rb = r * lxh;
    constexpr int S0 = Dag ? -1 : 1;
    char *base = smem + g * L.bytes;
    const char *lk = base + L.lk;
    const PairFields f = pair_fields(T, lxh);
    const float2 *sp0 = reinterpret_cast<const float2 *>(base + L.sp[0]);
    float2 *part = reinterpret_cast<float2 *>(base + L.sp[3]);  // z/t partial sums
    for (unsigned u = 0;; ++u) {
        if (!fs_mbar_wait(full + g, u & 1u, P)) return;
        const int item = slot[g];
        if (item < 0) return;
        const FsItem it = fs_item(P, item);
        // A: output odd (forward links at odd sites, backward at even); B: the reverse
        const int fX = it.b ? f.eX : f.oX, fY = it.b ? f.eY : f.oY, fZ = it.b ? f.eZ : f.oZ,
                  fT = it.b ? f.eT : f.oT;
        const int bX = it.b ? f.oX : f.eX, bY = it.b ? f.oY : f.eY, bYh = it.b ? f.oYh : f.eYh,
                  bZ = it.b ? f.oZ : f.eZ, bT = it.b ? f.oT : f.eT;
        const int out_parity = it.b ? 0 : 1;
        cx<float> acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {0.f, 0.f};
        if (q == 0) {
            cx<float> xv[12];
            if (active) {
                if (it.b) SpF32::load(P.in, P.vh, it.i0 + s, xv);  // axpy addend, in flight meanwhile
                const int y = it.y0 + r;
                const int par = (y + it.z + it.t + out_parity) & 1;
                const int xp = par ? (xh + 1 == lxh ? 0 : xh + 1) : xh;
                const int xm = par ? xh : (xh == 0 ? lxh - 1 : xh - 1);
                Field F = field(lk, fX, T);
                staged_dir<0, true, S0>(acc, sp0, T, rb + xp, F.l4, F.l2, T, s);
                F = field(lk, bX, T);
                staged_dir<0, false, S0>(acc, sp0, T, rb + xm, F.l4, F.l2, T, rb + xm);
                F = field(lk, fY, T);
                if (r + 1 < P.rows)
                    staged_dir<1, true, S0>(acc, sp0, T, rb + lxh + xh, F.l4, F.l2, T, s);
                else
                    staged_dir<1, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[2]), lxh, xh,
                                            F.l4, F.l2, T, s);
                if (r > 0) {
                    F = field(lk, bY, T);
                    staged_dir<1, false, S0>(acc, sp0, T, rb - lxh + xh, F.l4, F.l2, T, s - lxh);
                } else {
                    F = field(lk, bYh, lxh);
                    staged_dir<1, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[1]), lxh, xh,
                                             F.l4, F.l2, lxh, xh);
                }
            }
            if (!fs_mbar_wait(ready + team, u & 1u, P)) return;
            if (active) {
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const float2 v = part[c * T + s];
                    acc[c].r += v.x;
                    acc[c].i += v.y;
                }
            }
            // the stage is consumed: hand it back before the global stores
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + g);
            if (active) {
                if (it.b) {
                    float2 *o = P.out + it.i0 + s;
#pragma unroll
                    for (int c = 0; c < 12; ++c)
                        o[c * P.vh] = make_float2(fmaf(P.a, acc[c].r, xv[c].r), fmaf(P.a, acc[c].i, xv[c].i));
                } else {
                    float2 *o = P.mid + it.i0 + s;
#pragma unroll
                    for (int c = 0; c < 12; ++c) o[c * P.vh] = make_float2(acc[c].r, acc[c].i);
                }
            }
            if (!it.b) {
                // make the intermediate visible to the tensor copies of B items
                // (async proxy, other CTAs), then count this team's store with a
                // release-ordered reduction
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __syncwarp();
                if (lane == 0 && !P.inject)
                    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(P.ctrl + 3 + it.t) : "memory");
            }
        } else {
            if (active) {
                Field F = field(lk, fZ, T);
                staged_dir<2, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[3]), T, s, F.l4, F.l2,
                                        T, s);
                F = field(lk, bZ, T);
                staged_dir<2, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[4]), T, s, F.l4, F.l2,
                                         T, s);
                F = field(lk, fT, T);
                staged_dir<3, true, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[5]), T, s, F.l4, F.l2,
                                        T, s);
                F = field(lk, bT, T);
                staged_dir<3, false, S0>(acc, reinterpret_cast<const float2 *>(base + L.sp[6]), T, s, F.l4, F.l2,
                                         T, s);
#pragma unroll
                for (int c = 0; c < 12; ++c) part[c * T + s] = make_float2(acc[c].r, acc[c].i);
            }
            // the next copies into this stage write over the partial sums
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(ready + team);
        }
    }
}

// Pair blocks of tile j: thread (j, s) writes the eight T-site fields at local
// site s, and for s < Lx/2 the two halo fields.
__global__ void pack_pair_blocks_kernel(const HopParams p, int rows, char *out)
{
    const int T = rows * p.lxh;
    const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= p.vh) return;
    const int j = (int)(gi / T), s = (int)(gi - (long long)j * T);
    const PairFields f = pair_fields(T, p.lxh);
    char *blk = out + (long long)j * f.bytes;
    auto put = [&](int off, int n, int idx, int field_index, long long site) {
        cx<double> U[3][3];
        LkF32_18::load(p.gauge + field_index * p.gauge_pb, p.vh, site, U);
        float4 *q4 = reinterpret_cast<float4 *>(blk + off) + idx;
        q4[0] = make_float4(U[0][0].r, U[0][0].i, U[0][1].r, U[0][1].i);
        q4[n] = make_float4(U[0][2].r, U[0][2].i, U[1][0].r, U[1][0].i);
        q4[2 * n] = make_float4(U[1][1].r, U[1][1].i, U[1][2].r, U[1][2].i);
        q4[3 * n] = make_float4(U[2][0].r, U[2][0].i, U[2][1].r, U[2][1].i);
        reinterpret_cast<float2 *>(blk + off + 64 * n)[idx] = make_float2(U[2][2].r, U[2][2].i);
    };
    // packed field (mu, parity) at index 2 mu + parity
    put(f.oX, T, s, 1, gi);
    put(f.oY, T, s, 3, gi);
    put(f.oZ, T, s, 5, gi);
    put(f.oT, T, s, 7, gi);
    put(f.eX, T, s, 0, gi);
    put(f.eY, T, s, 2, gi);
    put(f.eZ, T, s, 4, gi);
    put(f.eT, T, s, 6, gi);
    if (s < p.lxh) {
        const int row0 = j * rows;
        const int plane = row0 / p.ly, y0 = row0 - plane * p.ly;
        const int ym = y0 == 0 ? p.ly - 1 : y0 - 1;
        const long long h = ((long long)plane * p.ly + ym) * p.lxh + s;
        put(f.eYh, p.lxh, s, 2, h);
        put(f.oYh, p.lxh, s, 3, h);
    }
}

// One CTA per SM, launched cooperatively: the static round-robin schedule
// relies on every CTA being resident (an item may wait for items of any other
// CTA), which a cooperative launch guarantees or refuses.
template <bool Dag, int NS>
int launch_fs(const FsParams &P, int sms, cudaStream_t s)
{
    auto kern = fused_staged_kernel<Dag, NS>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(fused_staged_kernel<Dag, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kFsSmemLimit);
    });
    WEO_CUDA(attr);
    const int threads = 32 * (2 * NS * P.tpt + 1);
    const size_t smem = fs_smem(P.L, NS);
    int per_sm = 0;
    WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return set_error(WEO_ERR_CUDA, "fused staged M_eo: kernel cannot be resident");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr_list[1];
    attr_list[0].id = cudaLaunchAttributeCooperative;
    attr_list[0].val.cooperative = 1;
    cfg.attrs = attr_list;
    cfg.numAttrs = 1;
    WEO_CUDA(cudaLaunchKernelEx(&cfg, kern, P));
    return WEO_OK;
}

// tile rows of the fused staged M_eo: as the staged hop (R divides Ly, R >= 2,
// R Lx/2 <= 64, Lx/2 even), and a ring of at least two stages that fits
int fs_rows(const wilson_eo_s *h, int *stages)
{
    const int lxh = h->dims[0] / 2, ly = h->dims[1];
    *stages = 0;
    if (lxh % 2 != 0 || 2 * h->vh >= (1ll << 31)) return 0;
    for (int r = 64 / lxh; r >= 2; --r) {
        if (ly % r) continue;
        FsLayout L;
        make_fs_layout(lxh, r, L);
        const int tpt = r * lxh > 32 ? 2 : 1;
        for (int ns = kFsMaxStages; ns >= 2; --ns)
            if (fs_smem(L, ns) <= (size_t)kFsSmemLimit && ns * tpt <= kFsTeams) {
                *stages = ns;
                return r;
            }
    }
    return 0;
}

}  // namespace

bool fstaged_eligible(const wilson_eo_s *h)
{
    int ns = 0;
    return h->prec == WEO_F32 && h->fmt == WEO_LINK18 && fs_rows(h, &ns) >= 2 && tma_encoder() != nullptr;
}

// pair blocks of field g (FP32 18-real), rebuilt when g changed (allocates;
// not while `s` is being captured)
static int fs_blocks(wilson_eo_s *h, const PackedGauge &g, int rows, cudaStream_t s, const char **out)
{
    const int lxh = h->dims[0] / 2, T = rows * lxh;
    const long long ntiles = h->vh / T;
    const PairFields f = pair_fields(T, lxh);
    if (!(h->fs_valid && h->fs_src == g.buf.ptr && h->fs_gen == g.gen && h->fs_tile == T)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        WEO_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return set_error(WEO_ERR_UNSUPPORTED, "fused staged M_eo: link blocks must be built before capture");
        WEO_TRY(h->fs_links.ensure((size_t)ntiles * f.bytes));
        HopParams p = geom_params(h);
        p.gauge = static_cast<const char *>(g.buf.ptr);
        p.gauge_pb = g.pb;
        pack_pair_blocks_kernel<<<(unsigned)((h->vh + 255) / 256), 256, 0, s>>>(p, rows,
                                                                               static_cast<char *>(h->fs_links.ptr));
        WEO_CUDA(cudaGetLastError());
        h->fs_valid = true;
        h->fs_src = g.buf.ptr;
        h->fs_gen = g.gen;
        h->fs_tile = T;
    }
    *out = static_cast<const char *>(h->fs_links.ptr);
    return WEO_OK;
}

int fstaged_prepare(wilson_eo_s *h, const PackedGauge &g, cudaStream_t s)
{
    if (h->algo != 2 || !fstaged_eligible(h) || g.prec != WEO_F32 || g.fmt != WEO_LINK18) return WEO_OK;
    int ns = 0;
    const int rows = fs_rows(h, &ns);
    const char *b = nullptr;
    WEO_TRY(fused_prepare(h, s));
    return fs_blocks(h, g, rows, s, &b);
}

int meo_fstaged(wilson_eo_s *h, const PackedGauge &g, void *mid, void *out, const void *in, bool dag,
                cudaStream_t s, bool inject)
{
    int ns = 0;
    const int rows = fs_rows(h, &ns);
    if (!rows || g.prec != WEO_F32 || g.fmt != WEO_LINK18 || !tma_encoder())
        return set_error(WEO_ERR_UNSUPPORTED, "fused staged M_eo: FP32 18-real handle and a tileable lattice only");
    auto aligned = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if (!aligned(in) || !aligned(mid) || !aligned(out))
        return set_error(WEO_ERR_UNSUPPORTED, "fused staged M_eo: arrays must be 16-byte aligned");
    const char *blocks = nullptr;
    WEO_TRY(fs_blocks(h, g, rows, s, &blocks));
    WEO_TRY(fused_prepare(h, s));
    const int L = h->dims[3];
    WEO_CUDA(cudaMemsetAsync(static_cast<unsigned int *>(h->fused_ctrl.ptr) + 1, 0,
                             (size_t)(2 + L) * sizeof(unsigned int), s));
    FsParams P;
    std::memset(&P, 0, sizeof(P));
    const int lxh = h->dims[0] / 2;
    const int T = rows * lxh;
    make_fs_layout(lxh, rows, P.L);
    const long long vh = h->vh;
    const cuuint64_t sd[2] = {(cuuint64_t)(2 * vh), 12};
    const cuuint64_t ss[1] = {(cuuint64_t)(8 * vh)};
    const cuuint32_t b_tile[2] = {(cuuint32_t)(2 * T), 12}, b_row[2] = {(cuuint32_t)(2 * lxh), 12};
    if (!tma_encode(&P.in_tile, in, 2, sd, ss, b_tile) || !tma_encode(&P.in_row, in, 2, sd, ss, b_row) ||
        !tma_encode(&P.mid_tile, mid, 2, sd, ss, b_tile) || !tma_encode(&P.mid_row, mid, 2, sd, ss, b_row))
        return set_error(WEO_ERR_CUDA, "fused staged M_eo: tensor map encoding failed");
    P.blocks = blocks;
    P.lxh = lxh;
    P.ly = h->dims[1];
    P.lz = h->dims[2];
    P.lt = L;
    P.rows = rows;
    P.tile = T;
    P.tpt = T > 32 ? 2 : 1;
    P.tps = P.lz * (P.ly / rows);
    P.lookahead = h->fused_lookahead < 1 ? 1 : (h->fused_lookahead > L - 1 ? L - 1 : h->fused_lookahead);
    if (P.lookahead < 1) P.lookahead = 1;
    P.total = 2 * L * P.tps;
    P.vh = vh;
    P.a = (float)(-h->kappa * h->kappa);
    P.in = static_cast<const float2 *>(in);
    P.mid = static_cast<float2 *>(mid);
    P.out = static_cast<float2 *>(out);
    P.ctrl = static_cast<unsigned int *>(h->fused_ctrl.ptr);
    P.limit_ns = inject ? 2000000ull : 1000000000ull;
    P.inject = inject ? 1 : 0;
    int sms = 0;
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int tok = prof_begin(h, kernel_label("fused_staged", WEO_F32, WEO_LINK18, dag, true).c_str(), s);
    int st;
    if (ns == 3)
        st = dag ? launch_fs<true, 3>(P, sms, s) : launch_fs<false, 3>(P, sms, s);
    else
        st = dag ? launch_fs<true, 2>(P, sms, s) : launch_fs<false, 2>(P, sms, s);
    prof_end(h, tok, s);
    return st;
}

}  // namespace weo
