// Mixed-lattice batch: M_eo (or M_eo^dag) on several lattices -- each with its
// own extents, kappa, links and number of right-hand sides -- in ONE persistent
// cooperative launch. The grid (a whole number of CTAs per SM, all resident)
// walks the tiles of every lattice's first hop, synchronises once across the
// grid, then walks the tiles of every second hop (with the axpy of Eq. 4). A
// tile is CTA-sized in sites and covers R right-hand sides, which share each
// link load; the tiles of one site block follow each other, so the other
// right-hand-side blocks find its links in L2. FP32 batches with several
// right-hand sides use tiles of 64 sites whose links are copied into shared
// memory once for all the lattice's right-hand sides. Lattices need not fill the GPU on their own: small and large
// lattices share one launch.
#include <cooperative_groups.h>

#include <vector>

#include "weo_internal.h"

namespace cg = cooperative_groups;

namespace weo {

constexpr int kMaxBatch = 24;
constexpr int kBatchThreads = 128;

struct BatchArgs {
    int n;
    long long tile_begin[kMaxBatch + 1];  // prefix sums of tiles per lattice
    long long lt_begin[kMaxBatch + 1];    // prefix sums of 64-site link tiles per lattice
    int site_tiles[kMaxBatch];            // CTA-sized site blocks per right-hand-side block
    HopParams first[kMaxBatch];           // H_oe onto odd sites
    HopParams second[kMaxBatch];          // in - kappa^2 H_eo tmp onto even sites
};

__device__ __forceinline__ int find_lattice(const BatchArgs &a, long long tile)
{
    int k = 0;
    while (k + 1 < a.n && tile >= a.tile_begin[k + 1]) ++k;
    return k;
}

template <class Sp, class Lk, bool Dag, int R>
__global__ void __launch_bounds__(kBatchThreads) batch_meo_kernel(const __grid_constant__ BatchArgs a)
{
    const long long total = a.tile_begin[a.n];
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int k = find_lattice(a, tile);
        const long long local = tile - a.tile_begin[k];
        // right-hand-side block fastest: the tiles sharing links run side by side
        const int nrb = (a.first[k].nrhs + R - 1) / R;
        const int rb = (int)(local % nrb);
        const long long site = (local / nrb) * kBatchThreads + threadIdx.x;
        if (site < a.first[k].vh) hop_site<Sp, Sp, Sp, Lk, Dag, false, R>(a.first[k], (int)site, rb * R);
    }
    cg::this_grid().sync();
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int k = find_lattice(a, tile);
        const long long local = tile - a.tile_begin[k];
        const int nrb = (a.second[k].nrhs + R - 1) / R;
        const int rb = (int)(local % nrb);
        const long long site = (local / nrb) * kBatchThreads + threadIdx.x;
        if (site < a.second[k].vh) hop_site<Sp, Sp, Sp, Lk, Dag, true, R>(a.second[k], (int)site, rb * R);
    }
}

// Several right-hand sides (FP32): the same cooperative walk over tiles of
// 64 sites whose eight links per site are first copied into shared memory,
// then used by all the lattice's right-hand sides, four at a time (one per
// thread) -- the tile-shared-link hop of the single-lattice path.
constexpr int kLinkTile = 64, kLinkGroups = 4;

__device__ __forceinline__ int find_lattice_lt(const BatchArgs &a, long long tile)
{
    int k = 0;
    while (k + 1 < a.n && tile >= a.lt_begin[k + 1]) ++k;
    return k;
}

template <class Lk, bool Dag, bool Axpy>
__device__ __forceinline__ void batch_link_tile(const HopParams &p, int tile, float2 *lk_sm)
{
    constexpr int T = kLinkTile;
    const int i0 = tile * T;
    const int in_par = p.out_parity ^ 1;
    for (int e = threadIdx.x; e < 8 * T; e += blockDim.x) {
        const int d = e / T, s = e - d * T;
        const int i = i0 + s;
        if (i >= p.vh) continue;
        int idx = i;
        if (d & 1) {
            int nb[8];
            site_neighbours(p, i, nb);
            idx = nb[d];
        }
        cx<float> U[3][3];
        Lk::load(p.gauge + (2 * (d >> 1) + ((d & 1) ? in_par : p.out_parity)) * p.gauge_pb, p.vh, idx, U);
#pragma unroll
        for (int k = 0; k < 9; ++k) lk_sm[(d * 9 + k) * T + s] = make_float2(U[k / 3][k % 3].r, U[k / 3][k % 3].i);
    }
    __syncthreads();
    const int s = (int)threadIdx.x % T, rl = (int)threadIdx.x / T;
    const int i = i0 + s;
    if (i < p.vh) {
        constexpr int S0 = Dag ? -1 : 1;
        const float2 *lk = lk_sm + s;
        for (int r = rl; r < p.nrhs; r += kLinkGroups) {
            int nb[8];
            site_neighbours(p, i, nb);
            cx<float> acc[1][12];
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[0][k] = {0.f, 0.f};
            hop_dir_shared<SpF32, 0, true, S0, 1>(acc, p, nb[0], lk + 0 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 0, false, S0, 1>(acc, p, nb[1], lk + 1 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 1, true, S0, 1>(acc, p, nb[2], lk + 2 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 1, false, S0, 1>(acc, p, nb[3], lk + 3 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 2, true, S0, 1>(acc, p, nb[4], lk + 4 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 2, false, S0, 1>(acc, p, nb[5], lk + 5 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 3, true, S0, 1>(acc, p, nb[6], lk + 6 * 9 * T, T, r, kLinkGroups);
            hop_dir_shared<SpF32, 3, false, S0, 1>(acc, p, nb[7], lk + 7 * 9 * T, T, r, kLinkGroups);
            if (Axpy) {
                cx<float> xv[12];
                SpF32::load(static_cast<const char *>(p.x) + r * p.x_stride, p.vh, i, xv);
                const float aa = float(p.a);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    acc[0][k].r = fmaf(aa, acc[0][k].r, xv[k].r);
                    acc[0][k].i = fmaf(aa, acc[0][k].i, xv[k].i);
                }
            }
            SpF32::store(static_cast<char *>(p.out) + r * p.out_stride, p.vh, i, acc[0]);
        }
    }
    __syncthreads();  // the next tile overwrites the links
}

template <class Lk, bool Dag>
__global__ void __launch_bounds__(kLinkTile * kLinkGroups, 3) batch_meo_tiles_kernel(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(16) float2 lk_sm[];
    const long long total = a.lt_begin[a.n];
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int k = find_lattice_lt(a, tile);
        batch_link_tile<Lk, Dag, false>(a.first[k], (int)(tile - a.lt_begin[k]), lk_sm);
    }
    cg::this_grid().sync();
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int k = find_lattice_lt(a, tile);
        batch_link_tile<Lk, Dag, true>(a.second[k], (int)(tile - a.lt_begin[k]), lk_sm);
    }
}

template <class Lk, bool Dag>
static int launch_batch_tiles(const BatchArgs &a, cudaStream_t s)
{
    auto kern = batch_meo_tiles_kernel<Lk, Dag>;
    const int threads = kLinkTile * kLinkGroups;
    const size_t smem = (size_t)576 * kLinkTile;
    int dev = 0, sms = 0, per_sm = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return set_error(WEO_ERR_CUDA, "batch kernel cannot be resident");
    long long grid = (long long)sms * per_sm;
    if (grid > a.lt_begin[a.n]) grid = a.lt_begin[a.n];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    WEO_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return WEO_OK;
}

template <class Sp, class Lk, bool Dag, int R>
static int launch_batch(const BatchArgs &a, cudaStream_t s)
{
    auto kern = batch_meo_kernel<Sp, Lk, Dag, R>;
    int dev = 0, sms = 0, per_sm = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    WEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, 0));
    if (per_sm < 1) return set_error(WEO_ERR_CUDA, "batch kernel cannot be resident");
    long long grid = (long long)sms * per_sm;
    if (grid > a.tile_begin[a.n]) grid = a.tile_begin[a.n];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    WEO_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    return WEO_OK;
}

template <class Sp, class Lk>
static int launch_batch_dag(const BatchArgs &a, bool dag, int R, cudaStream_t s)
{
    if (R == 2) return dag ? launch_batch<Sp, Lk, true, 2>(a, s) : launch_batch<Sp, Lk, false, 2>(a, s);
    return dag ? launch_batch<Sp, Lk, true, 1>(a, s) : launch_batch<Sp, Lk, false, 1>(a, s);
}

static int apply_batch_impl(int n, const wilson_eo_t *hs, void *const *outs, const void *const *ins,
                            const int *nrhs, int dag, void *stream)
{
    if (n < 1 || n > kMaxBatch) return set_error(WEO_ERR_ARG, "batch size must be in 1..24");
    if (!hs || !outs || !ins) return set_error(WEO_ERR_ARG, "NULL array of handles or fields");
    const int prec = hs[0] ? hs[0]->prec : -1, fmt = hs[0] ? hs[0]->fmt : -1;
    int dev = 0;
    WEO_CUDA(cudaGetDevice(&dev));
    int max_rhs = 1;
    for (int k = 0; k < n; ++k) {
        if (!hs[k] || !outs[k] || !ins[k]) return set_error(WEO_ERR_ARG, "NULL handle or field in batch");
        if (nrhs && (nrhs[k] < 1 || nrhs[k] > 1024)) return set_error(WEO_ERR_ARG, "nrhs per lattice must be in 1..1024");
        if (hs[k]->prec != prec || hs[k]->fmt != fmt)
            return set_error(WEO_ERR_UNSUPPORTED, "a batch needs one precision and link format");
        if (hs[k]->device != dev) return set_error(WEO_ERR_ARG, "batch handles must live on the current device");
        if (outs[k] == ins[k]) return set_error(WEO_ERR_ARG, "out must not alias in");
        for (int j = 0; j < k; ++j)
            if (hs[j] == hs[k]) return set_error(WEO_ERR_ARG, "a handle appears twice in the batch");
        if (nrhs && nrhs[k] > max_rhs) max_rhs = nrhs[k];
    }
    if (prec != WEO_F32 && prec != WEO_F64)
        return set_error(WEO_ERR_UNSUPPORTED, "batches are provided for FP64 and FP32 handles");
    // FP32 lattices with several right-hand sides share each link load over two
    const int R = (prec == WEO_F32 && max_rhs >= 2) ? 2 : 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.tile_begin[0] = 0;
    for (int k = 0; k < n; ++k) {
        wilson_eo_s *h = hs[k];
        const int nr = nrhs ? nrhs[k] : 1;
        const long long ext = h->vh * (prec == WEO_F64 ? 192 : 96);
        WEO_TRY(h->tmp.ensure((size_t)ext * nr));
        HopParams p = geom_params(h);
        p.nrhs = nr;
        p.gauge = static_cast<const char *>(h->gauge.buf.ptr);
        p.gauge_pb = h->gauge.pb;
        p.in_stride = p.out_stride = p.x_stride = ext;
        p.out_parity = 1;
        p.in = ins[k];
        p.out = h->tmp.ptr;
        a.first[k] = p;
        p.out_parity = 0;
        p.in = h->tmp.ptr;
        p.out = outs[k];
        p.x = ins[k];
        p.a = -h->kappa * h->kappa;
        a.second[k] = p;
        a.site_tiles[k] = (int)((h->vh + kBatchThreads - 1) / kBatchThreads);
        a.tile_begin[k + 1] = a.tile_begin[k] + (long long)a.site_tiles[k] * ((nr + R - 1) / R);
        a.lt_begin[k + 1] = a.lt_begin[k] + (h->vh + kLinkTile - 1) / kLinkTile;
    }
    const bool c = fmt == WEO_LINK12;
    int tok = prof_begin(hs[0], "batch_meo", s);
    int st;
    if (prec == WEO_F64)
        st = c ? launch_batch_dag<SpF64, LkF64_12>(a, dag != 0, 1, s) : launch_batch_dag<SpF64, LkF64_18>(a, dag != 0, 1, s);
    else if (max_rhs >= 2)  // tiles with their links in shared memory for all right-hand sides
        st = c ? (dag ? launch_batch_tiles<LkF32_12, true>(a, s) : launch_batch_tiles<LkF32_12, false>(a, s))
               : (dag ? launch_batch_tiles<LkF32_18, true>(a, s) : launch_batch_tiles<LkF32_18, false>(a, s));
    else
        st = c ? launch_batch_dag<SpF32, LkF32_12>(a, dag != 0, R, s) : launch_batch_dag<SpF32, LkF32_18>(a, dag != 0, R, s);
    prof_end(hs[0], tok, s);
    return st;
}

}  // namespace weo

using namespace weo;

extern "C" int wilson_eo_apply_batch(int n, const wilson_eo_t *hs, void *const *outs,
                                     const void *const *ins, int dag, void *stream)
{
    try {
        return apply_batch_impl(n, hs, outs, ins, nullptr, dag, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply_batch");
    }
}

extern "C" int wilson_eo_apply_batch_rhs(int n, const wilson_eo_t *hs, void *const *outs,
                                         const void *const *ins, const int *nrhs, int dag,
                                         void *stream)
{
    try {
        if (!nrhs) return set_error(WEO_ERR_ARG, "nrhs is NULL");
        return apply_batch_impl(n, hs, outs, ins, nrhs, dag, stream);
    } catch (...) {
        return set_error(WEO_ERR_OOM, "host exception in wilson_eo_apply_batch_rhs");
    }
}
