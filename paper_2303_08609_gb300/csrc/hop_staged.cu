// TMA-staged hopping kernel: handle-side management (tile shape, link blocks,
// readiness inside CUDA-graph capture) and the FP32 instances. The kernel
// itself is in hop_staged.cuh; the 16-bit instances are in hop_staged_h16.cu
// and hop_staged_b16.cu.
#include "hop_staged.cuh"

namespace weo {

namespace staged {

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn encoder()
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

// FP32 planar spinor: 12 planes of 2 vh floats; boxes of box_sites sites x 12 planes
bool encode_spinor_map(CUtensorMap *m, const void *ptr, long long vh, int box_sites)
{
    EncodeFn fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * vh), 12};
    const cuuint64_t strides[1] = {(cuuint64_t)(8 * vh)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * box_sites), 12};
    const cuuint32_t one[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

using LkF32_18S = LkF32_18T<LdPlain>;
using LkF32_12S = LkF32_12T<LdPlain>;

// rows of R per tile: R divides Ly, R >= 2, R * Lx/2 <= 64; the largest such
// R, or the requested one when it qualifies (0 if none does)
static int tile_rows(int lxh, int ly, int want)
{
    if (lxh % 2 != 0) return 0;  // rows must start on 16-byte boundaries
    auto ok = [&](int r) { return r >= 2 && ly % r == 0 && r * lxh <= kMaxTile; };
    if (want) return ok(want) ? want : 0;
    for (int r = kMaxTile / lxh; r >= 2; --r)
        if (ok(r)) return r;
    return 0;
}

// the packed field the hop parameters point to
static const PackedGauge *field_of(const wilson_eo_s *h, const char *gauge)
{
    if (gauge == h->gauge.buf.ptr) return &h->gauge;
    if (gauge == h->gauge_lo.buf.ptr) return &h->gauge_lo;
    return nullptr;
}

// ring depth cap when none is requested (measured best at tiles of 64 sites)
static int depth_cap(int prec) { return prec == WEO_F32 ? 3 : 4; }

static bool format_ok(const wilson_eo_s *h, int prec)
{
    // 16-bit row blocks (52 Lx/2 bytes) must start on 16-byte boundaries
    return prec == WEO_F32 || ((prec == WEO_F16 || prec == WEO_BF16) && (h->dims[0] / 2) % 4 == 0);
}

}  // namespace staged

using namespace staged;

void staged_shape(const wilson_eo_s *h, int *rows_out, int *depth_out)
{
    const int lxh = h->dims[0] / 2;
    const int prec = h->prec == WEO_F64 ? WEO_F32 : h->prec;
    int rows = tile_rows(lxh, h->dims[1], h->staged_rows), depth = 0;
    // TMA coordinates are 32-bit: 2 floats per site in the spinor boxes
    if (rows >= 2 && format_ok(h, prec) && 2 * h->vh < (1ll << 31)) {
        StageLayout L;
        make_layout(lxh, rows, 96, (int)link_site_bytes(prec, h->fmt), true, L);
        depth = pick_depth(L, rows * lxh, h->staged_depth, depth_cap(prec));
    }
    if (!depth) rows = 0;
    *rows_out = rows;
    *depth_out = depth;
}

bool staged_eligible(const wilson_eo_s *h)
{
    int rows, depth;
    staged_shape(h, &rows, &depth);
    return depth > 0 && encoder() != nullptr;
}

bool staged_arrays_ok(const HopParams &p, bool axpy)
{
    auto aligned = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    return aligned(p.in) && aligned(p.out) && (!axpy || aligned(p.x));
}

int staged_prepare(wilson_eo_s *h, const PackedGauge &g, cudaStream_t s)
{
    if (g.prec == WEO_F64 || g.prec == kPrecFF || !h->cfg[g.prec].staged) return WEO_OK;
    int rows, depth;
    staged_shape(h, &rows, &depth);
    if (!depth) return WEO_OK;
    const int T = rows * (h->dims[0] / 2);
    if (h->staged_valid && h->staged_src == g.buf.ptr && h->staged_gen == g.gen && h->staged_tile == T)
        return WEO_OK;
    h->staged_valid = false;
    WEO_TRY(h->staged_links.ensure((size_t)2 * 8 * link_site_bytes(g.prec, g.fmt) * h->vh));
    HopParams p = geom_params(h);
    p.gauge = static_cast<const char *>(g.buf.ptr);
    p.gauge_pb = g.pb;
    char *out = static_cast<char *>(h->staged_links.ptr);
    const bool c12 = g.fmt == WEO_LINK12;
    switch (g.prec) {
    case WEO_F32:
        WEO_TRY((c12 ? pack_link_blocks<LkF32_12, LkF32_12S>(p, T, out, s)
                     : pack_link_blocks<LkF32_18, LkF32_18S>(p, T, out, s)));
        break;
    case WEO_F16: WEO_TRY(staged_pack_h16(p, c12, T, out, s)); break;
    case WEO_BF16: WEO_TRY(staged_pack_b16(p, c12, T, out, s)); break;
    default: return WEO_OK;
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
    const PackedGauge *g = field_of(h, gauge);
    if (!g || !h->staged_valid || h->staged_src != g->buf.ptr || h->staged_gen != g->gen ||
        h->staged_tile != T)
        return nullptr;
    return static_cast<const char *>(h->staged_links.ptr);
}

bool staged_ready(wilson_eo_s *h, const HopParams &p, cudaStream_t s)
{
    const PackedGauge *g = field_of(h, p.gauge);
    if (!g || g->prec == WEO_F64 || g->prec == kPrecFF || !h->cfg[g->prec].staged ||
        !format_ok(h, g->prec) || p.nrhs != 1)
        return false;
    int rows, depth;
    staged_shape(h, &rows, &depth);
    if (!depth) return false;
    const int T = rows * p.lxh;
    if (staged_blocks(h, p.gauge, T)) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    return staged_prepare(h, *g, s) == WEO_OK && staged_blocks(h, p.gauge, T) != nullptr;
}

int launch_hop_staged(wilson_eo_s *h, int io, bool dag, bool axpy, const HopParams &p,
                      cudaStream_t s, bool inject)
{
    int rows, depth;
    staged_shape(h, &rows, &depth);
    const PackedGauge *g = field_of(h, p.gauge);
    const char *blocks = depth && g ? staged_blocks(h, p.gauge, rows * p.lxh) : nullptr;
    if (!blocks || !staged_arrays_ok(p, axpy) || !h->fused_ctrl.ptr)
        return set_error(WEO_ERR_UNSUPPORTED, "staged hop: lattice, link blocks or array alignment not ready");
    const int want = h->staged_depth, cap = depth_cap(g->prec);
    const bool c12 = g->fmt == WEO_LINK12;
    switch (g->prec) {
    case WEO_F32:
        if (io != IO_SAME) break;
        if (c12)
            return axpy ? launch_staged<InF32, OutF32, LkF32_12S, true, 2, 3>(h, dag, p, blocks, rows, want,
                                                                             cap, s, inject)
                        : launch_staged<InF32, OutF32, LkF32_12S, false, 2, 3>(h, dag, p, blocks, rows, want,
                                                                              cap, s, inject);
        return axpy ? launch_staged<InF32, OutF32, LkF32_18S, true, 2, 3, 4, 5>(h, dag, p, blocks, rows,
                                                                               want, cap, s, inject)
                    : launch_staged<InF32, OutF32, LkF32_18S, false, 2, 3, 4, 5>(h, dag, p, blocks, rows,
                                                                                want, cap, s, inject);
    case WEO_F16:
        if (io == IO_SAME) break;
        return staged_launch_h16(h, io, c12, dag, p, blocks, rows, want, cap, s, inject);
    case WEO_BF16:
        if (io == IO_SAME) break;
        return staged_launch_b16(h, io, c12, dag, p, blocks, rows, want, cap, s, inject);
    default: break;
    }
    return set_error(WEO_ERR_UNSUPPORTED, "staged hop: precision / storage combination not provided");
}

}  // namespace weo
