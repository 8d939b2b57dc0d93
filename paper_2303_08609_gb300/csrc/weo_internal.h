// Internal declarations shared by the translation units of libwilson_eo.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "../../include/wilson_eo.h"
#include "weo_dslash.cuh"

namespace weo {

// ------------------------------------------------------------------ errors --
int set_error(int status, const std::string &msg);
int fail_cuda(cudaError_t e, const char *what, const char *file, int line);

#define WEO_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::weo::fail_cuda(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define WEO_TRY(call)                \
    do {                             \
        int s_ = (call);             \
        if (s_ != WEO_OK) return s_; \
    } while (0)

// ----------------------------------------------------------------- formats --
// Internal operator precision next to weo_prec: float-float arithmetic with
// 18-real links (FP64-class accuracy from FP32 operations); spinors SpFF.
constexpr int kPrecFF = 4;

// Spinor storage kinds inside the library.
enum SpinorKind { SK_F64 = 0, SK_F32 = 1, SK_H16 = 2, SK_B16 = 3 };

inline long long spinor_site_bytes(int kind)
{
    return kind == SK_F64 ? 192 : kind == SK_F32 ? 96 : 52;
}
inline long long link_site_bytes(int prec, int fmt)
{
    const bool c = fmt == WEO_LINK12;
    switch (prec) {
    case WEO_F64: return c ? 96 : 144;
    case kPrecFF: return 144;
    case WEO_F32: return c ? 48 : 72;
    default: return c ? 24 : 36;
    }
}

// Device buffer that only grows.
struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    int ensure(size_t n);
    void release();
};

// A packed gauge field in one precision / link format.
struct PackedGauge {
    Buffer buf;
    int prec = -1;
    int fmt = -1;
    long long pb = 0;  // bytes of one (mu, parity) field
    bool valid = false;
    unsigned gen = 0;  // incremented by every pack
};

// Launch configuration chosen by the tuner (or defaults).
struct LaunchCfg {
    int threads = 128;
    int rhs_block = 1;   // right-hand sides per thread (register blocking)
    int lanes = 1;       // right-hand sides on neighbouring lanes sharing link loads
    int staged = 0;      // FP32 18-real, one RHS: operands staged in shared memory by TMA
    int tile_links = 0;  // several RHS: right-hand sides per pass over a tile whose links
                         // sit in shared memory (2, 4 or 8; 0 = off)
    int tile_rhs_per_thread = 1;  // ... and right-hand sides per thread sharing each link read (1, 2)
    int blocked = 0;     // one-site-per-thread hops: CTAs take 2x2x2 blocks of rows (y, z, t)
};

struct Profiler;
struct SolverState;

}  // namespace weo

struct wilson_eo_s {
    int dims[4];
    long long vh;
    double kappa;
    int prec;
    int fmt;
    int device;
    weo::PackedGauge gauge;      // in the handle's precision
    weo::PackedGauge gauge_f64;  // solver: true residual (lazy)
    weo::PackedGauge gauge_lo;   // solver: inner operator of an FP64 handle (lazy)
    weo::PackedGauge gauge_ff;   // float-float operator (lazy)
    weo::Buffer ff_in, ff_out, ff_tmp;  // float-float spinors of wilson_eo_apply_ff64
    weo::Buffer canon_gauge;     // device copy of the canonical field (kept for lazy packs)
    int canon_is_f64 = 1;
    weo::Buffer tmp;             // odd-site intermediate of M_eo
    weo::Buffer tmp2, tmp3;      // odd-site fields of the link gradient
    weo::Buffer even1;           // even-site field (force: 2 M_eo phi)
    weo::Buffer stage_in, stage_out, stage_aux;
    weo::LaunchCfg cfg[5];       // per operator precision (weo_prec, then kPrecFF)
    weo::Profiler *prof = nullptr;
    weo::SolverState *solver = nullptr;
    // M_eo algorithm for FP32 / 16-bit operators: 0 two hop launches, 1 fused,
    // 2 fused through the TMA-staged pipeline (FP32 18-real)
    int algo = 0;
    int alternate = 1;       // second hop walks the sites in reverse order
    int fused_lookahead = 4;     // t-slices the fused kernel's first hop runs ahead
    int fused_threads = 128;
    int staged_rows = 0;     // staged hop: lattice rows per tile (0: automatic)
    int staged_depth = 0;    // staged hop: shared-memory stages (0: automatic)
    weo::Buffer staged_links;   // staged hop: per-tile link blocks of both parities
    const void *staged_src = nullptr;  // ... packed from this field,
    unsigned staged_gen = 0;           // ... at this pack generation,
    int staged_tile = 0;               // ... for tiles of this many sites
    bool staged_valid = false;
    weo::Buffer fs_links;    // fused staged M_eo: pair link blocks of both parities
    const void *fs_src = nullptr;  // ... packed from this field,
    unsigned fs_gen = 0;           // ... at this pack generation,
    int fs_tile = 0;               // ... for tiles of this many sites
    bool fs_valid = false;
    weo::Buffer fused_ctrl;  // sticky error, ticket, completion counters
    weo::Buffer halo;        // face buffers of the domain-decomposed hop
};

namespace weo {

// geometry of a handle, without field pointers
HopParams geom_params(const wilson_eo_s *h);

// Launch the hopping kernel. io selects the storage combination:
//   IO_SAME  : in, out and x all in the precision `prec` (F64 or F32)
//   IO_TO16  : in FP32, out 16-bit (prec = WEO_F16 / WEO_BF16), hop mode only
//   IO_FROM16: in 16-bit, out FP32, x FP32
enum IoKind { IO_SAME = 0, IO_TO16 = 1, IO_FROM16 = 2 };
int launch_hop(int prec, int fmt, int io, bool dag, bool axpy, const HopParams &p,
               const LaunchCfg &cfg, cudaStream_t s);
int launch_hop_f64(int fmt, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s);
int launch_hop_ff(bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg, cudaStream_t s);
int launch_hop_f32(int fmt, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s);
int launch_hop_h16(int fmt, int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s);
int launch_hop_b16(int fmt, int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s);

// Per-kernel event timing (prof.cu). prof_begin returns a token (-1 when off).
int prof_begin(wilson_eo_s *h, const char *label, cudaStream_t s);
void prof_end(wilson_eo_s *h, int token, cudaStream_t s);
void prof_destroy(wilson_eo_s *h);
std::string kernel_label(const char *kind, int prec, int fmt, bool dag, bool axpy);

// hop_staged.cu: the hopping kernel fed by TMA boxes through a ring of
// shared-memory stages (FP32 spinors, 18-real FP32 links, one right-hand side)
bool staged_eligible(const wilson_eo_s *h);
void staged_shape(const wilson_eo_s *h, int *rows, int *depth);
bool staged_arrays_ok(const HopParams &p, bool axpy);
// link blocks of the staged hop for field g (no-op unless staging is on)
int staged_prepare(wilson_eo_s *h, const PackedGauge &g, cudaStream_t s);
// the link blocks for p.gauge are current, or were built now (never while
// the stream is being captured)
bool staged_ready(wilson_eo_s *h, const HopParams &p, cudaStream_t s);
int launch_hop_staged(wilson_eo_s *h, bool dag, bool axpy, const HopParams &p, cudaStream_t s,
                      bool inject = false);

// tensor maps (hop_staged.cu): cuTensorMapEncodeTiled through the runtime's
// driver entry point (null if unavailable); FP32 tensor of rank 2 or 3,
// dims[0] contiguous, strides in bytes of dims 1..
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn tma_encoder();
bool tma_encode(CUtensorMap *m, const void *ptr, int rank, const cuuint64_t *dims,
                const cuuint64_t *strides, const cuuint32_t *box);

// launch_hop for a handle, with its launch configuration and profiling
int handle_hop(wilson_eo_s *h, int prec, int fmt, int io, bool dag, bool axpy, const HopParams &p,
               cudaStream_t s);

// M_eo / M_eo^dag with a given packed gauge field (its precision decides the
// spinor formats) and odd-site buffer (api.cu)
int meo_with(wilson_eo_s *h, const PackedGauge &g, Buffer &tmp, void *out, const void *in,
             int nrhs, bool dag, cudaStream_t s);
// fused.cu: both hops in one persistent launch over a wavefront of t-slices
// (FP32 spinors, odd intermediate in `mid`); error word of its bounded waits
int meo_fused(wilson_eo_s *h, const PackedGauge &g, void *mid, void *out, const void *in, bool dag,
              cudaStream_t s, bool inject_timeout = false);
int fused_take_error(wilson_eo_s *h, cudaStream_t s, unsigned int *err);
// fused_staged.cu: both hops in one persistent launch fed by TMA, pair link
// blocks shared by the two hops (FP32 18-real, one right-hand side)
bool fstaged_eligible(const wilson_eo_s *h);
int fstaged_prepare(wilson_eo_s *h, const PackedGauge &g, cudaStream_t s);
int meo_fstaged(wilson_eo_s *h, const PackedGauge &g, void *mid, void *out, const void *in, bool dag,
                cudaStream_t s, bool inject = false);
int fused_prepare(wilson_eo_s *h, cudaStream_t s);
// halo.cu: hop with the lattice split along t and every crossing hop exchanged
int hop_split_device(wilson_eo_s *h, int ranks, int out_parity, bool dag, void *out,
                     const void *in, cudaStream_t s);
// M_eo / M_eo^dag on device arrays in the handle's external format (api.cu)
int meo_device(wilson_eo_s *h, void *out, const void *in, int nrhs, bool dag, cudaStream_t s);
// link gradient (force = 0) or force TA(G U^dag) (force = 1), force.cu
int link_grad_device(wilson_eo_s *h, void *out, const void *g, const void *phi, int force,
                     cudaStream_t s, const void *t_known = nullptr);
int scale_spinor(wilson_eo_s *h, void *v, int nrhs, double c, cudaStream_t s);

// solver.cu
int solve_device(wilson_eo_s *h, void *x_e, const void *b_e, bool x_host, bool b_host, int nrhs,
                 double tol, int maxiter, int mixed, int *iters_out, double *relres_out,
                 cudaStream_t user);
int solver_configure(wilson_eo_s *h, double delta, int chunk, int use_graphs);
int solver_stats(wilson_eo_s *h, int *iterations, int *reliable_updates, int *hi_applies,
                 int *ff_applies, double *seconds);
int solver_residual_mode(wilson_eo_s *h, int mode);
int solver_restart_mode(wilson_eo_s *h, int restart);
void solver_destroy(wilson_eo_s *h);
int prepare_source_device(wilson_eo_s *h, void *rhs_e, const void *eta_e, const void *eta_o,
                          cudaStream_t s);
int reconstruct_device(wilson_eo_s *h, void *xi_o, const void *eta_o, const void *xi_e,
                       cudaStream_t s);
int solve_full_device(wilson_eo_s *h, void *xi_e, void *xi_o, const void *eta_e,
                      const void *eta_o, const bool host[4], double tol, int maxiter, int mixed,
                      int *iters_out, double *relres_out, cudaStream_t user);

// Pack a canonical gauge field (device memory) into `g` (allocates).
// ff.cu: complex128 <-> float-float spinors (nrhs x V/2 sites), float-float gauge
int ff_from_f64(void *dst, const void *src, long long vh, int nrhs, cudaStream_t s);
int ff_to_f64(void *dst, const void *src, long long vh, int nrhs, cudaStream_t s);
int ff_gauge(wilson_eo_s *h, const PackedGauge **g, cudaStream_t s);
int pack_gauge(wilson_eo_s *h, PackedGauge &g, int prec, int fmt, const void *canon, int is_f64,
               cudaStream_t s);

}  // namespace weo
