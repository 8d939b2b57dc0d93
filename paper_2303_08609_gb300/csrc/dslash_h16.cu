// FP16 instances of the hopping kernel: links in FP16, the odd-site
// intermediate in FP16 with a per-site FP32 norm, FP32 arithmetic. The
// first hop reads FP32 spinors and writes 16-bit; the second reads 16-bit and
// writes FP32 with the axpy of Eq. 4. 1, 2 or 4 right-hand sides per thread
// share each link load.
#include "weo_launch.cuh"

namespace weo {

template <class Sp16T, class Lk, int R>
static int pass_r(int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                  cudaStream_t s)
{
    if (io == IO_TO16) {
        if (axpy) return set_error(WEO_ERR_UNSUPPORTED, "16-bit output pass has no axpy form");
        return dag ? launch_instance<SpF32, Sp16T, SpF32, Lk, true, false, R>(p, cfg, s)
                   : launch_instance<SpF32, Sp16T, SpF32, Lk, false, false, R>(p, cfg, s);
    }
    if (!axpy) return set_error(WEO_ERR_UNSUPPORTED, "16-bit input pass needs the axpy form");
    return dag ? launch_instance<Sp16T, SpF32, SpF32, Lk, true, true, R>(p, cfg, s)
               : launch_instance<Sp16T, SpF32, SpF32, Lk, false, true, R>(p, cfg, s);
}

template <class Sp16T, class Lk>
static int pass(int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                cudaStream_t s)
{
    int r = cfg.rhs_block;
    while (r > 1 && r > p.nrhs) r /= 2;
    switch (r) {
    case 4: return pass_r<Sp16T, Lk, 4>(io, dag, axpy, p, cfg, s);
    case 2: return pass_r<Sp16T, Lk, 2>(io, dag, axpy, p, cfg, s);
    default: return pass_r<Sp16T, Lk, 1>(io, dag, axpy, p, cfg, s);
    }
}

int launch_hop_h16(int fmt, int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s)
{
    return fmt == WEO_LINK12 ? pass<SpH16, LkH16_12>(io, dag, axpy, p, cfg, s)
                             : pass<SpH16, LkH16_18>(io, dag, axpy, p, cfg, s);
}

}  // namespace weo
