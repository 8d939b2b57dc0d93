// 16-bit instances of the hopping kernel: links in FP16 or BF16, the odd-site
// intermediate in 16-bit with a per-site FP32 norm, FP32 arithmetic. The first
// hop reads FP32 spinors and writes 16-bit; the second reads 16-bit and writes
// FP32 with the axpy of Eq. 4.
#include "weo_launch.cuh"

namespace weo {

template <class Sp16T, class Lk>
static int pass(int io, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                cudaStream_t s)
{
    if (io == IO_TO16) {
        if (axpy) return set_error(WEO_ERR_UNSUPPORTED, "16-bit output pass has no axpy form");
        return dag ? launch_instance<SpF32, Sp16T, SpF32, Lk, true, false, 1>(p, cfg, s)
                   : launch_instance<SpF32, Sp16T, SpF32, Lk, false, false, 1>(p, cfg, s);
    }
    if (!axpy) return set_error(WEO_ERR_UNSUPPORTED, "16-bit input pass needs the axpy form");
    return dag ? launch_instance<Sp16T, SpF32, SpF32, Lk, true, true, 1>(p, cfg, s)
               : launch_instance<Sp16T, SpF32, SpF32, Lk, false, true, 1>(p, cfg, s);
}

int launch_hop_16(int prec, int fmt, int io, bool dag, bool axpy, const HopParams &p,
                  const LaunchCfg &cfg, cudaStream_t s)
{
    if (prec == WEO_F16)
        return fmt == WEO_LINK12 ? pass<SpH16, LkH16_12>(io, dag, axpy, p, cfg, s)
                                 : pass<SpH16, LkH16_18>(io, dag, axpy, p, cfg, s);
    return fmt == WEO_LINK12 ? pass<SpB16, LkB16_12>(io, dag, axpy, p, cfg, s)
                             : pass<SpB16, LkB16_18>(io, dag, axpy, p, cfg, s);
}

}  // namespace weo
