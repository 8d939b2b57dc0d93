// FP64 instances of the hopping kernel (planar complex128 spinors, FP64 links).
#include "weo_launch.cuh"

namespace weo {

int launch_hop_f64(int fmt, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s)
{
    if (fmt == WEO_LINK12) return launch_da<SpF64, SpF64, SpF64, LkF64_12, 1>(dag, axpy, p, cfg, s);
    return launch_da<SpF64, SpF64, SpF64, LkF64_18, 1>(dag, axpy, p, cfg, s);
}

}  // namespace weo
