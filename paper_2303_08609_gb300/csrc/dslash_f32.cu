// FP32 instances of the hopping kernel (planar complex64 spinors, FP32 links),
// with 1, 2 or 4 right-hand sides per thread sharing each link load.
#include "weo_launch.cuh"

namespace weo {

template <class Lk>
static int f32_rhs(bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg, cudaStream_t s)
{
    int r = cfg.rhs_block;
    while (r > 1 && r > p.nrhs) r /= 2;  // never more right-hand sides per thread than exist
    switch (r) {
    case 4: return launch_da<SpF32, SpF32, SpF32, Lk, 4>(dag, axpy, p, cfg, s);
    case 2: return launch_da<SpF32, SpF32, SpF32, Lk, 2>(dag, axpy, p, cfg, s);
    default: return launch_da<SpF32, SpF32, SpF32, Lk, 1>(dag, axpy, p, cfg, s);
    }
}

int launch_hop_f32(int fmt, bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg,
                   cudaStream_t s)
{
    if (fmt == WEO_LINK12) return f32_rhs<LkF32_12>(dag, axpy, p, cfg, s);
    return f32_rhs<LkF32_18>(dag, axpy, p, cfg, s);
}

}  // namespace weo
