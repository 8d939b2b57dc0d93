// Float-float instances of the hopping kernel: the same stencil code with the
// arithmetic type ff (about 48 significant bits from FP32 operations), spinors
// in SpFF and links in LkFF18. FP64-class accuracy without the FP64 pipe.
//
// The kernel is bound by the latency of its float-float dependency chains at
// the occupancy its registers allow: three CTAs of 128 threads per SM (170
// registers, no spills) measured 1.55x the native FP64 kernel at 32^3 x 64,
// the uncapped build (one CTA of 256) 1.1x, and tighter caps spill and lose.
#include "weo_launch.cuh"

namespace weo {

template <bool Dag, bool Axpy>
__global__ void __launch_bounds__(128, 3) hop_kernel_ff(const HopParams p)
{
    const int b = p.reverse ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
    const int i = b * blockDim.x + threadIdx.x;
    if (i >= p.vh) return;
    hop_site<SpFF, SpFF, SpFF, LkFF18, Dag, Axpy, 1>(p, i, blockIdx.y);
}

template <bool Dag, bool Axpy>
static int launch_ff(const HopParams &p, cudaStream_t s)
{
    dim3 grid((unsigned)((p.vh + 127) / 128), (unsigned)p.nrhs);
    hop_kernel_ff<Dag, Axpy><<<grid, 128, 0, s>>>(p);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

int launch_hop_ff(bool dag, bool axpy, const HopParams &p, const LaunchCfg &, cudaStream_t s)
{
    if (dag) return axpy ? launch_ff<true, true>(p, s) : launch_ff<true, false>(p, s);
    return axpy ? launch_ff<false, true>(p, s) : launch_ff<false, false>(p, s);
}

}  // namespace weo
