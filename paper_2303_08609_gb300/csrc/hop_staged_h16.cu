// TMA-staged hops of FP16-storage operators (kernel in hop_staged.cuh): the first
// hop writes the 16-bit intermediate in row blocks, the second reads them.
#include "hop_staged.cuh"

namespace weo {

int staged_launch_h16(wilson_eo_s *h, int io, bool c12, bool dag, const HopParams &p,
                      const char *blocks, int rows, int want, int cap, cudaStream_t s, bool inject)
{
    return staged::launch_16<H16Traits>(h, io, c12, dag, p, blocks, rows, want, cap, s, inject);
}

int staged_pack_h16(const HopParams &p, bool c12, int T, char *out, cudaStream_t s)
{
    return staged::pack_16<H16Traits>(p, c12, T, out, s);
}

}  // namespace weo
