// TMA-staged hops of BF16-storage operators (kernel in hop_staged.cuh): the first
// hop writes the 16-bit intermediate in row blocks, the second reads them.
#include "hop_staged.cuh"

namespace weo {

int staged_launch_b16(wilson_eo_s *h, int io, bool c12, bool dag, const HopParams &p,
                      const char *blocks, int rows, int want, int cap, cudaStream_t s, bool inject)
{
    return staged::launch_16<B16Traits>(h, io, c12, dag, p, blocks, rows, want, cap, s, inject);
}

int staged_pack_b16(const HopParams &p, bool c12, int T, char *out, cudaStream_t s)
{
    return staged::pack_16<B16Traits>(p, c12, T, out, s);
}

}  // namespace weo
