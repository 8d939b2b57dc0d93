// Device helpers shared by the kernels that stage their operands in shared
// memory through the tensor-memory accelerator (TMA): mbarrier operations,
// bulk and tensor copies from global to shared memory, the global timer for
// bounded waits, and one hopping direction computed from shared memory.
// Inline PTX for sm_103a.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "weo_dslash.cuh"

namespace weo {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// L2 policy for data read again soon by another item (normal priority, above
// the evict-first streams)
__device__ __forceinline__ uint64_t policy_evict_normal()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                          uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// wait for the phase of `bar` with the given parity to complete, at most
// limit_ns nanoseconds; on expiry set bit 0 of *err and return false
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity,
                                                  unsigned long long limit_ns, unsigned int *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, 1u);
            return false;
        }
    }
    return true;
}

// one hopping direction from shared memory: spinor planes of stride `ss`
// (complex) at index si, link planes of stride `ls` at index li
template <int MU, bool FWD, int S0>
__device__ __forceinline__ void staged_dir(cx<float> (&acc)[12], const float2 *sp, int ss, int si,
                                           const float4 *l4, const float2 *l2, int ls, int li)
{
    constexpr int S = FWD ? S0 : -S0;
    const float4 a = l4[li], b = l4[ls + li], c = l4[2 * ls + li], d = l4[3 * ls + li];
    const float2 e = l2[li];
    cx<float> U[3][3];
    U[0][0] = {a.x, a.y};
    U[0][1] = {a.z, a.w};
    U[0][2] = {b.x, b.y};
    U[1][0] = {b.z, b.w};
    U[1][1] = {c.x, c.y};
    U[1][2] = {c.z, c.w};
    U[2][0] = {d.x, d.y};
    U[2][1] = {d.z, d.w};
    U[2][2] = {e.x, e.y};
    cx<float> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float2 q = sp[k * ss + si];
        v[k] = {q.x, q.y};
    }
    cx<float> h[2][3];
#pragma unroll
    for (int col = 0; col < 3; ++col)
        project<MU, S>(v[col], v[3 + col], v[6 + col], v[9 + col], h[0][col], h[1][col]);
    cx<float> w[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            cx<float> zz = {0.f, 0.f};
#pragma unroll
            for (int col = 0; col < 3; ++col)
                zz = FWD ? cfma(U[r][col], h[s][col], zz) : cfmaconj(U[col][r], h[s][col], zz);
            w[s][r] = zz;
        }
#pragma unroll
    for (int col = 0; col < 3; ++col)
        reconstruct<MU, S>(acc[col], acc[3 + col], acc[6 + col], acc[9 + col], w[0][col], w[1][col]);
}

}  // namespace weo
