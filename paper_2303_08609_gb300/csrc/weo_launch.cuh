// Template launcher for the hopping kernel: runtime (dag, axpy, rhs block) ->
// compile-time instance. Included by one translation unit per precision.
#pragma once

#include <mutex>
#include <type_traits>

#include "weo_internal.h"

namespace weo {

template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int NL>
int launch_lanes(const HopParams &p, const LaunchCfg &cfg, cudaStream_t s)
{
    const int sites = cfg.threads / NL;
    // (site block, right-hand-side block) pairs, right-hand-side block fastest
    dim3 grid((unsigned)(((p.vh + sites - 1) / sites) * ((p.nrhs + NL - 1) / NL)));
    hop_kernel_lanes<SIn, SOut, SX, Lk, Dag, Axpy, NL><<<grid, cfg.threads, 0, s>>>(p);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int NRL, int RP = 1>
int launch_tile_links(const HopParams &p, cudaStream_t s)
{
    constexpr int T = 256 / NRL;
    const size_t smem = (size_t)576 * T;
    auto kern = hop_kernel_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, NRL, RP>;
    if (smem > 48 * 1024) {  // opt in to more than 48 KB, once per instance
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [&] {
            attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        WEO_CUDA(attr);
    }
    kern<<<(unsigned)((p.vh + T - 1) / T), 256, smem, s>>>(p);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <class SIn, class SOut, class SX, class Lk, bool Dag, bool Axpy, int R>
int launch_instance(const HopParams &p, const LaunchCfg &cfg, cudaStream_t s)
{
    if constexpr (R == 1 && sizeof(typename SOut::real) == 4) {
        // several right-hand sides over tiles whose links sit in shared memory
        if (cfg.tile_links && p.nrhs >= 2) {
            // 2 right-hand sides per thread (sharing each link read) when asked
            // for and there are enough of them to fill a pass
            if (cfg.tile_rhs_per_thread == 2 && p.nrhs >= 2 * cfg.tile_links) {
                if (cfg.tile_links == 8) return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 8, 2>(p, s);
                if (cfg.tile_links == 4) return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 4, 2>(p, s);
                return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 2, 2>(p, s);
            }
            if (cfg.tile_links == 8) return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 8>(p, s);
            if (cfg.tile_links == 4) return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 4>(p, s);
            return launch_tile_links<SIn, SOut, SX, Lk, Dag, Axpy, 2>(p, s);
        }
        // right-hand sides sharing link loads across lanes (never more lanes than
        // right-hand sides)
        int nl = cfg.lanes;
        while (nl > 1 && nl > p.nrhs) nl /= 2;
        if (nl == 8) return launch_lanes<SIn, SOut, SX, Lk, Dag, Axpy, 8>(p, cfg, s);
        if (nl == 4) return launch_lanes<SIn, SOut, SX, Lk, Dag, Axpy, 4>(p, cfg, s);
        if (nl == 2) return launch_lanes<SIn, SOut, SX, Lk, Dag, Axpy, 2>(p, cfg, s);
    }
    // blocked site order: CTAs of 8 Lx/2 threads, one per 2x2x2 block of rows
    const bool blocked = cfg.blocked && 8 * p.lxh >= 64 && 8 * p.lxh <= 256;
    const int threads = blocked ? 8 * p.lxh : cfg.threads;
    const long long site_blocks = blocked ? (long long)(p.ly / 2) * (p.lz / 2) * (p.lt / 2)
                                          : (p.vh + threads - 1) / threads;
    HopParams q = p;
    q.blocked = blocked ? 1 : 0;
    dim3 grid((unsigned)(site_blocks * ((p.nrhs + R - 1) / R)));
    // the 64-register cap pays for 18-real FP32 and 16-bit links; the FP32
    // 12-real rebuild spills too much under it
    if constexpr (sizeof(typename SOut::real) == 4 && R == 1 && !std::is_same<Lk, LkF32_12>::value)
        hop_kernel_occ<SIn, SOut, SX, Lk, Dag, Axpy, R><<<grid, threads, 0, s>>>(q);
    else
        hop_kernel<SIn, SOut, SX, Lk, Dag, Axpy, R><<<grid, threads, 0, s>>>(q);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

template <class SIn, class SOut, class SX, class Lk, int R>
int launch_da(bool dag, bool axpy, const HopParams &p, const LaunchCfg &cfg, cudaStream_t s)
{
    if (dag)
        return axpy ? launch_instance<SIn, SOut, SX, Lk, true, true, R>(p, cfg, s)
                    : launch_instance<SIn, SOut, SX, Lk, true, false, R>(p, cfg, s);
    return axpy ? launch_instance<SIn, SOut, SX, Lk, false, true, R>(p, cfg, s)
                : launch_instance<SIn, SOut, SX, Lk, false, false, R>(p, cfg, s);
}

}  // namespace weo
