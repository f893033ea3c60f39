// Instantiation and dispatch of the tiled sweep for one storage type; each
// sweep_tiled_*.cu includes this with its element type.
#pragma once

#include <mutex>

#include "internal.h"
#include "sweep_tiled.cuh"

namespace stencil {
namespace tiled_detail {

constexpr int SMEM_LIMIT = 227 * 1024;

template <int R, int TX, int TY, typename E>
struct Inst {
    using S = TiledShape<R, TX, TY, E>;
    static constexpr bool fits = S::VALID && S::SMEM <= SMEM_LIMIT;

    static cudaError_t prepare()
    {
        if constexpr (!fits) {
            return cudaErrorInvalidConfiguration;
        } else {
            static std::once_flag once;
            static cudaError_t status = cudaSuccess;
            std::call_once(once, [] {
                status = cudaFuncSetAttribute(sweep_tiled_kernel<R, TX, TY, E, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
                if (status == cudaSuccess)
                    status = cudaFuncSetAttribute(sweep_tiled_kernel<R, TX, TY, E, true>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
                if constexpr (S::F32)
                    if (status == cudaSuccess)
                        status = cudaFuncSetAttribute(sweep_tiled_kernel<R, TX, TY, E, false, true>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
                if (status == cudaSuccess)
                    status = cudaFuncSetAttribute(sweep_grouped_kernel<R, TX, TY, E>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
                if constexpr (S::F32)
                    if (status == cudaSuccess)
                        status = cudaFuncSetAttribute(sweep_grouped_kernel<R, TX, TY, E, true>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
            });
            return status;
        }
    }

    static int blocks_per_sm()
    {
        if constexpr (!fits) {
            return 0;
        } else {
            if (prepare() != cudaSuccess) return 0;
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_tiled_kernel<R, TX, TY, E, false>, S::NT,
                                                              S::SMEM) != cudaSuccess)
                return 0;
            return n;
        }
    }

    static bool shape(TiledInfo *info)
    {
        info->smem = S::SMEM;
        info->threads = S::NT;
        info->hx = S::HX;
        info->zmax = S::ZMAX;
        return fits;
    }

    static cudaError_t launch(const TiledMaps &m, const SweepParams &p, cudaStream_t s)
    {
        if constexpr (!fits) {
            return cudaErrorInvalidConfiguration;
        } else {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
            const int tiles_x = (p.nx + TX - 1) / TX;
            const int tiles_y = (p.ny + TY - 1) / TY;
            const int zc = p.zchunk > 0 ? p.zchunk : p.nz;
            if (S::ZMAX && zc > S::ZMAX) return cudaErrorInvalidValue;
            const int nzc = (p.nz + zc - 1) / zc;
            if ((int64_t)tiles_x * tiles_y > 0x7fffffff || nzc > 65535) return cudaErrorInvalidConfiguration;
            SweepParams q = p;
            q.tiles_x = tiles_x;
            q.zchunk = zc;
            dim3 grid(tiles_x * tiles_y, nzc);
            if (q.absorb_w > 0) {
                if constexpr (S::F32)
                    sweep_tiled_kernel<R, TX, TY, E, false, true>
                        <<<grid, S::NT, S::SMEM, s>>>(m.u_halo, m.up_core, m.k_core, q);
                else
                    return cudaErrorInvalidValue;            // the layer needs FP32 storage
            } else if (q.energy_on)
                sweep_tiled_kernel<R, TX, TY, E, true><<<grid, S::NT, S::SMEM, s>>>(m.u_halo, m.up_core, m.k_core, q);
            else
                sweep_tiled_kernel<R, TX, TY, E, false><<<grid, S::NT, S::SMEM, s>>>(m.u_halo, m.up_core, m.k_core, q);
            return cudaGetLastError();
        }
    }

    static cudaError_t launch_grouped(const GroupShot *shots, const GroupItem *items, int n_items, int step_off,
                                      bool absorb, cudaStream_t s)
    {
        if constexpr (!fits) {
            return cudaErrorInvalidConfiguration;
        } else {
            cudaError_t e = prepare();
            if (e != cudaSuccess) return e;
            if (n_items <= 0) return cudaSuccess;
            if (absorb) {
                if constexpr (S::F32)
                    sweep_grouped_kernel<R, TX, TY, E, true><<<n_items, S::NT, S::SMEM, s>>>(shots, items, step_off);
                else
                    return cudaErrorInvalidValue;            // the layer needs FP32 storage
            } else {
                sweep_grouped_kernel<R, TX, TY, E><<<n_items, S::NT, S::SMEM, s>>>(shots, items, step_off);
            }
            return cudaGetLastError();
        }
    }
};

// One tile of a unit's tile list: CALL with I = the tile's instantiation
// when the runtime (tx, ty) matches.
#define STENCIL_ONE(R_, E, TX_, TY_, CALL) \
    if (tx == TX_ && ty == TY_) { using I = Inst<R_, TX_, TY_, E>; CALL; }

}  // namespace tiled_detail
}  // namespace stencil
