// Instantiations and dispatch of the tiled sweep (K1, FP32 storage).
#include <mutex>

#include "internal.h"
#include "sweep_tiled.cuh"

namespace stencil {

namespace {

constexpr int SMEM_LIMIT = 227 * 1024;

template <int R, int TX, int TY>
struct Inst {
    using S = TiledShape<R, TX, TY>;
    static constexpr bool fits = S::VALID && S::SMEM <= SMEM_LIMIT;

    static cudaError_t prepare()
    {
        static std::once_flag once;
        static cudaError_t status = cudaSuccess;
        std::call_once(once, [] {
            status = cudaFuncSetAttribute(sweep_tiled_kernel<R, TX, TY>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        });
        return status;
    }

    static int blocks_per_sm()
    {
        if constexpr (!fits) {
            return 0;
        } else {
            if (prepare() != cudaSuccess) return 0;
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_tiled_kernel<R, TX, TY>, S::NT, S::SMEM) !=
                cudaSuccess)
                return 0;
            return n;
        }
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
            const int nzc = (p.nz + zc - 1) / zc;
            if ((int64_t)tiles_x * tiles_y > 0x7fffffff || nzc > 65535) return cudaErrorInvalidConfiguration;
            SweepParams q = p;
            q.tiles_x = tiles_x;
            q.zchunk = zc;
            dim3 grid(tiles_x * tiles_y, nzc);
            sweep_tiled_kernel<R, TX, TY><<<grid, S::NT, S::SMEM, s>>>(m.u_halo, m.up_core, m.k_core, q);
            return cudaGetLastError();
        }
    }
};

template <int R, int TX>
cudaError_t launch_ty(int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s)
{
    switch (ty) {
    case 4: return Inst<R, TX, 4>::launch(m, p, s);
    case 8: return Inst<R, TX, 8>::launch(m, p, s);
    case 16: return Inst<R, TX, 16>::launch(m, p, s);
    case 32:
        if constexpr (TX / 4 * 32 <= 1024) return Inst<R, TX, 32>::launch(m, p, s);
        else return cudaErrorInvalidConfiguration;
    default: return cudaErrorInvalidConfiguration;
    }
}

template <int R>
cudaError_t launch_tx(int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s)
{
    switch (tx) {
    case 32: return launch_ty<R, 32>(ty, m, p, s);
    case 64: return launch_ty<R, 64>(ty, m, p, s);
    case 128: return launch_ty<R, 128>(ty, m, p, s);
    default: return cudaErrorInvalidConfiguration;
    }
}

template <int R>
int occupancy_r(int tx, int ty)
{
#define STENCIL_OCC(TX_, TY_) \
    if (tx == TX_ && ty == TY_) return Inst<R, TX_, TY_>::blocks_per_sm();
    STENCIL_OCC(32, 8) STENCIL_OCC(32, 16) STENCIL_OCC(32, 32)
    STENCIL_OCC(64, 4) STENCIL_OCC(64, 8) STENCIL_OCC(64, 16) STENCIL_OCC(64, 32)
    STENCIL_OCC(128, 4) STENCIL_OCC(128, 8) STENCIL_OCC(128, 16) STENCIL_OCC(128, 32)
#undef STENCIL_OCC
    return 0;
}

template <int R, int TX, int TY>
bool shape_of(int *smem, int *threads, int *hx)
{
    using S = TiledShape<R, TX, TY>;
    *smem = S::SMEM;
    *threads = S::NT;
    *hx = S::HX;
    return S::VALID && S::SMEM <= SMEM_LIMIT;
}

template <int R>
bool config_r(int tx, int ty, int *smem, int *threads, int *hx)
{
#define STENCIL_SHAPE(TX_, TY_) \
    if (tx == TX_ && ty == TY_) return shape_of<R, TX_, TY_>(smem, threads, hx);
    STENCIL_SHAPE(32, 4) STENCIL_SHAPE(32, 8) STENCIL_SHAPE(32, 16) STENCIL_SHAPE(32, 32)
    STENCIL_SHAPE(64, 4) STENCIL_SHAPE(64, 8) STENCIL_SHAPE(64, 16) STENCIL_SHAPE(64, 32)
    STENCIL_SHAPE(128, 4) STENCIL_SHAPE(128, 8) STENCIL_SHAPE(128, 16) STENCIL_SHAPE(128, 32)
#undef STENCIL_SHAPE
    return false;
}

}  // namespace

bool tiled_config(int R, int tx, int ty, int *smem, int *threads, int *hx)
{
    if (R == 4) return config_r<4>(tx, ty, smem, threads, hx);
    if (R == 5) return config_r<5>(tx, ty, smem, threads, hx);
    return false;
}

int tiled_blocks_per_sm(int R, int tx, int ty)
{
    if (R == 4) return occupancy_r<4>(tx, ty);
    if (R == 5) return occupancy_r<5>(tx, ty);
    return 0;
}

cudaError_t launch_tiled(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s)
{
    if (R == 4) return launch_tx<4>(tx, ty, m, p, s);
    if (R == 5) return launch_tx<5>(tx, ty, m, p, s);
    return cudaErrorInvalidConfiguration;
}

}  // namespace stencil
