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

cudaError_t launch_tiled(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s)
{
    if (R == 4) return launch_tx<4>(tx, ty, m, p, s);
    if (R == 5) return launch_tx<5>(tx, ty, m, p, s);
    return cudaErrorInvalidConfiguration;
}

}  // namespace stencil
