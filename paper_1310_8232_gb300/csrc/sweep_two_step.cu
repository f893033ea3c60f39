// Instantiation and launch of the two-step sweep (K7): tile 64 x 16 at R = 4,
// 64 x 14 at R = 5, so that stage A's items fit 256 threads (8 warps, two
// per scheduler: up to 255 registers a thread without spilling).
#include <mutex>

#include "internal.h"
#include "sweep_two_step.cuh"

namespace stencil {
namespace {

constexpr int T2_TX = 64;
template <int R>
constexpr int t2_ty() { return R == 5 ? 14 : 16; }

template <int R>
struct T2Inst {
    static constexpr int T2_TY = t2_ty<R>();
    using S = TwoStepShape<R, T2_TX, T2_TY>;
    static_assert(S::NT == 256, "8 warps");
    static cudaError_t prepare()
    {
        static std::once_flag once;
        static cudaError_t status = cudaSuccess;
        std::call_once(once, [] {
            status = cudaFuncSetAttribute(sweep_two_step_kernel<R, T2_TX, T2_TY>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        });
        return status;
    }
};

template <int R>
cudaError_t launch_r(const TwoStepMaps &m, const SweepParams &p, float *out1, float *out2, cudaStream_t s)
{
    constexpr int T2_TY = t2_ty<R>();
    using S = TwoStepShape<R, T2_TX, T2_TY>;
    cudaError_t e = T2Inst<R>::prepare();
    if (e != cudaSuccess) return e;
    SweepParams q = p;
    q.tiles_x = (p.nx + T2_TX - 1) / T2_TX;
    const int tiles_y = (p.ny + T2_TY - 1) / T2_TY;
    const int zc = p.zchunk > 0 ? p.zchunk : p.nz;
    const dim3 grid(q.tiles_x * tiles_y, (p.nz + zc - 1) / zc);
    sweep_two_step_kernel<R, T2_TX, T2_TY><<<grid, S::NT, S::SMEM, s>>>(m.u_halo, m.up_region, m.k_region, m.u_core,
                                                                         m.k_core, q, out1, out2);
    return cudaGetLastError();
}

}  // namespace

bool two_step_config(int R, int tx, int ty, TwoStepInfo *info)
{
    if (R == 4 && tx == T2_TX && ty == t2_ty<4>()) {
        using S = TwoStepShape<4, T2_TX, t2_ty<4>()>;
        *info = {S::SMEM, S::NT, S::EX, S::HX};
        return true;
    }
    if (R == 5 && tx == T2_TX && ty == t2_ty<5>()) {
        using S = TwoStepShape<5, T2_TX, t2_ty<5>()>;
        *info = {S::SMEM, S::NT, S::EX, S::HX};
        return true;
    }
    return false;
}

int two_step_tile_y(int R) { return R == 5 ? t2_ty<5>() : t2_ty<4>(); }

int two_step_blocks_per_sm(int R)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (R == 4 && T2Inst<4>::prepare() == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_two_step_kernel<4, T2_TX, t2_ty<4>()>,
                                                          T2Inst<4>::S::NT, T2Inst<4>::S::SMEM);
    if (R == 5 && T2Inst<5>::prepare() == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_two_step_kernel<5, T2_TX, t2_ty<5>()>,
                                                          T2Inst<5>::S::NT, T2Inst<5>::S::SMEM);
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_two_step(int R, const TwoStepMaps &m, const SweepParams &p, float *out1, float *out2,
                            cudaStream_t s)
{
    if (R == 4) return launch_r<4>(m, p, out1, out2, s);
    if (R == 5) return launch_r<5>(m, p, out1, out2, s);
    return cudaErrorInvalidValue;
}

}  // namespace stencil
