// Radius dispatch of the tiled sweep's compilation units (host code).
#include "internal.h"

namespace stencil {

#define STENCIL_UNIT_DECL(S)                                                                          \
    bool tiled_config_##S(int tx, int ty, TiledInfo *info);                                           \
    int tiled_blocks_per_sm_##S(int tx, int ty);                                                      \
    cudaError_t launch_tiled_##S(int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s); \
    cudaError_t launch_grouped_##S(int tx, int ty, const GroupShot *shots, const GroupItem *items, int n_items, \
                                   int step_off, bool absorb, cudaStream_t s);
STENCIL_UNIT_DECL(f32_r4)
STENCIL_UNIT_DECL(f32_r5)
STENCIL_UNIT_DECL(f16_r4)
STENCIL_UNIT_DECL(f16_r5)
STENCIL_UNIT_DECL(bf16_r4)
STENCIL_UNIT_DECL(bf16_r5)

#define STENCIL_UNIT_DISPATCH(S)                                                                      \
    bool tiled_config_##S(int R, int tx, int ty, TiledInfo *info)                                     \
    {                                                                                                 \
        return R == 4 ? tiled_config_##S##_r4(tx, ty, info) : R == 5 ? tiled_config_##S##_r5(tx, ty, info) : false; \
    }                                                                                                 \
    int tiled_blocks_per_sm_##S(int R, int tx, int ty)                                                \
    {                                                                                                 \
        return R == 4 ? tiled_blocks_per_sm_##S##_r4(tx, ty) : R == 5 ? tiled_blocks_per_sm_##S##_r5(tx, ty) : 0; \
    }                                                                                                 \
    cudaError_t launch_tiled_##S(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s) \
    {                                                                                                 \
        return R == 4   ? launch_tiled_##S##_r4(tx, ty, m, p, s)                                      \
               : R == 5 ? launch_tiled_##S##_r5(tx, ty, m, p, s)                                      \
                        : cudaErrorInvalidConfiguration;                                              \
    }                                                                                                 \
    cudaError_t launch_grouped_##S(int R, int tx, int ty, const GroupShot *shots, const GroupItem *items, \
                                   int n_items, int step_off, bool absorb, cudaStream_t s)           \
    {                                                                                                 \
        return R == 4   ? launch_grouped_##S##_r4(tx, ty, shots, items, n_items, step_off, absorb, s)  \
               : R == 5 ? launch_grouped_##S##_r5(tx, ty, shots, items, n_items, step_off, absorb, s)  \
                        : cudaErrorInvalidConfiguration;                                              \
    }
STENCIL_UNIT_DISPATCH(f32)
STENCIL_UNIT_DISPATCH(f16)
STENCIL_UNIT_DISPATCH(bf16)

}  // namespace stencil
