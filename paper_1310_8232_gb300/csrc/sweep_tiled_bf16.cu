// Tiled sweep, BF16 storage with per-plane scales: instantiations.
#include "sweep_tiled_inst.cuh"

namespace stencil {
using namespace tiled_detail;

#define TILES_16(R_, E, CALL)                                                                      \
    STENCIL_ONE(R_, E, 32, 16, CALL) STENCIL_ONE(R_, E, 32, 32, CALL) STENCIL_ONE(R_, E, 64, 8, CALL) \
    STENCIL_ONE(R_, E, 64, 16, CALL) STENCIL_ONE(R_, E, 64, 32, CALL) STENCIL_ONE(R_, E, 128, 8, CALL) \
    STENCIL_ONE(R_, E, 128, 16, CALL)

bool tiled_config_bf16(int R, int tx, int ty, TiledInfo *info)
{
    STENCIL_TILE_SWITCH(__nv_bfloat16, TILES_16, return I::shape(info), return false);
}
int tiled_blocks_per_sm_bf16(int R, int tx, int ty)
{
    STENCIL_TILE_SWITCH(__nv_bfloat16, TILES_16, return I::blocks_per_sm(), return 0);
}
cudaError_t launch_tiled_bf16(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s)
{
    STENCIL_TILE_SWITCH(__nv_bfloat16, TILES_16, return I::launch(m, p, s), return cudaErrorInvalidConfiguration);
}

cudaError_t launch_grouped_bf16(int R, int tx, int ty, const GroupShot *shots, const GroupItem *items, int n_items,
                              int step_off, cudaStream_t s)
{
    STENCIL_TILE_SWITCH(__nv_bfloat16, TILES_16, return I::launch_grouped(shots, items, n_items, step_off, s),
                        return cudaErrorInvalidConfiguration);
}

}  // namespace stencil
