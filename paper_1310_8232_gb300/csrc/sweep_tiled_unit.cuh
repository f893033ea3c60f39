// One compilation unit of the tiled sweep: the built tiles of one storage
// type at one radius (the units compile in parallel).  The including file
// defines UNIT_R (4 or 5), UNIT_E (element type), UNIT_TILES (tile list
// macro) and UNIT_NAME (function-name suffix).
#include "sweep_tiled_inst.cuh"

#define TILES_F32(R_, E, CALL)                                                                   \
    STENCIL_ONE(R_, E, 32, 8, CALL) STENCIL_ONE(R_, E, 32, 16, CALL) STENCIL_ONE(R_, E, 32, 32, CALL) \
    STENCIL_ONE(R_, E, 64, 4, CALL) STENCIL_ONE(R_, E, 64, 8, CALL) STENCIL_ONE(R_, E, 64, 16, CALL)  \
    STENCIL_ONE(R_, E, 64, 32, CALL) STENCIL_ONE(R_, E, 128, 4, CALL) STENCIL_ONE(R_, E, 128, 8, CALL) \
    STENCIL_ONE(R_, E, 128, 16, CALL)

#define TILES_16(R_, E, CALL)                                                                      \
    STENCIL_ONE(R_, E, 32, 16, CALL) STENCIL_ONE(R_, E, 32, 32, CALL) STENCIL_ONE(R_, E, 64, 8, CALL) \
    STENCIL_ONE(R_, E, 64, 16, CALL) STENCIL_ONE(R_, E, 64, 32, CALL) STENCIL_ONE(R_, E, 128, 8, CALL) \
    STENCIL_ONE(R_, E, 128, 16, CALL)

#define UNIT_CAT2(a, b) a##_##b
#define UNIT_CAT(a, b) UNIT_CAT2(a, b)

namespace stencil {
using namespace tiled_detail;

bool UNIT_CAT(tiled_config, UNIT_NAME)(int tx, int ty, TiledInfo *info)
{
    UNIT_TILES(UNIT_R, UNIT_E, return I::shape(info))
    return false;
}
int UNIT_CAT(tiled_blocks_per_sm, UNIT_NAME)(int tx, int ty)
{
    UNIT_TILES(UNIT_R, UNIT_E, return I::blocks_per_sm())
    return 0;
}
cudaError_t UNIT_CAT(launch_tiled, UNIT_NAME)(int tx, int ty, const TiledMaps &m, const SweepParams &p,
                                              cudaStream_t s)
{
    UNIT_TILES(UNIT_R, UNIT_E, return I::launch(m, p, s))
    return cudaErrorInvalidConfiguration;
}
cudaError_t UNIT_CAT(launch_grouped, UNIT_NAME)(int tx, int ty, const GroupShot *shots, const GroupItem *items,
                                                int n_items, int step_off, bool absorb, cudaStream_t s)
{
    UNIT_TILES(UNIT_R, UNIT_E, return I::launch_grouped(shots, items, n_items, step_off, absorb, s))
    return cudaErrorInvalidConfiguration;
}

}  // namespace stencil
