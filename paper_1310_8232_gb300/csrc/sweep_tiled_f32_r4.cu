// Tiled sweep, FP32 storage, radius 4: instantiations for every built tile.
#define UNIT_R 4
#define UNIT_E float
#define UNIT_TILES TILES_F32
#define UNIT_NAME f32_r4
#include "sweep_tiled_unit.cuh"
