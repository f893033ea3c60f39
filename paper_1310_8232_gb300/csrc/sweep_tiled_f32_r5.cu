// Tiled sweep, FP32 storage, radius 5: instantiations for every built tile.
#define UNIT_R 5
#define UNIT_E float
#define UNIT_TILES TILES_F32
#define UNIT_NAME f32_r5
#include "sweep_tiled_unit.cuh"
