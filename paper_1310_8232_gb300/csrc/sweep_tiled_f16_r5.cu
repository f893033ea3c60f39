// Tiled sweep, FP16 storage with per-plane scales, radius 5: instantiations for every built tile.
#define UNIT_R 5
#define UNIT_E __half
#define UNIT_TILES TILES_16
#define UNIT_NAME f16_r5
#include "sweep_tiled_unit.cuh"
