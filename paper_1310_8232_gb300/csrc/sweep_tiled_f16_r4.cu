// Tiled sweep, FP16 storage with per-plane scales, radius 4: instantiations for every built tile.
#define UNIT_R 4
#define UNIT_E __half
#define UNIT_TILES TILES_16
#define UNIT_NAME f16_r4
#include "sweep_tiled_unit.cuh"
