// Tiled sweep, BF16 storage with per-plane scales, radius 4: instantiations for every built tile.
#define UNIT_R 4
#define UNIT_E __nv_bfloat16
#define UNIT_TILES TILES_16
#define UNIT_NAME bf16_r4
#include "sweep_tiled_unit.cuh"
