// Launchers shared between the kernel translation units and the host runtime.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace stencil {

// ---- K0: one thread per point (the GPU "No-Blocksize" analogue) ----
cudaError_t launch_naive(int R, const SweepParams &p, cudaStream_t s);

// ---- K4: kappa = v^2 dt^2/dx^2 in place over a pitched copy of v; v range ----
// vmax_bits / n_bad are device scalars (uint32 bit pattern of the max, count
// of non-positive or non-finite velocities); the caller zeroes them first.
cudaError_t launch_coef_init(float *kv, int nx, int ny, int nz, int64_t pitch, double dt2_dx2,
                             unsigned *vmax_bits, unsigned long long *n_bad, cudaStream_t s);

// ---- K5: deterministic FP64 reductions (per-block partials, fixed-order sum) ----
constexpr int RED_BLOCKS = 1184;   // 152 SMs x 8, fixed so results are reproducible
constexpr int RED_THREADS = 256;
// energy: out[0] = sum (u1-u0)^2/kappa - u1*Lambda(u0)
cudaError_t launch_energy(int R, const float *u1, const float *u0, const float *kappa, int nx, int ny, int nz,
                          int64_t pitch, double *partials, double *out, cudaStream_t s);
// out[0] = sum (a - b)^2, out[1] = sum b^2; a pitched FP32, b dense FP64
cudaError_t launch_sqdiff(const float *a, const double *b, int nx, int ny, int nz, int64_t pitch,
                          double *partials, double *out, cudaStream_t s);

// n += k on the device (step counter between launch chunks)
cudaError_t launch_advance(int64_t *n, int k, cudaStream_t s);

// ---- K1: 2.5D tiled sweep (TMA-staged xy tile + halo, z register queue) ----
struct TiledMaps {
    CUtensorMap u_halo;   // u^n, box (tx + 2 hx) x (ty + 2R) x 1
    CUtensorMap up_core;  // u^{n-1}, box tx x ty x 1
    CUtensorMap k_core;   // kappa, box tx x ty x 1
};
// Returns true and the dynamic shared memory size if (R, tx, ty) is built
// and fits; hx = x-halo width loaded (R rounded up to 16 bytes).
bool tiled_config(int R, int tx, int ty, int *smem_bytes, int *threads, int *hx);
cudaError_t launch_tiled(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s);
// Resident blocks per SM of the tiled kernel (0 if not built / no device).
int tiled_blocks_per_sm(int R, int tx, int ty);

}  // namespace stencil
