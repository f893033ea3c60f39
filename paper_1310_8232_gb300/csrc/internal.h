// Launchers shared between the kernel translation units and the host runtime.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace stencil {

// ---- K0: one thread per point (the GPU "No-Blocksize" analogue) ----
cudaError_t launch_naive(int R, const SweepParams &p, cudaStream_t s);
cudaError_t launch_image_accumulate(const float *s, const float *u, float *img, int nx, int ny, int nz,
                                    int64_t pitch, float scale, cudaStream_t st);

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
// n = v on the device, in stream order (no host staging of the value)
cudaError_t launch_set_step(int64_t *n, int64_t v, cudaStream_t s);
// a[0..n) = b[0..n) = 0 and *step = v, one launch
cudaError_t launch_clear_levels(float *a, float *b, int64_t n, int64_t *step, int64_t v, cudaStream_t s);

// ---- per-step operations around the plain sweep (plane_ops.cu) ----
struct StepOps {
    int32_t nx, ny, nz;
    int64_t pitch, plane;
    const int64_t *step_base;       // n of this step = *step_base + step_off
    int32_t step_off;
    // absorbing layer: u^{n-1} of the layer's points saved before the sweep
    int32_t absorb_w;               // 0: none
    const float2 *absorb_tab;       // (g_d, h_d) = (1/(1+eta_d), eta_d/(1+eta_d)), d = 0..W
    int64_t shell_points;
    float *save;
    Source src;                     // added after the layer when absorb_w > 0
    // plane injection (FP32 storage)
    const float *inj;
    int64_t inj_n0;
    int32_t inj_steps, inj_reverse, inj_z, inj_y;
    float inj_scale;
    // plane record
    float *rec;
    const float *scale;             // 16-bit storage: [4][nz] per-plane scales; null for FP32
    int64_t rec_n0;
    int32_t rec_cap, rec_z, rec_y;
};
// points of the layer shell within w of a face
int64_t shell_points(int nx, int ny, int nz, int w);
// before the sweep (up = u^{n-1}) / after it (up = u^{n+1})
cudaError_t launch_step_pre(const StepOps &o, void *up, cudaStream_t s);
cudaError_t launch_step_post(const StepOps &o, void *up, int storage, cudaStream_t s);

// ---- K1 / K2: 2.5D tiled sweep (TMA-staged xy tile + halo, z register ring) ----
struct TiledMaps {
    CUtensorMap u_halo;   // u^n, box (tx + 2 hx) x (ty + 2R) x 1
    CUtensorMap up_core;  // u^{n-1}, box tx x ty x 1
    CUtensorMap k_core;   // kappa, box tx x ty x 1
};
struct TiledInfo {
    int smem;             // dynamic shared memory, bytes
    int threads;          // block size
    int hx;               // x halo loaded on each side (elements)
    int zmax;             // largest z-chunk (0 = any)
};
// storage: 0 FP32, 1 FP16, 2 BF16 (the values of stencil_storage)
bool tiled_config(int R, int storage, int tx, int ty, TiledInfo *info);
cudaError_t launch_tiled(int R, int storage, int tx, int ty, const TiledMaps &m, const SweepParams &p,
                         cudaStream_t s);
// Resident blocks per SM (0 if not built / no device).
int tiled_blocks_per_sm(int R, int storage, int tx, int ty);

bool tiled_config_f32(int R, int tx, int ty, TiledInfo *info);
bool tiled_config_f16(int R, int tx, int ty, TiledInfo *info);
bool tiled_config_bf16(int R, int tx, int ty, TiledInfo *info);
int tiled_blocks_per_sm_f32(int R, int tx, int ty);
int tiled_blocks_per_sm_f16(int R, int tx, int ty);
int tiled_blocks_per_sm_bf16(int R, int tx, int ty);
cudaError_t launch_tiled_f32(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s);
cudaError_t launch_tiled_f16(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s);
cudaError_t launch_tiled_bf16(int R, int tx, int ty, const TiledMaps &m, const SweepParams &p, cudaStream_t s);

// ---- K7: two time steps per sweep (FP32; tile 64 x 16 at R = 4, 64 x 14 at R = 5) ----
struct TwoStepMaps {
    CUtensorMap u_halo;     // u^n, box (tx + 2 ex + 2 hx) x (ty + 4R) x 1
    CUtensorMap up_region;  // u^{n-1}, box (tx + 2 ex) x (ty + 2R) x 1
    CUtensorMap k_region;   // kappa, box (tx + 2 ex) x (ty + 2R) x 1
    CUtensorMap u_core;     // u^n, box tx x ty x 1
    CUtensorMap k_core;     // kappa, box tx x ty x 1
};
struct TwoStepInfo {
    int smem;               // dynamic shared memory, bytes
    int threads;            // block size
    int ex;                 // ring of stage A around the tile, x columns on each side
    int hx;                 // x halo of the u^n box beyond that ring
};
bool two_step_config(int R, int tx, int ty, TwoStepInfo *info);
int two_step_tile_y(int R);
int two_step_blocks_per_sm(int R);
// u^{n+1} -> out1, u^{n+2} -> out2 (buffers other than the inputs)
cudaError_t launch_two_step(int R, const TwoStepMaps &m, const SweepParams &p, float *out1, float *out2,
                            cudaStream_t s);

// grouped launch: one time step of every shot in `shots` (device array),
// n_items blocks, block b doing items[b]; absorb: the variant with the
// absorbing layer (FP32; shots without a layer pass through it unchanged)
cudaError_t launch_grouped(int R, int storage, int tx, int ty, const GroupShot *shots, const GroupItem *items,
                           int n_items, int step_off, bool absorb, cudaStream_t s);
cudaError_t launch_grouped_f32(int R, int tx, int ty, const GroupShot *shots, const GroupItem *items, int n_items,
                               int step_off, bool absorb, cudaStream_t s);
cudaError_t launch_grouped_f16(int R, int tx, int ty, const GroupShot *shots, const GroupItem *items, int n_items,
                               int step_off, bool absorb, cudaStream_t s);
cudaError_t launch_grouped_bf16(int R, int tx, int ty, const GroupShot *shots, const GroupItem *items, int n_items,
                                int step_off, bool absorb, cudaStream_t s);
// n[i] = min(n[i] + k, n_end[i]) for the shots of a group
cudaError_t launch_group_advance(GroupShot *shots, int n_shots, int k, cudaStream_t s);
// the served migrations' per-step work (GroupRtm) of the shots shots[list[i]]
cudaError_t launch_group_rtm(const GroupShot *shots, const int *list, int n_list, int step_off, cudaStream_t s);

// ---- K2 helpers: 16-bit fields <-> FP32 with per-plane power-of-two scales ----
// pack: v = src (or src - sub when sub is not null), FP32 (pitch elements)
// -> dst 16-bit; writes amax[z] (max |v| over plane z, float bits) and
// scale[z] (the power of two used).
cudaError_t launch_pack16(int storage, const float *src, const float *sub, void *dst, int nx, int ny, int nz,
                          int64_t pitch, float *scale, unsigned *amax, cudaStream_t s);
// unpack: 16-bit src with scale[z] -> FP32 dst (same pitch)
cudaError_t launch_unpack16(int storage, const void *src, float *dst, int nx, int ny, int nz, int64_t pitch,
                            const float *scale, cudaStream_t s);
// u^{n-1} = u^n - d^n in FP32 from the 16-bit u and d and their plane scales
cudaError_t launch_unpack16_prev(int storage, const void *u, const void *d, float *dst, int nx, int ny, int nz,
                                 int64_t pitch, const float *scale_u, const float *scale_d, cudaStream_t s);

}  // namespace stencil
