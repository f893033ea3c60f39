// Per-step operations around the plain sweep, each a small kernel launched
// after (or, for the layer's save, before) the sweep on the same stream, so
// the hot sweep carries none of their code:
//   - the absorbing layer of the centred damped wave equation,
//         u^{n+1} = (2u^n - (1-eta) u^{n-1} + kappa Lambda(u^n)) / (1+eta)
//                 = (plain update + eta u^{n-1}) / (1+eta),
//     as a save of u^{n-1} on the layer's points before the sweep overwrites
//     it and an apply pass after it (eta = eta_max ((W-d)/W)^2 at distance
//     d < W from the nearest face, applied as plain * g_d + u^{n-1} * h_d
//     with g_d = 1/(1+eta), h_d = eta/(1+eta) from the plan's table; the
//     tiled FP32 sweep folds the same operations into its own update);
//   - the point source, when a layer is present (it is added after the
//     damping, as in the time loop's order);
//   - the injection of data on a plane (the adjoint source of RTM);
//   - the record of a plane of u^{n+1} (receiver traces, "sismic").
// Every kernel reads the step n from the device step counter, so captured
// graphs replay them at any step.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "stencil.h"

namespace stencil {

namespace {

__device__ __forceinline__ int64_t step_of(const StepOps &o) { return *o.step_base + o.step_off; }

// Layer index maps along one axis of n points with a layer of w: the c =
// min(n, 2w) indices within w of an end, and the n - c others.
__device__ __forceinline__ int layer_coord(int k, int n, int w)
{
    return 2 * w >= n ? k : (k < w ? k : n - 2 * w + k);
}

// The layer shell in three disjoint parts:
//   part 0: the planes z within w of an end; all rows, all x;
//   part 1: the other planes; the rows y within w of an end; all x;
//   part 2: the other planes and rows; the columns x within w of an end.
// Saved values sit at a compact index, the parts one after another.  Parts
// 0 and 1 are whole rows: a (x block, row group, plane) grid, SHELL_ROWS rows
// per block; part 2 packs the 2w-wide row ends of a plane densely, one
// division per thread.
constexpr int SHELL_ROWS = 8;

struct ShellPart {
    int planes, rows, width;        // extent of the part
    int64_t base;                   // first compact index of the part
};

__host__ __device__ inline ShellPart shell_part(int part, int nx, int ny, int nz, int w)
{
    const int cz = min(nz, 2 * w), cy = min(ny, 2 * w), cx = min(nx, 2 * w);
    const int64_t a = (int64_t)cz * ny * nx, b = (int64_t)(nz - cz) * cy * nx;
    if (part == 0) return {cz, ny, nx, 0};
    if (part == 1) return {nz - cz, cy, nx, a};
    return {nz - cz, ny - cy, cx, a + b};
}

template <bool APPLY>
__device__ __forceinline__ void shell_point_op(const StepOps &o, float *field, int64_t t, int x, int y, int z)
{
    float *q = field + z * o.plane + y * o.pitch + x;
    if (!APPLY) {
        o.save[t] = *q;
    } else {
        const int d = min(min(min(x, o.nx - 1 - x), min(y, o.ny - 1 - y)), min(z, o.nz - 1 - z));
        const float2 g = o.absorb_tab[min(d, o.absorb_w)];
        *q = fmaf(g.y, o.save[t], *q * g.x);
    }
}

// parts 0 and 1: blockIdx = (x block, row group, plane)
template <bool APPLY>
__global__ void shell_rows_kernel(StepOps o, float *field, int part)
{
    const ShellPart sp = shell_part(part, o.nx, o.ny, o.nz, o.absorb_w);
    const int w = o.absorb_w, k = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= o.nx) return;
    const int z = part == 0 ? layer_coord(k, o.nz, w) : w + k;
    const int r1 = min(sp.rows, (int)(blockIdx.y + 1) * SHELL_ROWS);
    for (int r = blockIdx.y * SHELL_ROWS; r < r1; ++r) {
        const int y = part == 0 ? r : layer_coord(r, o.ny, w);
        shell_point_op<APPLY>(o, field, sp.base + ((int64_t)k * sp.rows + r) * o.nx + x, x, y, z);
    }
}

// part 2: blockIdx = (chunk of the plane's packed row ends, plane)
template <bool APPLY>
__global__ void shell_ends_kernel(StepOps o, float *field)
{
    const ShellPart sp = shell_part(2, o.nx, o.ny, o.nz, o.absorb_w);
    const int w = o.absorb_w, k = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;     // packed index within the plane
    if (j >= sp.rows * sp.width) return;
    const int r = j / sp.width, i = j - r * sp.width;
    shell_point_op<APPLY>(o, field, sp.base + (int64_t)k * sp.rows * sp.width + j, layer_coord(i, o.nx, w), w + r,
                          w + k);
}

template <bool APPLY>
cudaError_t launch_shell(const StepOps &o, float *field, cudaStream_t s)
{
    for (int part = 0; part < 2; ++part) {
        const ShellPart sp = shell_part(part, o.nx, o.ny, o.nz, o.absorb_w);
        if (sp.planes <= 0 || sp.rows <= 0) continue;
        dim3 grid((o.nx + 127) / 128, (sp.rows + SHELL_ROWS - 1) / SHELL_ROWS, sp.planes);
        shell_rows_kernel<APPLY><<<grid, 128, 0, s>>>(o, field, part);
    }
    const ShellPart sp = shell_part(2, o.nx, o.ny, o.nz, o.absorb_w);
    if (sp.planes > 0 && sp.rows > 0 && sp.width > 0) {
        dim3 grid((int)(((int64_t)sp.rows * sp.width + 255) / 256), sp.planes);
        shell_ends_kernel<APPLY><<<grid, 256, 0, s>>>(o, field);
    }
    return cudaGetLastError();
}

__global__ void source_add_kernel(StepOps o, float *field)
{
    const double t = (double)step_of(o) * o.src.dt;
    field[o.src.z * o.plane + o.src.y * o.pitch + o.src.x] += (float)(o.src.scale * ricker(o.src.f, o.src.t0, t));
}

__global__ void inject_kernel(StepOps o, float *field)
{
    const int64_t m = step_of(o) - o.inj_n0;
    const int64_t idx = o.inj_reverse ? o.inj_steps - 1 - m : m;
    if (m < 0 || idx < 0 || idx >= o.inj_steps) return;
    const int rows = o.inj_y < 0 ? o.ny : 1;
    const float *d = o.inj + idx * rows * (int64_t)o.nx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)rows * o.nx;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / o.nx), x = (int)(t - (int64_t)r * o.nx);
        const int y = o.inj_y < 0 ? r : o.inj_y;
        field[o.inj_z * o.plane + y * o.pitch + x] += o.inj_scale * d[t];
    }
}

template <typename E>
__device__ __forceinline__ float to_f32(E h)
{
    if constexpr (std::is_same<E, float>::value) return h;
    else if constexpr (std::is_same<E, __half>::value) return __half2float(h);
    else return __bfloat162float(h);
}

template <typename E>
__global__ void record_kernel(StepOps o, const E *field)
{
    const int64_t n = step_of(o);
    const int64_t m = n - o.rec_n0;
    if (m < 0 || m >= o.rec_cap) return;
    // 16-bit storage: the plane's scale of level n+1
    const float s = o.scale ? o.scale[((n + 1) & 3) * o.nz + o.rec_z] : 1.0f;
    const int rows = o.rec_y < 0 ? o.ny : 1;
    float *d = o.rec + m * rows * (int64_t)o.nx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)rows * o.nx;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / o.nx), x = (int)(t - (int64_t)r * o.nx);
        const int y = o.rec_y < 0 ? r : o.rec_y;
        d[t] = to_f32(field[o.rec_z * o.plane + y * o.pitch + x]) * s;
    }
}

int blocks_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8)); }

}  // namespace

int64_t shell_points(int nx, int ny, int nz, int w)
{
    if (w <= 0) return 0;
    const int64_t cz = std::min(nz, 2 * w), cy = std::min(ny, 2 * w), cx = std::min(nx, 2 * w);
    return cz * ny * nx + (nz - cz) * cy * nx + (nz - cz) * (ny - cy) * cx;
}

cudaError_t launch_step_pre(const StepOps &o, void *up, cudaStream_t s)
{
    if (o.absorb_w > 0 && o.shell_points > 0) return launch_shell<false>(o, static_cast<float *>(up), s);
    return cudaGetLastError();
}

cudaError_t launch_step_post(const StepOps &o, void *up, int storage, cudaStream_t s)
{
    if (o.absorb_w > 0 && o.shell_points > 0) {
        cudaError_t e = launch_shell<true>(o, static_cast<float *>(up), s);
        if (e != cudaSuccess) return e;
    }
    if (o.absorb_w > 0 && o.src.on) source_add_kernel<<<1, 1, 0, s>>>(o, static_cast<float *>(up));
    if (o.inj && o.inj_z >= 0) {
        const int64_t work = (int64_t)(o.inj_y < 0 ? o.ny : 1) * o.nx;
        inject_kernel<<<blocks_for(work), 256, 0, s>>>(o, static_cast<float *>(up));
    }
    if (o.rec && o.rec_z >= 0) {
        const int64_t work = (int64_t)(o.rec_y < 0 ? o.ny : 1) * o.nx;
        if (storage == STENCIL_FP32)
            record_kernel<float><<<blocks_for(work), 256, 0, s>>>(o, static_cast<const float *>(up));
        else if (storage == STENCIL_FP16)
            record_kernel<__half><<<blocks_for(work), 256, 0, s>>>(o, static_cast<const __half *>(up));
        else
            record_kernel<__nv_bfloat16><<<blocks_for(work), 256, 0, s>>>(o, static_cast<const __nv_bfloat16 *>(up));
    }
    return cudaGetLastError();
}

}  // namespace stencil
