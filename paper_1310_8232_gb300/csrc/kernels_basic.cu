// K0 (naive sweep), K4 (coefficient init + velocity range), K5 (FP64
// validation reductions), the step-counter kernel and the imaging condition.
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace stencil {

// ---------------------------------------------------------------------------
// K0: one thread per grid point; every neighbour is read from global memory
// with an explicit bounds test (ghost zeros).  The GPU counterpart of the
// paper's "No-Blocksize" variant (Sec. 3.1): no data staging at all.
// NAIVE_NT threads a block: TXN = nx rounded up to a warp (at most 128)
// along x times NAIVE_NT / TXN rows, so a narrow grid does not leave most
// threads idle; grid (ceil(nx/TXN), ceil(ny/(NAIVE_NT/TXN)), nz).  Each step is launched as a
// programmatic dependent of the previous one: its blocks are scheduled while
// that step drains and wait before touching memory, which hides most of the
// launch latency on the small grids this kernel serves.
// ---------------------------------------------------------------------------
constexpr int NAIVE_NT = 128;

template <int R, bool REC>
__global__ void __launch_bounds__(NAIVE_NT) sweep_naive_kernel(SweepParams p)
{
    grid_dependency_wait();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const bool in = x < p.nx && y < p.ny;
    if (!REC && !in) return;
    float e = 0.0f;                           // REC: this point's energy term
    if (in) {
        const int64_t q = (int64_t)z * p.plane + (int64_t)y * p.pitch + x;
        const float *u = static_cast<const float *>(p.u);
        float *up = static_cast<float *>(p.up);
        const float c = u[q];
        float acc = 3.0f * wf<R>(0) * c;
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            float s = (x - r >= 0) ? u[q - r] : 0.0f;
            s += (x + r < p.nx) ? u[q + r] : 0.0f;
            s += (y - r >= 0) ? u[q - r * p.pitch] : 0.0f;
            s += (y + r < p.ny) ? u[q + r * p.pitch] : 0.0f;
            s += (z - r >= 0) ? u[q - r * p.plane] : 0.0f;
            s += (z + r < p.nz) ? u[q + r * p.plane] : 0.0f;
            acc = fmaf(wf<R>(r), s, acc);
        }
        const float kap = p.kappa[q];
        float nxt = fmaf(kap, acc, 2.0f * c - up[q]);
        if (p.src.on && x == p.src.x && y == p.src.y && z == p.src.z) {
            const double t = (double)current_step(p) * p.src.dt;
            nxt += (float)(p.src.scale * ricker(p.src.f, p.src.t0, t));
        }
        up[q] = nxt;
        if (REC && p.energy_on) {
            const float d = nxt - c;
            e = __fdividef(d * d, kap) - nxt * acc;
        }
    }
    if (REC && p.energy_on) {
        // block partial (FP32 per warp, FP64 over the warps in order), then
        // the last block adds every partial in a fixed order with all its threads
        __shared__ double wsum[NAIVE_NT / 32];
        __shared__ int last;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if ((tid & 31) == 0) wsum[tid >> 5] = (double)e;
        __syncthreads();
        const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
        if (tid == 0) {
            const unsigned id = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            double b = 0.0;
            for (int w = 0; w < NAIVE_NT / 32; ++w) b += wsum[w];
            p.energy_part[id] = b;
            __threadfence();
            last = atomicAdd(p.energy_count, 1u) == nblk - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            __shared__ double tsum[NAIVE_NT];
            double a = 0.0;
            for (unsigned k = tid; k < nblk; k += NAIVE_NT) a += *((volatile const double *)p.energy_part + k);
            tsum[tid] = a;
            __syncthreads();
            for (int w = NAIVE_NT / 2; w > 0; w >>= 1) {
                if (tid < w) tsum[tid] += tsum[tid + w];
                __syncthreads();
            }
            if (tid == 0) {
                const int64_t m = current_step(p) - p.rec_n0;
                if (m >= 0 && m < p.rec_cap) p.energy[m] = tsum[0];
                *p.energy_count = 0u;
            }
        }
    }
}

cudaError_t launch_naive(int R, const SweepParams &p, cudaStream_t s)
{
    const int txn = std::min(128, (p.nx + 31) / 32 * 32);
    const int tyn = NAIVE_NT / txn;
    const int gy = (p.ny + tyn - 1) / tyn;
    if (gy > 65535 || p.nz > 65535) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nx + txn - 1) / txn, gy, p.nz);
    cfg.blockDim = dim3(txn, tyn, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool rec = p.energy_on != 0;
    if (R == 4 && rec) return cudaLaunchKernelEx(&cfg, sweep_naive_kernel<4, true>, p);
    if (R == 4) return cudaLaunchKernelEx(&cfg, sweep_naive_kernel<4, false>, p);
    if (R == 5 && rec) return cudaLaunchKernelEx(&cfg, sweep_naive_kernel<5, true>, p);
    if (R == 5) return cudaLaunchKernelEx(&cfg, sweep_naive_kernel<5, false>, p);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// K4: kappa[p] = v[p]^2 dt^2 / dx^2, written over the pitched copy of v; also
// the largest velocity (bit pattern max, valid for positive floats) and the
// number of invalid velocities.
//
// FP32 only (FP64 runs at a small fraction of the FP32 rate on this part):
// v^2 is kept exactly as p + e (e = fma(v, v, -p)), the constant as
// c_hi + c_lo (two floats), and the product is rounded once at the end, so
// kappa is the float nearest v^2 c except within ~2^-46 of a rounding
// midpoint.  One warp per row, 16-byte accesses where the rows allow them:
// no index division, 8 B per point of HBM traffic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kappa_of(float v, float c_hi, float c_lo, unsigned &vmax, unsigned &bad)
{
    if (!(v > 0.0f) || !isfinite(v)) {
        ++bad;
        return 0.0f;
    }
    vmax = max(vmax, __float_as_uint(v));
    const float p = v * v;
    const float e = fmaf(v, v, -p);
    return fmaf(p, c_hi, fmaf(p, c_lo, e * c_hi));
}

__global__ void coef_init_kernel(float *kv, int nx, int64_t rows, int64_t pitch, float c_hi, float c_lo,
                                 unsigned *vmax_bits, unsigned long long *n_bad)
{
    constexpr int DEPTH = 4;               // 16-byte loads in flight per lane and row pass
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool vec = pitch % 4 == 0 && reinterpret_cast<uintptr_t>(kv) % 16 == 0;
    const int nx4 = vec ? nx / 4 : 0;
    unsigned local_max = 0, local_bad = 0;
    for (int64_t row = warp; row < rows; row += n_warps) {
        float *r = kv + row * pitch;
        float4 *r4 = reinterpret_cast<float4 *>(r);
        for (int base = 0; base < nx4; base += 32 * DEPTH) {
            float4 q[DEPTH];
#pragma unroll
            for (int j = 0; j < DEPTH; ++j) {
                const int i = base + 32 * j + lane;
                if (i < nx4) q[j] = r4[i];
            }
#pragma unroll
            for (int j = 0; j < DEPTH; ++j) {
                const int i = base + 32 * j + lane;
                if (i < nx4) {
                    q[j].x = kappa_of(q[j].x, c_hi, c_lo, local_max, local_bad);
                    q[j].y = kappa_of(q[j].y, c_hi, c_lo, local_max, local_bad);
                    q[j].z = kappa_of(q[j].z, c_hi, c_lo, local_max, local_bad);
                    q[j].w = kappa_of(q[j].w, c_hi, c_lo, local_max, local_bad);
                    r4[i] = q[j];
                }
            }
        }
        for (int x = 4 * nx4 + lane; x < nx; x += 32) r[x] = kappa_of(r[x], c_hi, c_lo, local_max, local_bad);
    }
    local_max = __reduce_max_sync(0xffffffffu, local_max);
    local_bad = __reduce_add_sync(0xffffffffu, local_bad);
    if (lane == 0) {
        if (local_max) atomicMax(vmax_bits, local_max);
        if (local_bad) atomicAdd(n_bad, (unsigned long long)local_bad);
    }
}

cudaError_t launch_coef_init(float *kv, int nx, int ny, int nz, int64_t pitch, double dt2_dx2,
                             unsigned *vmax_bits, unsigned long long *n_bad, cudaStream_t s)
{
    const float c_hi = (float)dt2_dx2;
    const float c_lo = (float)(dt2_dx2 - (double)c_hi);
    coef_init_kernel<<<152 * 8, 256, 0, s>>>(kv, nx, (int64_t)ny * nz, pitch, c_hi, c_lo, vmax_bits, n_bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K5: FP64 reductions.  Each thread walks a fixed grid-stride sequence, each
// block reduces in a fixed tree, one block sums the per-block partials in
// index order: the result depends only on the data, not on scheduling.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void block_sum_store(double (&v)[N], double *dst)
{
    __shared__ double red[N][RED_THREADS / 32];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double s = 0.0;
            for (int w = 0; w < RED_THREADS / 32; ++w) s += red[k][w];
            dst[k] = s;
        }
    }
}

template <int N>
__global__ void sum_partials_kernel(const double *partials, int nblocks, double *out)
{
    // one block: thread t sums partials t, t+256, ... in order, then the tree
    double v[N];
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] += partials[(int64_t)b * N + k];
    block_sum_store<N>(v, out);
}

template <int R>
__device__ __forceinline__ double at_d(const float *u, int x, int y, int z, int nx, int ny, int nz,
                                       int64_t pitch, int64_t plane)
{
    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) return 0.0;
    return (double)u[(int64_t)z * plane + (int64_t)y * pitch + x];
}

template <int R>
__global__ void __launch_bounds__(RED_THREADS) energy_kernel(const float *u1, const float *u0,
                                                             const float *kappa, int nx, int ny, int nz,
                                                             int64_t pitch, double *partials)
{
    const int64_t plane = pitch * ny;
    const int64_t total = (int64_t)nx * ny * nz;
    double e[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nx;
        const int x = (int)(i - row * nx);
        const int z = (int)(row / ny);
        const int y = (int)(row - (int64_t)z * ny);
        const int64_t q = (int64_t)z * plane + (int64_t)y * pitch + x;
        double lap = 3.0 * wd<R>(0) * (double)u0[q];
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            double s = at_d<R>(u0, x - r, y, z, nx, ny, nz, pitch, plane);
            s += at_d<R>(u0, x + r, y, z, nx, ny, nz, pitch, plane);
            s += at_d<R>(u0, x, y - r, z, nx, ny, nz, pitch, plane);
            s += at_d<R>(u0, x, y + r, z, nx, ny, nz, pitch, plane);
            s += at_d<R>(u0, x, y, z - r, nx, ny, nz, pitch, plane);
            s += at_d<R>(u0, x, y, z + r, nx, ny, nz, pitch, plane);
            lap += wd<R>(r) * s;
        }
        const double a = (double)u1[q];
        const double d = a - (double)u0[q];
        e[0] += d * d / (double)kappa[q] - a * lap;
    }
    block_sum_store<1>(e, partials + blockIdx.x);
}

cudaError_t launch_energy(int R, const float *u1, const float *u0, const float *kappa, int nx, int ny, int nz,
                          int64_t pitch, double *partials, double *out, cudaStream_t s)
{
    if (R == 4)
        energy_kernel<4><<<RED_BLOCKS, RED_THREADS, 0, s>>>(u1, u0, kappa, nx, ny, nz, pitch, partials);
    else if (R == 5)
        energy_kernel<5><<<RED_BLOCKS, RED_THREADS, 0, s>>>(u1, u0, kappa, nx, ny, nz, pitch, partials);
    else
        return cudaErrorInvalidValue;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<1><<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(RED_THREADS) sqdiff_kernel(const float *a, const double *b, int nx, int ny,
                                                             int nz, int64_t pitch, double *partials)
{
    const int64_t plane = pitch * ny;
    const int64_t total = (int64_t)nx * ny * nz;
    double v[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / nx;
        const int x = (int)(i - row * nx);
        const int z = (int)(row / ny);
        const int y = (int)(row - (int64_t)z * ny);
        const double av = (double)a[(int64_t)z * plane + (int64_t)y * pitch + x];
        const double bv = b[i];
        const double d = av - bv;
        v[0] += d * d;
        v[1] += bv * bv;
    }
    block_sum_store<2>(v, partials + 2 * blockIdx.x);
}

cudaError_t launch_sqdiff(const float *a, const double *b, int nx, int ny, int nz, int64_t pitch,
                          double *partials, double *out, cudaStream_t s)
{
    sqdiff_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, nx, ny, nz, pitch, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<2><<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, out);
    return cudaGetLastError();
}

__global__ void advance_kernel(int64_t *n, int k) { *n += k; }
__global__ void set_step_kernel(int64_t *n, int64_t v) { *n = v; }

// Zero two FP32 arrays of n elements (16-byte aligned when vec) and set the
// step counter: the reset of a plan's two levels in one launch.
__global__ void clear_levels_kernel(float *a, float *b, int64_t n, int vec, int64_t *step, int64_t v)
{
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i0 == 0) *step = v;
    if (vec) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = i0; i < n / 4; i += stride) {
            reinterpret_cast<float4 *>(a)[i] = z;
            reinterpret_cast<float4 *>(b)[i] = z;
        }
    } else {
        for (int64_t i = i0; i < n; i += stride) {
            a[i] = 0.0f;
            b[i] = 0.0f;
        }
    }
}

// each shot's counter moves k steps, but never past its last step
__global__ void group_advance_kernel(GroupShot *shots, int n_shots, int k)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_shots; i += gridDim.x * blockDim.x) {
        int64_t *n = const_cast<int64_t *>(shots[i].prm.step_base);
        const int64_t v = *n + k;
        *n = v < shots[i].n_end ? v : shots[i].n_end;
    }
}

cudaError_t launch_group_advance(GroupShot *shots, int n_shots, int k, cudaStream_t s)
{
    if (n_shots <= 0) return cudaSuccess;
    group_advance_kernel<<<(n_shots + 127) / 128, 128, 0, s>>>(shots, n_shots, k);
    return cudaGetLastError();
}

// The per-step work of served migrations (GroupRtm), after the grouped sweep
// of step n = *step_base + step_off; blockIdx.y picks the shot from `list`.
// On most steps only the receiver rows are touched (record going forward,
// injection of the reversed traces going back); on the steps whose field is
// a snapshot time the blocks sweep the whole field, the receiver-row work of
// a row first, then the snapshot copy (forward) or the imaging condition
// (backward).  One warp per row (no index division per point), 16-byte
// accesses where the rows allow them.  The arithmetic is that of the single
// plan's record, injection and imaging kernels: a copy, u += 1 * trace, and
// img = fmaf(scale * s, u, img).
__global__ void group_rtm_kernel(const GroupShot *shots, const int *list, int step_off)
{
    const GroupShot &g = shots[list[blockIdx.y]];
    const int64_t n = *g.prm.step_base + step_off;
    if (n >= g.n_end) return;                           // uniform over the block
    const GroupRtm o = g.rtm;
    const int nx = g.prm.nx, ny = g.prm.ny, nz = g.prm.nz;
    const int64_t pitch = g.prm.pitch, plane = g.prm.plane;
    float *u = static_cast<float *>(g.buf[(int)((n + 1 + g.parity_base) & 1)]);   // u^{n+1}
    const int rows = o.y < 0 ? ny : 1;
    const int64_t per = (int64_t)rows * nx;             // elements of one trace step
    const bool fwd = o.phase == 1;
    const int64_t tb = o.T - n;                         // backward: forward time of the field after this step
    const bool field = fwd ? (n + 1) % o.k == 0 : (tb % o.k == 0 && tb >= o.k);
    const float inj_scale = 1.0f;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float *trace = o.traces + (fwd ? n : o.T - 1 - n) * per;   // this step's trace
    // one receiver row: record (u -> trace) or inject (u += trace)
    auto receiver_row = [&](float *ur, float *tr) {
        for (int x = lane; x < nx; x += 32) {
            if (fwd) tr[x] = ur[x];
            else ur[x] += inj_scale * tr[x];
        }
    };
    if (!field) {
        for (int64_t r = warp; r < rows; r += n_warps)
            receiver_row(u + o.z * plane + (int64_t)(o.y < 0 ? (int)r : o.y) * pitch, trace + r * nx);
        return;
    }
    const int64_t pts = (int64_t)nx * ny * nz, sl = fwd ? (n + 1) / o.k - 1 : tb / o.k - 1;
    float *snap = o.snaps + sl * pts;
    // snapshots and the image are dense (row r at r * nx); u is pitched
    const bool vec = (nx & 3) == 0 && (pitch & 3) == 0 && (reinterpret_cast<uintptr_t>(snap) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(o.image) & 15) == 0 && (reinterpret_cast<uintptr_t>(u) & 15) == 0;
    const int64_t all_rows = (int64_t)ny * nz;
    for (int64_t row = warp; row < all_rows; row += n_warps) {
        const int z = (int)(row / ny), y = (int)(row - (int64_t)z * ny);
        float *ur = u + row * pitch;
        float *sr = snap + row * nx;
        float *ir = o.image + row * nx;
        if (z == o.z && (o.y < 0 || y == o.y)) {
            receiver_row(ur, trace + (int64_t)(o.y < 0 ? y : 0) * nx);
            __syncwarp();                               // the imaging below reads the injected row
        }
        if (vec) {
            for (int x4 = lane; x4 < nx / 4; x4 += 32) {
                const float4 uv = reinterpret_cast<const float4 *>(ur)[x4];
                if (fwd) {
                    reinterpret_cast<float4 *>(sr)[x4] = uv;
                } else {
                    const float4 sv = reinterpret_cast<const float4 *>(sr)[x4];
                    float4 iv = reinterpret_cast<const float4 *>(ir)[x4];
                    iv.x = fmaf(o.image_scale * sv.x, uv.x, iv.x);
                    iv.y = fmaf(o.image_scale * sv.y, uv.y, iv.y);
                    iv.z = fmaf(o.image_scale * sv.z, uv.z, iv.z);
                    iv.w = fmaf(o.image_scale * sv.w, uv.w, iv.w);
                    reinterpret_cast<float4 *>(ir)[x4] = iv;
                }
            }
        } else {
            for (int x = lane; x < nx; x += 32) {
                if (fwd) sr[x] = ur[x];
                else ir[x] = fmaf(o.image_scale * sr[x], ur[x], ir[x]);
            }
        }
    }
}

cudaError_t launch_group_rtm(const GroupShot *shots, const int *list, int n_list, int step_off, cudaStream_t s)
{
    if (n_list <= 0) return cudaSuccess;
    group_rtm_kernel<<<dim3(152 * 8, n_list), 256, 0, s>>>(shots, list, step_off);
    return cudaGetLastError();
}

cudaError_t launch_clear_levels(float *a, float *b, int64_t n, int64_t *step, int64_t v, cudaStream_t s)
{
    const int vec = n % 4 == 0 && reinterpret_cast<uintptr_t>(a) % 16 == 0 && reinterpret_cast<uintptr_t>(b) % 16 == 0;
    const int64_t work = vec ? n / 4 : n;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
    clear_levels_kernel<<<blocks, 256, 0, s>>>(a, b, n, vec, step, v);
    return cudaGetLastError();
}

cudaError_t launch_set_step(int64_t *n, int64_t v, cudaStream_t s)
{
    set_step_kernel<<<1, 1, 0, s>>>(n, v);
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *n, int k, cudaStream_t s)
{
    advance_kernel<<<1, 1, 0, s>>>(n, k);
    return cudaGetLastError();
}

}  // namespace stencil

namespace stencil {

// ---------------------------------------------------------------------------
// Zero-lag cross-correlation imaging condition: img += scale * s * u over a
// dense (s, img) and a pitched u grid.  One warp per row (no index division
// per point), 16-byte accesses when every row of the three arrays starts on
// a 16-byte boundary.  HBM-bound: 16 B per point.
// ---------------------------------------------------------------------------
__global__ void image_accumulate_kernel(const float *s, const float *u, float *img, int nx, int64_t rows,
                                        int64_t pitch, float scale, int vec)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += n_warps) {
        const float *sr = s + row * nx;
        const float *ur = u + row * pitch;
        float *ir = img + row * nx;
        if (vec) {
            for (int x4 = lane; x4 < nx / 4; x4 += 32) {
                const float4 sv = reinterpret_cast<const float4 *>(sr)[x4];
                const float4 uv = reinterpret_cast<const float4 *>(ur)[x4];
                float4 iv = reinterpret_cast<const float4 *>(ir)[x4];
                iv.x = fmaf(scale * sv.x, uv.x, iv.x);
                iv.y = fmaf(scale * sv.y, uv.y, iv.y);
                iv.z = fmaf(scale * sv.z, uv.z, iv.z);
                iv.w = fmaf(scale * sv.w, uv.w, iv.w);
                reinterpret_cast<float4 *>(ir)[x4] = iv;
            }
        } else {
            for (int x = lane; x < nx; x += 32) ir[x] = fmaf(scale * sr[x], ur[x], ir[x]);
        }
    }
}

cudaError_t launch_image_accumulate(const float *s, const float *u, float *img, int nx, int ny, int nz,
                                    int64_t pitch, float scale, cudaStream_t st)
{
    const int64_t rows = (int64_t)ny * nz;
    const int64_t want = (rows + 7) / 8;                 // 8 warps a block, one row each per pass
    const int blocks = (int)std::min<int64_t>(want, 152 * 8);
    const int vec = (nx % 4 == 0) && (pitch % 4 == 0) && reinterpret_cast<uintptr_t>(s) % 16 == 0 &&
                    reinterpret_cast<uintptr_t>(u) % 16 == 0 && reinterpret_cast<uintptr_t>(img) % 16 == 0;
    image_accumulate_kernel<<<blocks, 256, 0, st>>>(s, u, img, nx, rows, pitch, scale, vec);
    return cudaGetLastError();
}

}  // namespace stencil
