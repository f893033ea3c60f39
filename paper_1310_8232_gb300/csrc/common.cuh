// Shared device-side definitions of libstencil: finite-difference weights,
// the wavelet, launch parameter blocks and the mbarrier / TMA wrappers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stencil {

// Device-side error bits, OR-ed into the plan's error word.
enum : int { ERR_TIMEOUT = 1, ERR_BAD_STATE = 2 };

// Exact central 2nd-difference weights of order 2R (Sec. 2, "10th order in
// space": R = 5; R = 4 also built), c_0..c_R as rationals num/den.  These
// make the symmetric stencil exact on polynomials of degree <= 2R+1; the
// paper prints no coefficients.
template <int R>
__host__ __device__ constexpr double wnum(int r);
template <int R>
__host__ __device__ constexpr double wden(int r);
template <>
__host__ __device__ constexpr double wnum<4>(int r)
{
    return r == 0 ? -205.0 : r == 1 ? 8.0 : r == 2 ? -1.0 : r == 3 ? 8.0 : -1.0;
}
template <>
__host__ __device__ constexpr double wden<4>(int r)
{
    return r == 0 ? 72.0 : r == 1 ? 5.0 : r == 2 ? 5.0 : r == 3 ? 315.0 : 560.0;
}
template <>
__host__ __device__ constexpr double wnum<5>(int r)
{
    return r == 0 ? -5269.0 : r == 1 ? 5.0 : r == 2 ? -5.0 : r == 3 ? 5.0 : r == 4 ? -5.0 : 1.0;
}
template <>
__host__ __device__ constexpr double wden<5>(int r)
{
    return r == 0 ? 1800.0 : r == 1 ? 3.0 : r == 2 ? 21.0 : r == 3 ? 126.0 : r == 4 ? 1008.0 : 3150.0;
}
template <int R>
__host__ __device__ constexpr float wf(int r) { return (float)(wnum<R>(r) / wden<R>(r)); }
template <int R>
__host__ __device__ constexpr double wd(int r) { return wnum<R>(r) / wden<R>(r); }

// Ricker wavelet of peak frequency f centred on t0, in FP64.
__device__ __forceinline__ double ricker(double f, double t0, double t)
{
    const double pi = 3.141592653589793238462643;
    const double a = pi * pi * f * f * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}

// Point source: u^{n+1}[s] += scale * w(n dt), scale = amp * v_s^2 dt^2.
struct Source {
    int32_t on;          // 0 = no source
    int32_t x, y, z;
    double scale;
    double f, t0, dt;
};

// Per-launch parameters of one sweep (one time step) over one grid.
struct SweepParams {
    int32_t nx, ny, nz;
    int64_t pitch;                 // row pitch, elements (same for the wavefields and kappa)
    int64_t plane;                 // pitch * ny
    const void *u;                 // u^n (FP32, or FP16/BF16 scaled per plane)
    void *up;                      // FP32: in u^{n-1}, out u^{n+1} (in place); 16-bit: out u^{n+1}
    const float *kappa;            // v^2 dt^2 / dx^2
    // reduced-precision storage only.  The state is (u^n, d^n) with the
    // difference d^n = u^n - u^{n-1} stored instead of u^{n-1}; d is updated
    // in place (in d^n, out d^{n+1}).  Per-plane power-of-two scales and
    // amax (float bit patterns) of each time level, slot = level mod 4, for
    // u (scale, amax) and for d (scale_d, amax_d).
    void *dv;                      // [field] d^n -> d^{n+1}
    float *scale;                  // [4][nz]
    unsigned *amax;                // [4][nz]
    float *scale_d;                // [4][nz]
    unsigned *amax_d;              // [4][nz]
    float growth;                  // kappa_max * 3W: bound on |kappa Lambda(u)| / max |u| over the star
    float src_bound;               // |source amplitude|, |w| <= 1
    int32_t zchunk;                // planes per thread block in z
    int32_t tiles_x;               // tiles along x (tiled kernel)
    Source src;
    const int64_t *step_base;      // device: n of the first step of this launch chunk
    int32_t step_off;              // this launch's offset within the chunk
    int *err;                      // device error word
    // energy of each step n -> n+1 (single-plan launches; off when
    // energy_on == 0): record index m = n - rec_n0, m < rec_cap
    double *energy;                // [rec_cap] E^{n+1/2}
    double *energy_part;           // [grid blocks] per-block partial of the step's energy
    unsigned *energy_count;        // blocks that have added their partial for the current step
    int64_t rec_n0;
    int32_t rec_cap;
    int32_t energy_on;
    // failure-path testing: limit of every shared-memory wait (0 = 2 s), and
    // extra bytes the first u copy of each block is expected to bring (> 0
    // makes that wait run out)
    uint32_t wait_ns;
    uint32_t fault_tx;
    // absorbing layer folded into the sweep (FP32 tiled kernel; 0 = none):
    // u^{n+1} = (plain update + eta u^{n-1}) / (1 + eta), eta = eta_max
    // ((W-d)/W)^2 at distance d < W from the nearest face, taken as
    // plain * g_d + u^{n-1} * h_d from the table absorb_tab[d] = (g_d, h_d) =
    // (1/(1+eta), eta/(1+eta)), d = 0..W (entry W = (1, 0)); then the source
    int32_t absorb_w;
    const float2 *absorb_tab;
};

// Widest absorbing layer: its damping table (W + 1 entries) is staged in
// shared memory by every block of the absorbing sweep.
constexpr int ABSORB_MAX_W = 255;

// Distance of coordinate a to the nearer face of [0, n), clamped to [0, W]
// (a outside the grid, such as a row's padding, gives 0: written, never read).
__device__ __forceinline__ int absorb_dist(int a, int n, int W) { return max(0, min(W, min(a, n - 1 - a))); }

// What a thread's 4 consecutive points (x = gx..gx+3) need of the layer for
// its whole z-march: their x distances, 16 bits each, and whether all four
// are at least W from both x faces.
struct AbsorbX {
    unsigned x01 = 0, x23 = 0;
    bool inner = true;
};
__device__ __forceinline__ AbsorbX absorb_x(int gx, int nx, int W)
{
    AbsorbX a;
    a.x01 = (unsigned)absorb_dist(gx, nx, W) | (unsigned)absorb_dist(gx + 1, nx, W) << 16;
    a.x23 = (unsigned)absorb_dist(gx + 2, nx, W) | (unsigned)absorb_dist(gx + 3, nx, W) << 16;
    a.inner = gx >= W && gx + 3 <= nx - 1 - W;
    return a;
}

// The same from the coordinates alone (point gx..gx+3 of row y, plane z),
// for kernels with no registers to spare for the distances above.
__device__ __forceinline__ void absorb4_at(int W, const float2 *tab, int nx, int ny, int nz, int gx, int y, int z,
                                           float4 &v, const float4 &prev)
{
    if (W <= 0) return;
    const int dyz = min(min(z, nz - 1 - z), min(y, ny - 1 - y));
    if (dyz >= W && gx >= W && gx + 3 <= nx - 1 - W) return;
    float *pv = &v.x;
    const float *pp = &prev.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int d = max(0, min(W, min(dyz, min(gx + j, nx - 1 - gx - j))));
        const float2 t = tab[d];
        pv[j] = fmaf(t.y, pp[j], pv[j] * t.x);
    }
}

// The layer on the 4 points of one row in one plane: dy = the row's clamped
// y distance, dz = the plane's z distance; d = min(x, y, z distances).
__device__ __forceinline__ void absorb4(int W, const float2 *tab, const AbsorbX &ax, int dy, int dz, float4 &v,
                                        const float4 &prev)
{
    if (W <= 0) return;                       // a shot without a layer in a grouped launch
    const int dyz = min(dy, dz);              // <= W: dy is clamped
    if (dyz >= W && ax.inner) return;
    const float2 t0 = tab[min(dyz, (int)(ax.x01 & 0xffffu))];
    const float2 t1 = tab[min(dyz, (int)(ax.x01 >> 16))];
    const float2 t2 = tab[min(dyz, (int)(ax.x23 & 0xffffu))];
    const float2 t3 = tab[min(dyz, (int)(ax.x23 >> 16))];
    v.x = fmaf(t0.y, prev.x, v.x * t0.x);
    v.y = fmaf(t1.y, prev.y, v.y * t1.x);
    v.z = fmaf(t2.y, prev.z, v.z * t2.x);
    v.w = fmaf(t3.y, prev.w, v.w * t3.x);
}

// The per-step work of a migration served in a group (reverse-time
// migration around the sweep: record and snapshots going forward, reversed
// injection and the imaging condition going back), done after each grouped
// sweep by group_rtm_kernel.  Each phase counts its steps from 0.
struct GroupRtm {
    int32_t phase;          // 0 none, 1 forward, 2 backward
    int32_t z, y;           // receiver plane and row (y < 0: every row)
    int32_t T, k;           // steps of each phase, snapshot interval (T a multiple of k)
    float image_scale;
    float *traces;          // [T][rows][nx]: recorded forward, injected reversed backward
    float *snaps;           // [T / k][nz][ny][nx]: u at forward times k, 2k, ..., T
    float *image;           // [nz][ny][nx]
};

// A shot of a grouped launch: its tensor maps (by parity of the level),
// buffers and parameters, in 64-byte aligned device memory.
struct alignas(64) GroupShot {
    CUtensorMap halo[2];           // u^n halo boxes, by which buffer holds u^n
    CUtensorMap core[2];           // FP32: u^{n-1} core boxes, by buffer; 16-bit: the d box (both)
    CUtensorMap kcore;             // kappa
    SweepParams prm;               // u, up are set per step from buf[]
    void *buf[2];
    int64_t n_end;                 // step counter value at which the shot stops
    int32_t parity_base;           // buffer of u^n = (n + parity_base) & 1
    int32_t pad;
    GroupRtm rtm;                  // a served migration's per-step work (phase 0: none)
};
struct GroupItem {
    int32_t shot, bx, by, z0, z1;
};

__device__ __forceinline__ int64_t current_step(const SweepParams &p)
{
    return *p.step_base + p.step_off;
}

// A kernel launched as a programmatic dependent of the previous one in its
// stream (cudaLaunchAttributeProgrammaticStreamSerialization) may start while
// that one drains; this waits until it has completed and its writes are
// visible.  Without the attribute it returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- PTX wrappers (mbarrier + TMA; sm_90 and later, used on sm_103a) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1/x to about one ulp (the hardware reciprocal; used for energy sums only)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity, giving up after
// `limit_ns` nanoseconds: then set ERR_TIMEOUT in *err and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err,
                                          uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Same, with an L2 cache-policy hint (createpolicy result).
__device__ __forceinline__ void tma_load_3d_hint(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                                 int y, int z, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}

// Make a tensor map that was (re)written in global memory visible to this
// thread's TMA copies.
__device__ __forceinline__ void fence_tensormap(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

}  // namespace stencil
