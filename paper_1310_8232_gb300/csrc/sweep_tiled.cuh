// K1 / K2: 2.5D-blocked sweep, one time step per launch; wavefields stored
// in FP32 (K1) or in FP16 / BF16 with a power-of-two scale per z plane and
// time level (K2); the arithmetic is FP32 either way.
//
// The GPU form of the paper's loop tiling (Sec. 3, Fig. 1b): instead of a
// cache blocksize (i, j, k) each thread block owns a TX x TY tile of the xy
// plane and marches through a chunk of z planes.  Per plane:
//   * one TMA box of u^n, (TX + 2 HX) x (TY + 2R), lands in a shared-memory
//     ring of SU stages (out-of-range coordinates are zero-filled by the TMA
//     unit, which is exactly the ghost-zero Dirichlet boundary);
//   * TMA boxes of u^{n-1} (16-bit storage: d^n, see below) and kappa
//     (TX x TY) land in a ring of SA stages;
//   * each thread owns 4 consecutive x points in each of 2 rows (the y
//     neighbours it loads serve both rows).  When plane p lands, the thread
//     reads its own values and its x and y neighbours (shared-memory
//     vectors) and immediately forms the partial sum of output plane p: x
//     and y terms, the z centre and the z terms of the R planes below p,
//     which it keeps in registers.  Plane p also adds its z term to the
//     partial sums of the R-1 outputs below it and completes output p-R,
//     which is then updated with u^{n-1} and kappa and written over u^{n-1}.
//     A u stage is therefore free again right after its plane has been read,
//     so shared memory holds copies in flight rather than planes waiting for
//     their turn, and a small footprint (4 stages) lets three blocks share an
//     SM;
//   * arithmetic runs two points at a time with packed FP32 instructions;
//     the register ring of (u, partial) pairs is rotated by unrolling.
// Thread 0 issues every copy right after the block barrier that ends each
// plane, into the stages that plane freed; "full" mbarriers (expect_tx)
// signal arrival.  Every wait is bounded: a stuck wait sets ERR_TIMEOUT and
// the whole block leaves at the next barrier, after the copies it issued
// have landed (also bounded).
//
// 16-bit storage (difference form): the state is u^n and the difference
// d^n = u^n - u^{n-1}, both in 16 bits; one step is
//     d^{n+1} = d^n + kappa Lambda(u^n) (+ source),   u^{n+1} = u^n + d^{n+1}
// in FP32, the same update as 2 u^n - u^{n-1} + kappa Lambda(u^n) in exact
// arithmetic.  Storing d instead of u^{n-1} keeps the step-to-step change at
// the format's full relative precision: with u^{n-1} stored, the difference
// u^n - u^{n-1} (a few per cent of u where the wave is slow against dx/dt)
// keeps only the few low bits that survive the cancellation, and each
// rounding of u then acts as a velocity kick that the scheme integrates.
// u^{n+1} goes to the second u buffer (its neighbours still read u^n), d is
// rewritten in place.  A stored value h of plane z at level n means h *
// s_n[z], s a power of two (so scaling is exact), one scale table for u and
// one for d.  The scales of each output plane are fixed before anything is
// written, from bounds every block computes the same way:
//     |d^{n+1}| <= max|d^n| at z + kappa_max 3W max|u^n| over planes z-R..z+R
//                  (+ the source amplitude on the source plane),
//     |u^{n+1}| <= max|u^n| at z + that bound,
// and the stored magnitudes are kept below 2^15.  Each block reduces
// max|u^{n+1}| and max|d^{n+1}| of its tile per plane and merges them with
// one atomicMax each.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"

namespace stencil {

// ---- element access ----------------------------------------------------------------
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ld4(const __half *p)
{
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p)
{
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float *p, const float4 &v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st4(__half *p, const float4 &v)
{
    const __half2 a = __floats2half2_rn(v.x, v.y);
    const __half2 b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&a);
    u.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void st4(__nv_bfloat16 *p, const float4 &v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&a);
    u.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

// Smallest power of two s >= 2^-126 with b / s <= 2^15 (1 for b == 0), and
// its reciprocal (exact: also a power of two).
__device__ __forceinline__ void pow2_scale(float b, float &s, float &inv)
{
    int k = 0;                     // s = 2^k
    if (b > 0.0f) {
        if (isinf(b)) {
            k = 127;
        } else {
            int e;
            frexpf(b, &e);         // b = f * 2^e, f in [0.5, 1): b < 2^e
            k = max(e - 15, -126);
        }
    }
    s = ldexpf(1.0f, k);
    inv = ldexpf(1.0f, -k);
}

template <int R, int TX, int TY, typename E>
struct TiledShape {
    static constexpr bool F32 = std::is_same<E, float>::value;
    static constexpr int ES = sizeof(E);
    static constexpr int HX = F32 ? ((R + 3) / 4) * 4 : 8;   // x halo rounded to 16 bytes
    static constexpr int BW = TX + 2 * HX;              // u box width
    static constexpr int BH = TY + 2 * R;               // u box height
    static constexpr int TPR = TX / 4;                  // threads per row
    static constexpr int ROWS = 2;                      // rows per thread
    static constexpr int NT = TPR * TY / ROWS;          // threads per block
    static constexpr int RING = R + 1;                  // register ring of (u, partial) per plane
    // ring slot chosen at run time (16-bit: the unrolled body outgrows the
    // instruction cache); FP32 keeps the fully unrolled ring
    static constexpr bool SPLIT = !F32;
    static constexpr int SU = 4;                        // u stages: 1 being read + 3 in flight
    static constexpr int SA = 4;                        // u_prev / kappa stages
    static constexpr int ZMAX = F32 ? 0 : 256;          // largest z-chunk (16-bit: scale tables)
    static constexpr uint32_t U_BYTES = BW * BH * ES;
    static constexpr uint32_t P_BYTES = TX * TY * ES;
    static constexpr uint32_t K_BYTES = TX * TY * 4;
    static constexpr int U_STAGE = ((U_BYTES + 127) / 128) * 128;
    static constexpr int P_STAGE = ((P_BYTES + 127) / 128) * 128;
    static constexpr int K_STAGE = K_BYTES;
    static constexpr int P_OFF = SU * U_STAGE;
    static constexpr int K_OFF = P_OFF + SA * P_STAGE;
    static constexpr int SIG_OFF = K_OFF + SA * K_STAGE;
    // 16-bit: u scales of the planes entering the ring, d scales of the
    // outputs' level n, reciprocal u and d scales of the outputs' level n+1,
    // plus per-warp maxima of u and d (double-buffered by plane parity)
    static constexpr int SIG_BYTES = F32 ? 0 : ((ZMAX + 2 * R) + 3 * ZMAX + 4 * (NT / 32)) * 4;
    static constexpr int BAR_OFF = ((SIG_OFF + SIG_BYTES + 15) / 16) * 16;
    static constexpr int EN_OFF = BAR_OFF + (SU + SA) * 8;     // per-warp FP64 energy sums
    static constexpr int FLAG_OFF = EN_OFF + (NT / 32) * 8;
    static constexpr int SMEM = FLAG_OFF + 16;
    static_assert(TX % 32 == 0 && TX >= 32 && BW <= 256 && BH <= 256, "TMA box limits");
    static_assert(TY % ROWS == 0, "whole thread rows");
    static constexpr bool VALID = NT <= 1024 && NT % 32 == 0;
    // blocks per SM the register allocation is held to: three 128-thread
    // blocks per SM are what keep enough planes in flight (<= 170 registers)
    static constexpr int MINB = NT == 128 ? 3 : 1;
};

// compile-time loop: f(integral_constant<K>) for K = 0..N-1
template <int K, int N>
struct Unroll {
    template <class F>
    __device__ __forceinline__ static void run(F &f)
    {
        f(std::integral_constant<int, K>{});
        Unroll<K + 1, N>::run(f);
    }
};
template <int N>
struct Unroll<N, N> {
    template <class F>
    __device__ __forceinline__ static void run(F &)
    {
    }
};

// run-time index k -> f(integral_constant<K>) for the K == k, K = 0..N-1
template <int N, class F>
__device__ __forceinline__ void dispatch(int k, F &f)
{
    static_assert(N >= 1 && N <= 6, "ring sizes 1 .. 6");
    switch (k) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: if constexpr (N > 1) f(std::integral_constant<int, 1>{}); break;
    case 2: if constexpr (N > 2) f(std::integral_constant<int, 2>{}); break;
    case 3: if constexpr (N > 3) f(std::integral_constant<int, 3>{}); break;
    case 4: if constexpr (N > 4) f(std::integral_constant<int, 4>{}); break;
    default: if constexpr (N > 5) f(std::integral_constant<int, 5>{}); break;
    }
}

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
// 1 / (kappa + FLT_MIN) for two points (the hardware reciprocal; energy sums
// only).  The packed add leaves every kappa >= 2^-100 unchanged and keeps
// the reciprocal finite where kappa is the zero fill outside the grid (there
// u^{n+1} - u^n = 0, so the term is 0, not NaN).
__device__ __forceinline__ float2 rcp_kappa2(const float2 &k)
{
    const float2 kk = __fadd2_rn(k, make_float2(1.17549435e-38f, 1.17549435e-38f));
    return make_float2(rcp_approx(kk.x), rcp_approx(kk.y));
}
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 scale4(const float4 &v, float s)
{
    const float2 ss = make_float2(s, s);
    const float2 a = __fmul2_rn(lo2(v), ss);
    const float2 b = __fmul2_rn(hi2(v), ss);
    return make_float4(a.x, a.y, b.x, b.y);
}

// One block's work: tile (bx, by) of the xy plane, output planes [z0, z1)
// of one shot, at time level n.  map_* are the shot's tensor maps (kernel
// parameters or 64-byte aligned global memory).
// ABS_HOIST: with the layer, keep the thread's distances to the faces in
// registers for the whole z-march (the single-shot kernel) or recompute them
// per point (the grouped kernel, which has no registers to spare).
template <int R, int TX, int TY, typename E, bool REC, bool ABS = false, bool ABS_HOIST = true>
__device__ __forceinline__ void sweep_tile(const CUtensorMap *map_u, const CUtensorMap *map_up,
                                           const CUtensorMap *map_k, const SweepParams &params, int bx, int by,
                                           int z0, int z1, int64_t n_level, unsigned char *smem)
{
    using S = TiledShape<R, TX, TY, E>;
    static_assert(!ABS || (S::F32 && !REC), "the folded absorbing layer is an FP32 variant without the energy");
    constexpr bool SPLIT = S::SPLIT;
    // a private copy: the inline-asm waits and copies clobber memory, which
    // would otherwise force every field to be reloaded after each of them
    const SweepParams p = params;
    unsigned char *su = smem;
    unsigned char *sp = smem + S::P_OFF;
    unsigned char *sk = smem + S::K_OFF;
    float *sig_in = reinterpret_cast<float *>(smem + S::SIG_OFF);   // [ZMAX + 2R]: u scale, level n, planes pz0 + j
    float *sig_dn = sig_in + (S::ZMAX + 2 * R);                      // [ZMAX]: d scale, level n, outputs z0 + j
    float *inv_u = sig_dn + S::ZMAX;                                 // [ZMAX]: 1 / u scale, level n+1, outputs
    float *inv_d = inv_u + S::ZMAX;                                  // [ZMAX]: 1 / d scale, level n+1, outputs
    unsigned *wmax = reinterpret_cast<unsigned *>(inv_d + S::ZMAX);  // [2 parities][u, d][NT/32]
    uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);
    uint64_t *full_a = full_u + S::SU;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + S::FLAG_OFF);

    const uint64_t wait_limit = p.wait_ns ? p.wait_ns : 2000000000ull;
    const int tid = threadIdx.x;
    const int x0 = bx * TX;
    const int y0 = by * TY;
    double *en_warp = reinterpret_cast<double *>(smem + S::EN_OFF);   // per-warp energy sums
    if (REC && tid < S::NT / 32) en_warp[tid] = 0.0;
    if (z0 >= z1) return;                     // uniform over the block
    const int nout = z1 - z0;                 // output planes
    const int nin = nout + 2 * R;             // planes through the ring: z0-R .. z1+R-1
    const int pz0 = z0 - R;

    auto issue_u = [&](int t) {               // plane pz0 + t into stage t % SU
        const int st = t % S::SU;
        mbar_arrive_expect_tx(&full_u[st], S::U_BYTES + (t == 0 ? p.fault_tx : 0u));
        tma_load_3d(su + st * S::U_STAGE, map_u, &full_u[st], x0 - S::HX, y0 - R, pz0 + t);
    };
    auto issue_a = [&](int ja) {              // u^{n-1} and kappa of output z0 + ja into stage ja % SA
        const int st = ja % S::SA;
        mbar_arrive_expect_tx(&full_a[st], S::P_BYTES + S::K_BYTES);
        tma_load_3d(sp + st * S::P_STAGE, map_up, &full_a[st], x0, y0, z0 + ja);
        tma_load_3d(sk + st * S::K_STAGE, map_k, &full_a[st], x0, y0, z0 + ja);
    };

    if (tid == 0) {
        for (int i = 0; i < S::SU; ++i) mbar_init(&full_u[i], 1);
        for (int i = 0; i < S::SA; ++i) mbar_init(&full_a[i], 1);
        *abort_flag = 0;
        fence_barrier_init();
        for (int t = 0; t < S::SU && t < nin; ++t) issue_u(t);
        for (int ja = 0; ja < S::SA && ja < nout; ++ja) issue_a(ja);
    }
    int slot_out = 0;                         // 16-bit: slot of level n+1 in the scale / amax tables
    if constexpr (!S::F32) {
        // scales of this block's planes, and those of its outputs (every block
        // computes the same value; tile 0 of each z-chunk publishes them)
        const int64_t n = n_level;
        const int s_n = (int)(n & 3);
        slot_out = (int)((n + 1) & 3);
        const int s_clear = (int)((n + 2) & 3);
        const float *scale_n = p.scale + (int64_t)s_n * p.nz;
        const float *scale_dn = p.scale_d + (int64_t)s_n * p.nz;
        const unsigned *amax_n = p.amax + (int64_t)s_n * p.nz;
        const unsigned *amax_dn = p.amax_d + (int64_t)s_n * p.nz;
        for (int j = tid; j < nin; j += S::NT) {
            const int z = pz0 + j;
            sig_in[j] = (z >= 0 && z < p.nz) ? scale_n[z] : 1.0f;
        }
        for (int j = tid; j < nout; j += S::NT) {
            const int o = z0 + j;
            sig_dn[j] = scale_dn[o];
            float m = 0.0f;
            for (int d = -R; d <= R; ++d)
                if (o + d >= 0 && o + d < p.nz) m = fmaxf(m, __uint_as_float(amax_n[o + d]));
            float bd = p.growth * m + __uint_as_float(amax_dn[o]);
            if (p.src.on && o == p.src.z) bd += p.src_bound;
            const float bu = __uint_as_float(amax_n[o]) + bd;
            float su, sd;
            pow2_scale(bu, su, inv_u[j]);
            pow2_scale(bd, sd, inv_d[j]);
            if (bx == 0 && by == 0) {
                p.scale[(int64_t)slot_out * p.nz + o] = su;
                p.scale_d[(int64_t)slot_out * p.nz + o] = sd;
            }
        }
        // level n-2's slots become level n+2's: clear them for the next step
        if (bx == 0 && by == 0 && z0 == 0)
            for (int z = tid; z < p.nz; z += S::NT) {
                p.amax[(int64_t)s_clear * p.nz + z] = 0u;
                p.amax_d[(int64_t)s_clear * p.nz + z] = 0u;
            }
    }
    __syncthreads();

    const int tx4 = tid % S::TPR;
    const int ty0 = (tid / S::TPR) * S::ROWS;              // first of this thread's rows
    const int gx = x0 + 4 * tx4;
    const int gy0 = y0 + ty0;
    const bool x_ok = gx < p.nx;
    const int own = (R + ty0) * S::BW + S::HX + 4 * tx4;   // own 4 points of row 0 in a u stage (elements)
    const int own_a = ty0 * TX + 4 * tx4;
    E *dst = static_cast<E *>(p.up) + (int64_t)gy0 * p.pitch + gx;          // u^{n+1}
    E *dst_d = S::F32 ? nullptr : static_cast<E *>(p.dv) + (int64_t)gy0 * p.pitch + gx;   // 16-bit: d^{n+1}
    const int src_row = p.src.y - gy0;                     // this thread's row holding the source, if any
    const bool src_here = p.src.on && (unsigned)src_row < (unsigned)S::ROWS && (unsigned)(p.src.x - gx) < 4u &&
                          p.src.z >= z0 && p.src.z < z1;
    // the source term of this step, w(n dt) scaled (one value for the whole
    // launch: evaluated once, outside the unrolled plane loop)
    float src_add = 0.0f;
    if (src_here) src_add = (float)(p.src.scale * ricker(p.src.f, p.src.t0, (double)n_level * p.src.dt));

    // ABS: the layer's damping table in shared memory, the x distances of the
    // thread's points and the y distances of its rows (fixed for the whole
    // z-march)
    AbsorbX abs_x;
    int abs_dy[S::ROWS];
    __shared__ float2 abs_tab[ABS ? ABSORB_MAX_W + 1 : 1];
    if constexpr (ABS) {
        if (p.absorb_w > 0)                   // a shot of a grouped launch may have none
            for (int j = tid; j <= p.absorb_w; j += S::NT) abs_tab[j] = p.absorb_tab[j];
        __syncthreads();
        if constexpr (ABS_HOIST) {
            abs_x = absorb_x(gx, p.nx, p.absorb_w);
#pragma unroll
            for (int h = 0; h < S::ROWS; ++h) abs_dy[h] = absorb_dist(gy0 + h, p.ny, p.absorb_w);
        }
    }

    // ring slot j holds, per row, plane i's u values and output i's partial
    // sum for the planes i with i mod RING == j (i counts planes from z0 - R)
    float4 uq[S::ROWS][S::RING];
    float2 pa[S::ROWS][S::RING], pb[S::ROWS][S::RING];
#pragma unroll
    for (int h = 0; h < S::ROWS; ++h)
#pragma unroll
        for (int j = 0; j < S::RING; ++j) {
            uq[h][j] = make_float4(0.f, 0.f, 0.f, 0.f);
            pa[h][j] = make_float2(0.f, 0.f);
            pb[h][j] = make_float2(0.f, 0.f);
        }

    const float2 two = make_float2(2.0f, 2.0f);
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float2 c0x3 = make_float2(3.0f * wf<R>(0), 3.0f * wf<R>(0));
    int done = 0;                           // planes fully processed (block-uniform)
    // REC: this thread's energy terms, FP32 over each group of RING planes,
    // then FP64 over the z-chunk; one warp sum at the end.  Points outside the
    // grid add exactly zero: their u^{n+1} and u^n are zero (zero-filled
    // inputs, kappa = 0 there), and 1/kappa is taken of kappa + FLT_MIN,
    // which keeps 0 * (1/kappa) finite, so no point needs a mask.
    double eacc = 0.0;

    if constexpr (!SPLIT) {
        // FP32 storage: the ring rotated by unrolling over its R+1 slots
        static_assert(S::F32, "the unrolled ring loop is the FP32 path");
        int su_stage = 0, su_phase = 0;     // stage / parity of plane i
        int sa_stage = 0, sa_phase = 0;     // aux stage / parity of output ja = i - 2R
        for (int i0 = 0; i0 < nin; i0 += S::RING) {
            float2 ekin = make_float2(0.f, 0.f);    // REC: energy terms of this group of RING planes
            float2 epot = make_float2(0.f, 0.f);
            auto body = [&](auto kc) {
                constexpr int K = decltype(kc)::value;          // slot of plane i
                const int i = i0 + K;
                if (i >= nin) return;                           // block-uniform
                if (!mbar_wait(&full_u[su_stage], su_phase, p.err, wait_limit)) *abort_flag = 1;
                const E *pl = reinterpret_cast<const E *>(su + su_stage * S::U_STAGE) + own;
                // column of the thread's x group: rows -R .. ROWS-1+R around row 0
                float4 col[S::ROWS + 2 * R];
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) col[R + h] = ld4(pl + h * S::BW);
                float2 nA[S::ROWS], nB[S::ROWS];
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    nA[h] = make_float2(0.f, 0.f);
                    nB[h] = make_float2(0.f, 0.f);
                }
                if (i >= R && i < R + nout) {
                    // partial sums of output plane i: centre, x, y, and z below
#pragma unroll
                    for (int r = 1; r <= R; ++r) {
                        col[R - r] = ld4(pl - r * S::BW);
                        col[R + S::ROWS - 1 + r] = ld4(pl + (S::ROWS - 1 + r) * S::BW);
                    }
#pragma unroll
                    for (int h = 0; h < S::ROWS; ++h) {
                        const E *ph = pl + h * S::BW;
                        const float4 c = col[R + h];
                        float2 aA = __fmul2_rn(c0x3, lo2(c));
                        float2 aB = __fmul2_rn(c0x3, hi2(c));
                        // row[m] = u[gx - 8 + m], m = 0..19; own points are m = 8..11
                        float row[20];
                        {
                            const float4 l1 = ld4(ph - 4);
                            const float4 r1 = ld4(ph + 4);
                            row[4] = l1.x; row[5] = l1.y; row[6] = l1.z; row[7] = l1.w;
                            row[8] = c.x; row[9] = c.y; row[10] = c.z; row[11] = c.w;
                            row[12] = r1.x; row[13] = r1.y; row[14] = r1.z; row[15] = r1.w;
                            if constexpr (R > 4) {
                                const float4 l2 = ld4(ph - 8);
                                const float4 r2 = ld4(ph + 8);
                                row[0] = l2.x; row[1] = l2.y; row[2] = l2.z; row[3] = l2.w;
                                row[16] = r2.x; row[17] = r2.y; row[18] = r2.z; row[19] = r2.w;
                            } else {
                                row[0] = row[1] = row[2] = row[3] = 0.f;
                                row[16] = row[17] = row[18] = row[19] = 0.f;
                            }
                        }
#pragma unroll
                        for (int r = 1; r <= R; ++r) {
                            const float4 ym = col[R + h - r];
                            const float4 yp = col[R + h + r];
                            const float4 zm = uq[h][(K + S::RING - r) % S::RING];   // plane i - r (true values)
                            float2 sA, sB;
                            if (r % 2 == 0) {
                                sA = __fadd2_rn(make_float2(row[8 - r], row[9 - r]),
                                                make_float2(row[8 + r], row[9 + r]));
                                sB = __fadd2_rn(make_float2(row[10 - r], row[11 - r]),
                                                make_float2(row[10 + r], row[11 + r]));
                            } else {
                                // odd shifts pair values across register pairs: add them singly
                                sA = make_float2(row[8 - r] + row[8 + r], row[9 - r] + row[9 + r]);
                                sB = make_float2(row[10 - r] + row[10 + r], row[11 - r] + row[11 + r]);
                            }
                            sA = __fadd2_rn(sA, __fadd2_rn(lo2(ym), lo2(yp)));
                            sB = __fadd2_rn(sB, __fadd2_rn(hi2(ym), hi2(yp)));
                            const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                            sA = __fadd2_rn(sA, lo2(zm));
                            sB = __fadd2_rn(sB, hi2(zm));
                            aA = __ffma2_rn(cr, sA, aA);
                            aB = __ffma2_rn(cr, sB, aB);
                        }
                        nA[h] = aA;
                        nB[h] = aB;
                    }
                }
                if (++su_stage == S::SU) {
                    su_stage = 0;
                    su_phase ^= 1;
                }
                // plane i is the z neighbour above outputs i-1 .. i-(R-1)
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    const float4 c = col[R + h];
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                        pa[h][(K + S::RING - r) % S::RING] = __ffma2_rn(cr, lo2(c), pa[h][(K + S::RING - r) % S::RING]);
                        pb[h][(K + S::RING - r) % S::RING] = __ffma2_rn(cr, hi2(c), pb[h][(K + S::RING - r) % S::RING]);
                    }
                }
                if (i >= 2 * R) {
                    // ... and the last one above output i - R, which is now complete
                    constexpr int KF = (K + 1) % S::RING;             // slot of plane i - R
                    const float2 cR = make_float2(wf<R>(R), wf<R>(R));
                    const int ja = i - 2 * R;
                    if (!mbar_wait(&full_a[sa_stage], sa_phase, p.err, wait_limit)) *abort_flag = 1;
                    float4 prev[S::ROWS], kap[S::ROWS];
#pragma unroll
                    for (int h = 0; h < S::ROWS; ++h) {
                        prev[h] = ld4(reinterpret_cast<const E *>(sp + sa_stage * S::P_STAGE) + own_a + h * TX);
                        kap[h] = ld4(reinterpret_cast<const float *>(sk + sa_stage * S::K_STAGE) + own_a + h * TX);
                    }
                    if (++sa_stage == S::SA) {
                        sa_stage = 0;
                        sa_phase ^= 1;
                    }
                    const int o = z0 + ja;
#pragma unroll
                    for (int h = 0; h < S::ROWS; ++h) {
                        const float4 c = col[R + h];
                        const float2 fA = __ffma2_rn(cR, lo2(c), pa[h][KF]);
                        const float2 fB = __ffma2_rn(cR, hi2(c), pb[h][KF]);
                        const float4 cc = uq[h][KF];
                        // u^{n+1} = kappa * Lambda + (2 u^n - u^{n-1})
                        const float2 oA =
                            __ffma2_rn(lo2(kap[h]), fA, __ffma2_rn(neg1, lo2(prev[h]), __fmul2_rn(two, lo2(cc))));
                        const float2 oB =
                            __ffma2_rn(hi2(kap[h]), fB, __ffma2_rn(neg1, hi2(prev[h]), __fmul2_rn(two, hi2(cc))));
                        float4 nxt = make_float4(oA.x, oA.y, oB.x, oB.y);
                        if constexpr (ABS) {
                            if constexpr (ABS_HOIST)
                                absorb4(p.absorb_w, abs_tab, abs_x, abs_dy[h], min(o, p.nz - 1 - o), nxt, prev[h]);
                            else
                                absorb4_at(p.absorb_w, abs_tab, p.nx, p.ny, p.nz, gx, gy0 + h, o, nxt, prev[h]);
                        }
                        if (src_here && src_row == h && o == p.src.z) {
                            const int k = p.src.x - gx;
                            if (k == 0) nxt.x += src_add;
                            else if (k == 1) nxt.y += src_add;
                            else if (k == 2) nxt.z += src_add;
                            else nxt.w += src_add;
                        }
                        if (REC) {
                            // E^{n+1/2} terms (u^{n+1} - u^n)^2 / kappa (into ekin) and
                            // u^{n+1} Lambda(u^n) (into epot)
                            const float2 uA = lo2(nxt), uB = hi2(nxt);
                            const float2 dA = __ffma2_rn(neg1, lo2(cc), uA);
                            const float2 dB = __ffma2_rn(neg1, hi2(cc), uB);
                            ekin = __ffma2_rn(__fmul2_rn(dA, dA), rcp_kappa2(lo2(kap[h])), ekin);
                            ekin = __ffma2_rn(__fmul2_rn(dB, dB), rcp_kappa2(hi2(kap[h])), ekin);
                            epot = __ffma2_rn(uA, fA, epot);
                            epot = __ffma2_rn(uB, fB, epot);
                        }
                        if (x_ok && gy0 + h < p.ny) st4(dst + (int64_t)h * p.pitch + (int64_t)o * p.plane, nxt);
                    }
                }
                // slot K held plane i - R - 1, which nothing needs any more
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    uq[h][K] = col[R + h];
                    pa[h][K] = nA[h];
                    pb[h][K] = nB[h];
                }
                // every thread is done with plane i's u stage and output (i-2R)'s
                // aux stage: refill them
                __syncthreads();
                done = i + 1;
                if (*abort_flag) {
                    i0 = nin;                                    // block-uniform exit
                    return;
                }
                if (tid == 0) {
                    if (i + S::SU < nin) issue_u(i + S::SU);
                    if (i >= 2 * R && i - 2 * R + S::SA < nout) issue_a(i - 2 * R + S::SA);
                }
            };
            Unroll<0, S::RING>::run(body);
            if (REC) eacc += (double)((ekin.x + ekin.y) - (epot.x + epot.y));
        }
    } else {
        // The same per-plane work with the ring slot chosen at run time.  The
        // shared-memory reads, the 16-bit conversions and the centre, x and y
        // sums do not depend on the slot and are emitted once; only the parts
        // that name ring registers (z terms, the completed output, the ring
        // store) are instantiated per slot.  The loop body stays a fraction
        // of the fully unrolled one, which keeps the instruction fetch ahead.
        static_assert(!S::F32, "the dispatched ring loop is the 16-bit difference-form path");
        float2 ekin = make_float2(0.f, 0.f);        // REC: energy terms of the current group of RING planes
        float2 epot = make_float2(0.f, 0.f);
        int k = 0;                                  // ring slot of plane i (i mod RING)
        static_assert(S::SU == 4 && S::SA == 4, "stage and parity from the plane index bits");
        for (int i = 0; i < nin; ++i) {
            if (!mbar_wait(&full_u[i & 3], (i >> 2) & 1, p.err, wait_limit)) *abort_flag = 1;
            const E *pl = reinterpret_cast<const E *>(su + (i & 3) * S::U_STAGE) + own;
            const float sgi = sig_in[i];
            float4 col[S::ROWS + 2 * R];
#pragma unroll
            for (int h = 0; h < S::ROWS; ++h) col[R + h] = ld4(pl + h * S::BW);
            const bool has_out = i >= R && i < R + nout;
            float2 xA[S::ROWS], xB[S::ROWS];        // centre, x and y terms of output i (stored units)
            if (has_out) {
#pragma unroll
                for (int r = 1; r <= R; ++r) {
                    col[R - r] = ld4(pl - r * S::BW);
                    col[R + S::ROWS - 1 + r] = ld4(pl + (S::ROWS - 1 + r) * S::BW);
                }
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    const E *ph = pl + h * S::BW;
                    const float4 c = col[R + h];
                    float2 aA = __fmul2_rn(c0x3, lo2(c));
                    float2 aB = __fmul2_rn(c0x3, hi2(c));
                    float row[20];                  // row[m] = u[gx - 8 + m]; own points m = 8..11
                    {
                        const float4 l1 = ld4(ph - 4);
                        const float4 r1 = ld4(ph + 4);
                        row[4] = l1.x; row[5] = l1.y; row[6] = l1.z; row[7] = l1.w;
                        row[8] = c.x; row[9] = c.y; row[10] = c.z; row[11] = c.w;
                        row[12] = r1.x; row[13] = r1.y; row[14] = r1.z; row[15] = r1.w;
                        if constexpr (R > 4) {
                            const float4 l2 = ld4(ph - 8);
                            const float4 r2 = ld4(ph + 8);
                            row[0] = l2.x; row[1] = l2.y; row[2] = l2.z; row[3] = l2.w;
                            row[16] = r2.x; row[17] = r2.y; row[18] = r2.z; row[19] = r2.w;
                        } else {
                            row[0] = row[1] = row[2] = row[3] = 0.f;
                            row[16] = row[17] = row[18] = row[19] = 0.f;
                        }
                    }
#pragma unroll
                    for (int r = 1; r <= R; ++r) {
                        const float4 ym = col[R + h - r];
                        const float4 yp = col[R + h + r];
                        float2 sA, sB;
                        if (r % 2 == 0) {
                            sA = __fadd2_rn(make_float2(row[8 - r], row[9 - r]), make_float2(row[8 + r], row[9 + r]));
                            sB = __fadd2_rn(make_float2(row[10 - r], row[11 - r]),
                                            make_float2(row[10 + r], row[11 + r]));
                        } else {
                            // odd shifts pair values across register pairs: add them singly
                            sA = make_float2(row[8 - r] + row[8 + r], row[9 - r] + row[9 + r]);
                            sB = make_float2(row[10 - r] + row[10 + r], row[11 - r] + row[11 + r]);
                        }
                        sA = __fadd2_rn(sA, __fadd2_rn(lo2(ym), lo2(yp)));
                        sB = __fadd2_rn(sB, __fadd2_rn(hi2(ym), hi2(yp)));
                        const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                        aA = __ffma2_rn(cr, sA, aA);
                        aB = __ffma2_rn(cr, sB, aB);
                    }
                    xA[h] = aA;
                    xB[h] = aB;
                }
            }
#pragma unroll
            for (int h = 0; h < S::ROWS; ++h) col[R + h] = scale4(col[R + h], sgi);
            // d^n and kappa of output i - R, completed by this plane
            const bool fin = i >= 2 * R;
            const E *aux_d = nullptr;
            const float *aux_k = nullptr;
            float sgd = 1.0f, iu = 1.0f, id = 1.0f;
            int o = 0;
            if (fin) {
                const int ja = i - 2 * R;
                if (!mbar_wait(&full_a[ja & 3], (ja >> 2) & 1, p.err, wait_limit)) *abort_flag = 1;
                aux_d = reinterpret_cast<const E *>(sp + (ja & 3) * S::P_STAGE) + own_a;
                aux_k = reinterpret_cast<const float *>(sk + (ja & 3) * S::K_STAGE) + own_a;
                sgd = sig_dn[ja];
                iu = inv_u[ja];
                id = inv_d[ja];
                o = z0 + ja;
            }
            const bool src_plane = src_here && o == p.src.z && fin;   // this thread adds the source now
            float umax = 0.0f, dmax = 0.0f;
            auto ring = [&](auto kc) {
                constexpr int K = decltype(kc)::value;          // slot of plane i
                constexpr int KF = (K + 1) % S::RING;           // slot of plane i - R
                const float2 ss = make_float2(sgi, sgi);
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    // plane i is the z neighbour above outputs i-1 .. i-(R-1)
                    const float4 c = col[R + h];
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                        pa[h][(K + S::RING - r) % S::RING] =
                            __ffma2_rn(cr, lo2(c), pa[h][(K + S::RING - r) % S::RING]);
                        pb[h][(K + S::RING - r) % S::RING] =
                            __ffma2_rn(cr, hi2(c), pb[h][(K + S::RING - r) % S::RING]);
                    }
                    if (fin) {
                        // ... and the last one above output i - R, which is now complete
                        const float2 cR = make_float2(wf<R>(R), wf<R>(R));
                        const float2 fA = __ffma2_rn(cR, lo2(c), pa[h][KF]);
                        const float2 fB = __ffma2_rn(cR, hi2(c), pb[h][KF]);
                        const float4 cc = uq[h][KF];                      // u^n
                        const float4 dn = scale4(ld4(aux_d + h * TX), sgd);   // d^n
                        const float4 kap = ld4(aux_k + h * TX);
                        // d^{n+1} = d^n + kappa * Lambda (+ source), u^{n+1} = u^n + d^{n+1}
                        const float2 eA = __ffma2_rn(lo2(kap), fA, lo2(dn));
                        const float2 eB = __ffma2_rn(hi2(kap), fB, hi2(dn));
                        float4 dnx = make_float4(eA.x, eA.y, eB.x, eB.y);
                        if (src_plane && src_row == h) {
                            const int q = p.src.x - gx;
                            if (q == 0) dnx.x += src_add;
                            else if (q == 1) dnx.y += src_add;
                            else if (q == 2) dnx.z += src_add;
                            else dnx.w += src_add;
                        }
                        const float2 oA = __fadd2_rn(lo2(cc), lo2(dnx));
                        const float2 oB = __fadd2_rn(hi2(cc), hi2(dnx));
                        const float4 nxt = make_float4(oA.x, oA.y, oB.x, oB.y);
                        const bool ok = x_ok && gy0 + h < p.ny;
                        if (REC) {
                            // (u^{n+1} - u^n) = d^{n+1}: its square over kappa, and u^{n+1} Lambda(u^n)
                            const float2 dA = lo2(dnx), dB = hi2(dnx);
                            ekin = __ffma2_rn(__fmul2_rn(dA, dA), rcp_kappa2(lo2(kap)), ekin);
                            ekin = __ffma2_rn(__fmul2_rn(dB, dB), rcp_kappa2(hi2(kap)), ekin);
                            epot = __ffma2_rn(lo2(nxt), fA, epot);
                            epot = __ffma2_rn(hi2(nxt), fB, epot);
                        }
                        const float mu = fmaxf(fmaxf(fabsf(nxt.x), fabsf(nxt.y)), fmaxf(fabsf(nxt.z), fabsf(nxt.w)));
                        const float md = fmaxf(fmaxf(fabsf(dnx.x), fabsf(dnx.y)), fmaxf(fabsf(dnx.z), fabsf(dnx.w)));
                        umax = fmaxf(umax, ok ? mu : 0.0f);
                        dmax = fmaxf(dmax, ok ? md : 0.0f);
                        if (ok) {
                            const int64_t at = (int64_t)h * p.pitch + (int64_t)o * p.plane;
                            st4(dst + at, scale4(nxt, iu));
                            st4(dst_d + at, scale4(dnx, id));
                        }
                    }
                    // output i's partial: (centre, x, y) * s_n + z terms of
                    // planes i-1 .. i-R; slot K held plane i - R - 1, now free
                    if (has_out) {
                        const float4 z1 = uq[h][(K + S::RING - 1) % S::RING];
                        const float2 c1 = make_float2(wf<R>(1), wf<R>(1));
                        float2 zA = __fmul2_rn(c1, lo2(z1)), zB = __fmul2_rn(c1, hi2(z1));
#pragma unroll
                        for (int r = 2; r <= R; ++r) {
                            const float4 zm = uq[h][(K + S::RING - r) % S::RING];
                            const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                            zA = __ffma2_rn(cr, lo2(zm), zA);
                            zB = __ffma2_rn(cr, hi2(zm), zB);
                        }
                        pa[h][K] = __ffma2_rn(ss, xA[h], zA);
                        pb[h][K] = __ffma2_rn(ss, xB[h], zB);
                    } else {
                        pa[h][K] = pb[h][K] = make_float2(0.f, 0.f);
                    }
                    uq[h][K] = c;
                }
            };
            dispatch<S::RING>(k, ring);
            if (fin) {
                const unsigned wu = __reduce_max_sync(0xffffffffu, __float_as_uint(umax));
                const unsigned wd = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
                if ((tid & 31) == 0) {
                    wmax[(i & 1) * 2 * (S::NT / 32) + (tid >> 5)] = wu;
                    wmax[(i & 1) * 2 * (S::NT / 32) + (S::NT / 32) + (tid >> 5)] = wd;
                }
            }
            if (REC && (k == S::RING - 1 || i == nin - 1)) {
                eacc += (double)((ekin.x + ekin.y) - (epot.x + epot.y));
                ekin = epot = make_float2(0.f, 0.f);
            }
            if (++k == S::RING) k = 0;
            // every thread is done with plane i's u stage and output (i-2R)'s
            // aux stage: refill them
            __syncthreads();
            done = i + 1;
            if (*abort_flag) break;                 // block-uniform exit
            if (tid == 0) {
                if (i + S::SU < nin) issue_u(i + S::SU);
                if (fin && i - 2 * R + S::SA < nout) issue_a(i - 2 * R + S::SA);
            }
            // the plane's maxima, merged by the last warp (the first one issues the copies)
            if (fin && tid == S::NT - 32) {
                const unsigned *wm = wmax + (i & 1) * 2 * (S::NT / 32);
                unsigned mu = 0, md = 0;
                for (int w = 0; w < S::NT / 32; ++w) {
                    mu = max(mu, wm[w]);
                    md = max(md, wm[S::NT / 32 + w]);
                }
                const int64_t at = (int64_t)slot_out * p.nz + z0 + (i - 2 * R);
                if (mu) atomicMax(p.amax + at, mu);
                if (md) atomicMax(p.amax_d + at, md);
            }
        }
    }
    if (REC) {
        // the warp's sum of its threads' FP64 energy terms (fixed order)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, off);
        if ((tid & 31) == 0) en_warp[tid >> 5] = eacc;
    }
    if (*abort_flag && tid == 0) {
        // let the copies already issued land before the block's shared
        // memory is released (bounded).  After the barrier of plane
        // done - 1, planes done .. done+SU-2 and the aux planes from the
        // first unconsumed one up to the last issued one are in flight.
        const int i = done - 1;
        for (int t = done; t < min(nin, done + S::SU - 1); ++t)
            mbar_wait(&full_u[t % S::SU], (t / S::SU) & 1, p.err, 100000000ull);
        const int cons_a = i >= 2 * R ? i - 2 * R + 1 : 0;
        const int iss_a = min(nout, i >= 2 * R + 1 ? i - 2 * R + S::SA : S::SA);
        for (int ja = cons_a; ja < iss_a; ++ja)
            mbar_wait(&full_a[ja % S::SA], (ja / S::SA) & 1, p.err, 100000000ull);
    }
}

// One shot per launch: block (tile, z-chunk) from the grid position.  REC:
// the variant that also sums the step's energy (launched only when
// p.energy_on is set, so the kernel does not test it); ABS: the variant with the
// absorbing layer folded in (FP32).
template <int R, int TX, int TY, typename E, bool REC = false, bool ABS = false>
__global__ void __launch_bounds__(TiledShape<R, TX, TY, E>::NT, TiledShape<R, TX, TY, E>::MINB)
    sweep_tiled_kernel(const __grid_constant__ CUtensorMap map_u, const __grid_constant__ CUtensorMap map_up,
                       const __grid_constant__ CUtensorMap map_k, const SweepParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int bx = blockIdx.x % p.tiles_x;
    const int by = blockIdx.x / p.tiles_x;
    const int z0 = blockIdx.y * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int64_t n = current_step(p);
    sweep_tile<R, TX, TY, E, REC, ABS>(&map_u, &map_up, &map_k, p, bx, by, z0, z1, n, smem);
    if constexpr (REC) {
        // block partial (warps in order); the last block to finish then
        // adds all partials: thread t the blocks t, t + NT, ... in order,
        // then a fixed tree over the threads.  The step's energy depends
        // only on the data, and the tail after the last block's sweep is
        // ~nblk / NT loads per thread instead of nblk serial ones.
        using S = TiledShape<R, TX, TY, E>;
        __shared__ double red[S::NT];
        __shared__ unsigned last;
        const unsigned nblk = gridDim.x * gridDim.y;
        __syncthreads();
        if (threadIdx.x == 0) {
            const double *en_warp = reinterpret_cast<const double *>(smem + S::EN_OFF);
            double b = 0.0;
            for (int w = 0; w < S::NT / 32; ++w) b += en_warp[w];
            p.energy_part[blockIdx.y * gridDim.x + blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(p.energy_count, 1u) == nblk - 1;
        }
        __syncthreads();
        if (last) {                                  // uniform over the block
            __threadfence();
            double acc = 0.0;
            for (unsigned k = threadIdx.x; k < nblk; k += S::NT) acc += __ldcg(p.energy_part + k);
            red[threadIdx.x] = acc;
            __syncthreads();
#pragma unroll
            for (int w = S::NT / 2; w > 0; w >>= 1) {
                if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const int64_t m = n - p.rec_n0;
                if (m >= 0 && m < p.rec_cap) p.energy[m] = red[0];
                *p.energy_count = 0u;
            }
        }
    }
}

// Many shots per launch (one time step of each): block b does work item
// items[b] of shot items[b].shot.  ABS: the variant with the absorbing layer
// (shots of the group without one have absorb_w = 0 and pass unchanged).  A shot whose step counter has reached its
// last step is left as it is (its blocks return at once), so shots with
// different step counts share one launch sequence.
template <int R, int TX, int TY, typename E, bool ABS = false>
__global__ void __launch_bounds__(TiledShape<R, TX, TY, E>::NT, TiledShape<R, TX, TY, E>::MINB)
    sweep_grouped_kernel(const GroupShot *shots, const GroupItem *items, int step_off)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const GroupItem it = items[blockIdx.x];
    const GroupShot &g = shots[it.shot];
    const int64_t n = *g.prm.step_base + step_off;
    if (n >= g.n_end) return;                       // uniform over the block
    const int par = (int)((n + g.parity_base) & 1);
    SweepParams p = g.prm;
    p.u = g.buf[par];
    p.up = g.buf[par ^ 1];
    p.step_off = step_off;
    if (threadIdx.x == 0) {                         // the copy-issuing thread
        fence_tensormap(&g.halo[par]);
        fence_tensormap(&g.core[par ^ 1]);
        fence_tensormap(&g.kcore);
    }
    sweep_tile<R, TX, TY, E, false, ABS, false>(&g.halo[par], &g.core[par ^ 1], &g.kcore, p, it.bx, it.by, it.z0, it.z1, n,
                                         smem);
}

}  // namespace stencil
