// K1: 2.5D-blocked sweep, one time step per launch.
//
// The GPU form of the paper's loop tiling (Sec. 3, Fig. 1b): instead of a
// cache blocksize (i, j, k) each thread block owns a TX x TY tile of the xy
// plane and marches through a chunk of z planes.  Per plane:
//   * one TMA box of u^n, (TX + 2 HX) x (TY + 2R), lands in a shared-memory
//     ring of SU stages (out-of-range coordinates are zero-filled by the TMA
//     unit, which is exactly the ghost-zero Dirichlet boundary);
//   * TMA boxes of u^{n-1} and kappa (TX x TY) land in a ring of SA stages;
//   * each thread owns 4 consecutive x points in each of 2 rows (the y
//     neighbours it loads serve both rows).  When plane p lands, the thread
//     reads its own values and its x and y neighbours (16-byte shared-memory
//     vectors) and immediately forms the partial sum of output plane p: x
//     and y terms, the z centre and the z terms of the R planes below p,
//     which it keeps in registers.  Plane p also adds its z term to the
//     partial sums of the R-1 outputs below it and completes output p-R,
//     which is then updated with u^{n-1} and kappa and written over u^{n-1}
//     with 16-byte stores.  A u stage is therefore free again right after
//     its plane has been read, so shared memory holds copies in flight
//     rather than planes waiting for their turn, and a small footprint
//     (4 stages) lets three blocks share an SM;
//   * arithmetic runs two points at a time with packed FP32 instructions;
//     the register ring of (u, partial) pairs is rotated by unrolling.
// Thread 0 issues every copy right after the block barrier that ends each
// plane, into the stages that plane freed; "full" mbarriers (expect_tx)
// signal arrival.  Every wait is bounded: a stuck wait sets ERR_TIMEOUT and
// the whole block leaves at the next barrier, after the copies it issued
// have landed (also bounded).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace stencil {

template <int R, int TX, int TY>
struct TiledShape {
    static constexpr int HX = ((R + 3) / 4) * 4;        // x halo rounded to 16 bytes
    static constexpr int BW = TX + 2 * HX;              // u box width
    static constexpr int BH = TY + 2 * R;               // u box height
    static constexpr int TPR = TX / 4;                  // threads per row
    static constexpr int ROWS = 2;                      // rows per thread
    static constexpr int NT = TPR * TY / ROWS;          // threads per block
    static constexpr int RING = R + 1;                  // register ring of (u, partial) per plane
    static constexpr int SU = 4;                        // u stages: 1 being read + 3 in flight
    static constexpr int SA = 4;                        // u_prev / kappa stages
    static constexpr int U_ELEMS = ((BW * BH * 4 + 127) / 128) * 32;   // stage size in floats (128 B aligned)
    static constexpr int A_ELEMS = TX * TY;
    static constexpr uint32_t U_BYTES = BW * BH * 4;
    static constexpr uint32_t A_BYTES = TX * TY * 4;
    static constexpr int BAR_OFF = (SU * U_ELEMS + 2 * SA * A_ELEMS) * 4;
    static constexpr int FLAG_OFF = BAR_OFF + (SU + SA) * 8;
    static constexpr int SMEM = FLAG_OFF + 16;
    static_assert(TX % 32 == 0 && TX >= 32 && BW <= 256 && BH <= 256, "TMA box limits");
    static_assert(TY % ROWS == 0, "whole thread rows");
    static constexpr bool VALID = NT <= 1024 && NT % 32 == 0;
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

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

template <int R, int TX, int TY>
__global__ void __launch_bounds__(TiledShape<R, TX, TY>::NT)
    sweep_tiled_kernel(const __grid_constant__ CUtensorMap map_u, const __grid_constant__ CUtensorMap map_up,
                       const __grid_constant__ CUtensorMap map_k, const SweepParams p)
{
    using S = TiledShape<R, TX, TY>;
    extern __shared__ __align__(128) unsigned char smem[];
    float *su = reinterpret_cast<float *>(smem);
    float *sp = su + S::SU * S::U_ELEMS;
    float *sk = sp + S::SA * S::A_ELEMS;
    uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);
    uint64_t *full_a = full_u + S::SU;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + S::FLAG_OFF);

    const int tid = threadIdx.x;
    const int bx = blockIdx.x % p.tiles_x;
    const int by = blockIdx.x / p.tiles_x;
    const int x0 = bx * TX;
    const int y0 = by * TY;
    const int z0 = blockIdx.y * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    if (z0 >= z1) return;                     // uniform over the block
    const int nout = z1 - z0;                 // output planes
    const int nin = nout + 2 * R;             // planes through the ring: z0-R .. z1+R-1
    const int pz0 = z0 - R;

    auto issue_u = [&](int t) {               // plane pz0 + t into stage t % SU
        const int st = t % S::SU;
        mbar_arrive_expect_tx(&full_u[st], S::U_BYTES);
        tma_load_3d(su + st * S::U_ELEMS, &map_u, &full_u[st], x0 - S::HX, y0 - R, pz0 + t);
    };
    auto issue_a = [&](int ja) {              // u^{n-1} and kappa of output z0 + ja into stage ja % SA
        const int st = ja % S::SA;
        mbar_arrive_expect_tx(&full_a[st], 2 * S::A_BYTES);
        tma_load_3d(sp + st * S::A_ELEMS, &map_up, &full_a[st], x0, y0, z0 + ja);
        tma_load_3d(sk + st * S::A_ELEMS, &map_k, &full_a[st], x0, y0, z0 + ja);
    };

    if (tid == 0) {
        for (int i = 0; i < S::SU; ++i) mbar_init(&full_u[i], 1);
        for (int i = 0; i < S::SA; ++i) mbar_init(&full_a[i], 1);
        *abort_flag = 0;
        fence_barrier_init();
        for (int t = 0; t < S::SU && t < nin; ++t) issue_u(t);
        for (int ja = 0; ja < S::SA && ja < nout; ++ja) issue_a(ja);
    }
    __syncthreads();

    const int tx4 = tid % S::TPR;
    const int ty0 = (tid / S::TPR) * S::ROWS;              // first of this thread's rows
    const int gx = x0 + 4 * tx4;
    const int gy0 = y0 + ty0;
    const bool x_ok = gx < p.nx;
    const int own = (R + ty0) * S::BW + S::HX + 4 * tx4;   // own 4 points of row 0 in a u stage
    const int own_a = ty0 * TX + 4 * tx4;
    float *dst = p.up + (int64_t)gy0 * p.pitch + gx;
    const int src_row = p.src.y - gy0;                     // this thread's row holding the source, if any
    const bool src_here = p.src.on && (unsigned)src_row < (unsigned)S::ROWS && (unsigned)(p.src.x - gx) < 4u &&
                          p.src.z >= z0 && p.src.z < z1;

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
    int su_stage = 0, su_phase = 0;         // stage / parity of plane i
    int sa_stage = 0, sa_phase = 0;         // aux stage / parity of output ja = i - 2R
    int done = 0;                           // planes fully processed (block-uniform)

    for (int i0 = 0; i0 < nin; i0 += S::RING) {
        auto body = [&](auto kc) {
            constexpr int K = decltype(kc)::value;          // slot of plane i
            const int i = i0 + K;
            if (i >= nin) return;                           // block-uniform
            if (!mbar_wait(&full_u[su_stage], su_phase, p.err)) *abort_flag = 1;
            const float *pl = su + su_stage * S::U_ELEMS + own;
            // column of the thread's x group: rows -R .. ROWS-1+R around row 0
            float4 col[S::ROWS + 2 * R];
#pragma unroll
            for (int h = 0; h < S::ROWS; ++h) col[R + h] = *reinterpret_cast<const float4 *>(pl + h * S::BW);
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
                    col[R - r] = *reinterpret_cast<const float4 *>(pl - r * S::BW);
                    col[R + S::ROWS - 1 + r] = *reinterpret_cast<const float4 *>(pl + (S::ROWS - 1 + r) * S::BW);
                }
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    const float *ph = pl + h * S::BW;
                    const float4 c = col[R + h];
                    float2 aA = __fmul2_rn(c0x3, lo2(c));
                    float2 aB = __fmul2_rn(c0x3, hi2(c));
                    // row[m] = u[gx - 8 + m], m = 0..19; own points are m = 8..11
                    float row[20];
                    {
                        const float4 l1 = *reinterpret_cast<const float4 *>(ph - 4);
                        const float4 r1 = *reinterpret_cast<const float4 *>(ph + 4);
                        row[4] = l1.x; row[5] = l1.y; row[6] = l1.z; row[7] = l1.w;
                        row[8] = c.x; row[9] = c.y; row[10] = c.z; row[11] = c.w;
                        row[12] = r1.x; row[13] = r1.y; row[14] = r1.z; row[15] = r1.w;
                        if constexpr (R > 4) {
                            const float4 l2 = *reinterpret_cast<const float4 *>(ph - 8);
                            const float4 r2 = *reinterpret_cast<const float4 *>(ph + 8);
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
                        const float4 zm = uq[h][(K + S::RING - r) % S::RING];   // plane i - r
                        float2 sA =
                            __fadd2_rn(make_float2(row[8 - r], row[9 - r]), make_float2(row[8 + r], row[9 + r]));
                        float2 sB =
                            __fadd2_rn(make_float2(row[10 - r], row[11 - r]), make_float2(row[10 + r], row[11 + r]));
                        sA = __fadd2_rn(sA, __fadd2_rn(lo2(ym), lo2(yp)));
                        sB = __fadd2_rn(sB, __fadd2_rn(hi2(ym), hi2(yp)));
                        sA = __fadd2_rn(sA, lo2(zm));
                        sB = __fadd2_rn(sB, hi2(zm));
                        const float2 cr = make_float2(wf<R>(r), wf<R>(r));
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
                if (!mbar_wait(&full_a[sa_stage], sa_phase, p.err)) *abort_flag = 1;
                float4 prev[S::ROWS], kap[S::ROWS];
#pragma unroll
                for (int h = 0; h < S::ROWS; ++h) {
                    prev[h] = *reinterpret_cast<const float4 *>(sp + sa_stage * S::A_ELEMS + own_a + h * TX);
                    kap[h] = *reinterpret_cast<const float4 *>(sk + sa_stage * S::A_ELEMS + own_a + h * TX);
                }
                if (++sa_stage == S::SA) {
                    sa_stage = 0;
                    sa_phase ^= 1;
                }
                const int o = z0 + (i - 2 * R);
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
                    if (src_here && src_row == h && o == p.src.z) {
                        const double t = (double)current_step(p) * p.src.dt;
                        const float add = (float)(p.src.scale * ricker(p.src.f, p.src.t0, t));
                        const int k = p.src.x - gx;
                        if (k == 0) nxt.x += add;
                        else if (k == 1) nxt.y += add;
                        else if (k == 2) nxt.z += add;
                        else nxt.w += add;
                    }
                    if (x_ok && gy0 + h < p.ny)
                        *reinterpret_cast<float4 *>(dst + (int64_t)h * p.pitch + (int64_t)o * p.plane) = nxt;
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

}  // namespace stencil
