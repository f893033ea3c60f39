// K7: two time steps per sweep (temporal blocking of the 2.5D z-march), FP32.
//
// The related-work direction the paper points to (Sec. 4, "3.5D" blocking:
// 2.5D spatial blocking plus blocking in time).  One launch advances
// u^{n-1}, u^n to u^{n+1}, u^{n+2}.  A thread block owns a TX x TY tile of
// the xy plane and a chunk of z planes and marches through z once:
//   * stage A computes u^{n+1} on the tile plus a ring of EX >= R columns
//     and R rows around it (the "ghost zone": the points of the neighbouring
//     tiles that stage B reads), for the planes of the chunk plus R above
//     and below.  u^n arrives per plane as one TMA box with the stencil's
//     halo around that region, u^{n-1} and kappa as boxes of the region;
//     each thread owns 4 x points in 2 rows and keeps the z terms in a
//     register ring, as the one-step kernel does;
//   * each completed plane of u^{n+1} on the region goes to a shared-memory
//     plane (two, alternating); stage B reads its x and y neighbours there
//     (one thread per 4 x points in 1 row of the tile, its own register
//     ring for the z terms) and completes u^{n+2} R planes behind, with u^n
//     and kappa of the tile from two more TMA boxes (read for the second
//     time within a few planes, so from L2);
//   * u^{n+1} (tile points, the chunk's planes) and u^{n+2} go to two
//     further buffers: no input is overwritten, since neighbouring blocks
//     still read u^{n-1} and u^n of this tile for their own ghost zones.
// Algorithmic traffic: read u^n, u^{n-1}, kappa, write u^{n+1}, u^{n+2}:
// 20 B per two point updates, 10 B per update (16 B for the one-step sweep).
// The price is the ghost zone: stage A evaluates the stencil on
// (TX + 2 EX)(TY + 2R) points per TX TY outputs.
//
// Points of the region outside the grid come out as zero (every input box
// is zero-filled there by the TMA unit), which is the ghost-zero boundary
// stage B needs.  The point source is added by stage A at time n (on every
// region that contains it, so the ghost copies match the owner's values)
// and by stage B at time n+1.  Every wait is bounded, as in the one-step
// kernel.
#pragma once

#include "sweep_tiled.cuh"

namespace stencil {

template <int R, int TX, int TY>
struct TwoStepShape {
    static constexpr int EX = ((R + 3) / 4) * 4;        // ring columns on each side (>= R, whole quads)
    static constexpr int HX = ((R + 3) / 4) * 4;        // x halo of stage A's stencil (16-byte rounded)
    static constexpr int WA = TX + 2 * EX;              // stage A region width
    static constexpr int HA = TY + 2 * R;               // stage A region height
    static constexpr int BW = WA + 2 * HX;              // u^n box width
    static constexpr int BH = HA + 2 * R;               // u^n box height
    static constexpr int AQX = WA / 4;                  // stage A: quads per row
    static constexpr int AROWS = 2;                     // stage A: rows per thread
    static constexpr int AIT = AQX * (HA / AROWS);      // stage A items
    static constexpr int BQX = TX / 4;                  // stage B: quads per row (1 row per thread)
    static constexpr int BIT = BQX * TY;                // stage B items
    static constexpr int NT = ((AIT > BIT ? AIT : BIT) + 31) / 32 * 32;
    static constexpr int RING = R + 1;
    static constexpr int SU = 3;                        // u^n stages
    static constexpr int SA = 2;                        // stage A aux (u^{n-1}, kappa) stages
    static constexpr int SB = 2;                        // stage B aux (u^n, kappa of the tile) stages
    static constexpr uint32_t U_BYTES = BW * BH * 4;
    static constexpr uint32_t A_BYTES = WA * HA * 4;    // one of u^{n-1}, kappa
    static constexpr uint32_t B_BYTES = TX * TY * 4;    // one of u^n, kappa
    static constexpr int U_STAGE = (U_BYTES + 127) / 128 * 128;
    static constexpr int A_STAGE = (2 * A_BYTES + 127) / 128 * 128;
    static constexpr int B_STAGE = (2 * B_BYTES + 127) / 128 * 128;
    static constexpr int S1_BYTES = (A_BYTES + 127) / 128 * 128;
    static constexpr int A_OFF = SU * U_STAGE;
    static constexpr int B_OFF = A_OFF + SA * A_STAGE;
    static constexpr int S1_OFF = B_OFF + SB * B_STAGE;
    static constexpr int BAR_OFF = S1_OFF + 2 * S1_BYTES;
    static constexpr int FLAG_OFF = BAR_OFF + (SU + SA + SB) * 8;
    static constexpr int SMEM = FLAG_OFF + 16;
    static_assert(TX % 32 == 0 && HA % AROWS == 0 && WA % 4 == 0, "tile shape");
    static_assert(BW <= 256 && BH <= 256 && WA <= 256 && HA <= 256, "TMA box limits");
    static_assert(R <= 2 * HX && R <= 8, "x neighbours within two quads");
};

template <int R, int TX, int TY>
__global__ void __launch_bounds__(TwoStepShape<R, TX, TY>::NT, 1)
    sweep_two_step_kernel(const __grid_constant__ CUtensorMap map_u,    // u^n, box BW x BH
                          const __grid_constant__ CUtensorMap map_ua,   // u^{n-1}, box WA x HA
                          const __grid_constant__ CUtensorMap map_ka,   // kappa, box WA x HA
                          const __grid_constant__ CUtensorMap map_uc,   // u^n, box TX x TY
                          const __grid_constant__ CUtensorMap map_kc,   // kappa, box TX x TY
                          const SweepParams prm, float *out1, float *out2)
{
    using S = TwoStepShape<R, TX, TY>;
    extern __shared__ __align__(128) unsigned char smem[];
    const SweepParams p = prm;
    unsigned char *su = smem;
    unsigned char *sa = smem + S::A_OFF;
    unsigned char *sb = smem + S::B_OFF;
    float *s1 = reinterpret_cast<float *>(smem + S::S1_OFF);
    uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);
    uint64_t *full_a = full_u + S::SU;
    uint64_t *full_b = full_a + S::SA;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + S::FLAG_OFF);

    const uint64_t wait_limit = p.wait_ns ? p.wait_ns : 2000000000ull;
    const int tid = threadIdx.x;
    const int x0 = (blockIdx.x % p.tiles_x) * TX;
    const int y0 = (blockIdx.x / p.tiles_x) * TY;
    const int z0 = blockIdx.y * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    if (z0 >= z1) return;
    const int nout = z1 - z0;                 // stage B outputs (planes z0 .. z1-1)
    const int nouta = nout + 2 * R;           // stage A outputs (planes z0-R .. z1+R-1)
    const int nin = nouta + 2 * R;            // u^n planes z0-2R .. z1+2R-1
    const int niter = nin + 1;                // stage B runs one plane behind stage A

    auto issue_u = [&](int t) {               // u^n plane z0 - 2R + t
        const int st = t % S::SU;
        mbar_arrive_expect_tx(&full_u[st], S::U_BYTES + (t == 0 ? p.fault_tx : 0u));
        tma_load_3d(su + st * S::U_STAGE, &map_u, &full_u[st], x0 - S::EX - S::HX, y0 - 2 * R, z0 - 2 * R + t);
    };
    auto issue_a = [&](int ja) {              // u^{n-1}, kappa of stage A output ja (plane z0 - R + ja)
        const int st = ja % S::SA;
        unsigned char *d = sa + st * S::A_STAGE;
        mbar_arrive_expect_tx(&full_a[st], 2 * S::A_BYTES);
        tma_load_3d(d, &map_ua, &full_a[st], x0 - S::EX, y0 - R, z0 - R + ja);
        tma_load_3d(d + S::A_BYTES, &map_ka, &full_a[st], x0 - S::EX, y0 - R, z0 - R + ja);
    };
    auto issue_b = [&](int jb) {              // u^n, kappa of stage B output jb (plane z0 + jb)
        const int st = jb % S::SB;
        unsigned char *d = sb + st * S::B_STAGE;
        mbar_arrive_expect_tx(&full_b[st], 2 * S::B_BYTES);
        tma_load_3d(d, &map_uc, &full_b[st], x0, y0, z0 + jb);
        tma_load_3d(d + S::B_BYTES, &map_kc, &full_b[st], x0, y0, z0 + jb);
    };
    if (tid == 0) {
        for (int i = 0; i < S::SU; ++i) mbar_init(&full_u[i], 1);
        for (int i = 0; i < S::SA; ++i) mbar_init(&full_a[i], 1);
        for (int i = 0; i < S::SB; ++i) mbar_init(&full_b[i], 1);
        *abort_flag = 0;
        fence_barrier_init();
        for (int t = 0; t < S::SU && t < nin; ++t) issue_u(t);
        for (int j = 0; j < S::SA && j < nouta; ++j) issue_a(j);
        for (int j = 0; j < S::SB && j < nout; ++j) issue_b(j);
    }
    __syncthreads();

    // ---- roles ----
    const bool has_a = tid < S::AIT;
    const int aq = tid % S::AQX;
    const int ar0 = (tid / S::AQX) * S::AROWS;             // first region row of this thread
    const int own_u = (R + ar0) * S::BW + S::HX + 4 * aq;  // own points of row 0 in a u^n stage
    const int own_r = ar0 * S::WA + 4 * aq;                // ... in the region (aux boxes, s1)
    const int gxa = x0 - S::EX + 4 * aq;
    const int gya = y0 - R + ar0;
    // this stage A quad lies in the tile (its u^{n+1} is this block's to store)
    const bool a_in_tile_x = 4 * aq >= S::EX && 4 * aq < S::EX + TX;
    const bool has_b = tid < S::BIT;
    const int bq = tid % S::BQX;
    const int brow = tid / S::BQX;
    const int own_s1 = (R + brow) * S::WA + S::EX + 4 * bq;  // own points in s1
    const int own_b = brow * TX + 4 * bq;                   // ... in the stage B aux boxes
    const int gxb = x0 + 4 * bq;
    const int gyb = y0 + brow;

    const int64_t n_level = current_step(p);
    float src_a = 0.0f, src_b = 0.0f;       // the source terms of steps n and n+1
    if (p.src.on) {
        src_a = (float)(p.src.scale * ricker(p.src.f, p.src.t0, (double)n_level * p.src.dt));
        src_b = (float)(p.src.scale * ricker(p.src.f, p.src.t0, (double)(n_level + 1) * p.src.dt));
    }
    const int sxa = p.src.x - gxa, sya = p.src.y - gya;     // source within this stage A quad?
    const bool src_a_here = p.src.on && has_a && (unsigned)sxa < 4u && (unsigned)sya < (unsigned)S::AROWS;
    const bool src_b_here = p.src.on && has_b && (unsigned)(p.src.x - gxb) < 4u && p.src.y == gyb;

    float4 uq[S::AROWS][S::RING];             // stage A ring: u^n (own points) and partial sums
    float2 pa[S::AROWS][S::RING], pb[S::AROWS][S::RING];
    float4 vq[S::RING];                       // stage B ring: u^{n+1} and partial sums
    float2 qa[S::RING], qb[S::RING];
#pragma unroll
    for (int j = 0; j < S::RING; ++j) {
#pragma unroll
        for (int h = 0; h < S::AROWS; ++h) {
            uq[h][j] = make_float4(0.f, 0.f, 0.f, 0.f);
            pa[h][j] = pb[h][j] = make_float2(0.f, 0.f);
        }
        vq[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        qa[j] = qb[j] = make_float2(0.f, 0.f);
    }
    const float2 two = make_float2(2.0f, 2.0f);
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float2 c0x3 = make_float2(3.0f * wf<R>(0), 3.0f * wf<R>(0));

    // The Laplacian's x, y and centre terms at 4 points of one row: p0 is
    // the own quad in a row-major plane of row stride `ld` (floats), with at
    // least 8 columns to the left and right when R > 4 (4 when R <= 4).
    auto xy_terms = [&](const float *p0, int ld, float2 &aA, float2 &aB) {
        const float4 c = *reinterpret_cast<const float4 *>(p0);
        aA = __fmul2_rn(c0x3, lo2(c));
        aB = __fmul2_rn(c0x3, hi2(c));
        float row[20];                          // row[m] = u[x - 8 + m]; own points m = 8..11
        {
            const float4 l1 = *reinterpret_cast<const float4 *>(p0 - 4);
            const float4 r1 = *reinterpret_cast<const float4 *>(p0 + 4);
            row[4] = l1.x; row[5] = l1.y; row[6] = l1.z; row[7] = l1.w;
            row[8] = c.x; row[9] = c.y; row[10] = c.z; row[11] = c.w;
            row[12] = r1.x; row[13] = r1.y; row[14] = r1.z; row[15] = r1.w;
            if constexpr (R > 4) {
                const float4 l2 = *reinterpret_cast<const float4 *>(p0 - 8);
                const float4 r2 = *reinterpret_cast<const float4 *>(p0 + 8);
                row[0] = l2.x; row[1] = l2.y; row[2] = l2.z; row[3] = l2.w;
                row[16] = r2.x; row[17] = r2.y; row[18] = r2.z; row[19] = r2.w;
            } else {
                row[0] = row[1] = row[2] = row[3] = 0.f;
                row[16] = row[17] = row[18] = row[19] = 0.f;
            }
        }
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            const float4 ym = *reinterpret_cast<const float4 *>(p0 - r * ld);
            const float4 yp = *reinterpret_cast<const float4 *>(p0 + r * ld);
            float2 sA = make_float2(row[8 - r] + row[8 + r], row[9 - r] + row[9 + r]);
            float2 sB = make_float2(row[10 - r] + row[10 + r], row[11 - r] + row[11 + r]);
            sA = __fadd2_rn(sA, __fadd2_rn(lo2(ym), lo2(yp)));
            sB = __fadd2_rn(sB, __fadd2_rn(hi2(ym), hi2(yp)));
            const float2 cr = make_float2(wf<R>(r), wf<R>(r));
            aA = __ffma2_rn(cr, sA, aA);
            aB = __ffma2_rn(cr, sB, aB);
        }
    };
    auto add_src = [](float4 &v, int k, float s) {
        if (k == 0) v.x += s;
        else if (k == 1) v.y += s;
        else if (k == 2) v.z += s;
        else v.w += s;
    };

    int done = 0;                              // iterations fully processed (block-uniform)
    for (int i0 = 0; i0 < niter; i0 += S::RING) {
        auto body = [&](auto kc) {
            constexpr int K = decltype(kc)::value;              // stage A ring slot of u^n plane i
            constexpr int KB = (K + 4 * S::RING - 2 * R - 1) % S::RING;   // stage B slot of A output i-2R-1
            const int i = i0 + K;
            if (i >= niter) return;                             // block-uniform
            // ---- stage A: u^n plane i (z = z0 - 2R + i) ----
            if (i < nin) {
                if (!mbar_wait(&full_u[i % S::SU], (i / S::SU) & 1, p.err, wait_limit)) *abort_flag = 1;
                const float *pl = reinterpret_cast<const float *>(su + (i % S::SU) * S::U_STAGE) + own_u;
                const int ja = i - 2 * R;                       // stage A output completed now
                const bool fin = ja >= 0;
                if (fin && has_a)
                    if (!mbar_wait(&full_a[ja % S::SA], (ja / S::SA) & 1, p.err, wait_limit)) *abort_flag = 1;
                if (has_a) {
                    float4 cen[S::AROWS];
                    float2 nA[S::AROWS], nB[S::AROWS];
                    const bool has_out = i >= R && i < R + nouta;
#pragma unroll
                    for (int h = 0; h < S::AROWS; ++h) {
                        cen[h] = *reinterpret_cast<const float4 *>(pl + h * S::BW);
                        nA[h] = nB[h] = make_float2(0.f, 0.f);
                        if (has_out) {
                            float2 aA, aB;
                            xy_terms(pl + h * S::BW, S::BW, aA, aB);
#pragma unroll
                            for (int r = 1; r <= R; ++r) {   // z terms of the R planes below
                                const float4 zm = uq[h][(K + S::RING - r) % S::RING];
                                const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                                aA = __ffma2_rn(cr, lo2(zm), aA);
                                aB = __ffma2_rn(cr, hi2(zm), aB);
                            }
                            nA[h] = aA;
                            nB[h] = aB;
                        }
                        // plane i is the z neighbour above outputs i-1 .. i-(R-1)
#pragma unroll
                        for (int r = 1; r < R; ++r) {
                            const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                            pa[h][(K + S::RING - r) % S::RING] =
                                __ffma2_rn(cr, lo2(cen[h]), pa[h][(K + S::RING - r) % S::RING]);
                            pb[h][(K + S::RING - r) % S::RING] =
                                __ffma2_rn(cr, hi2(cen[h]), pb[h][(K + S::RING - r) % S::RING]);
                        }
                    }
                    if (fin) {
                        // ... and the last one above output i - R: u^{n+1} on the region
                        constexpr int KF = (K + 1) % S::RING;
                        const float2 cR = make_float2(wf<R>(R), wf<R>(R));
                        const float *aux = reinterpret_cast<const float *>(sa + (ja % S::SA) * S::A_STAGE) + own_r;
                        float *dst_s1 = s1 + (ja & 1) * (S::S1_BYTES / 4) + own_r;
                        const int za = z0 - R + ja;
                        const bool store_plane = za >= z0 && za < z1;
#pragma unroll
                        for (int h = 0; h < S::AROWS; ++h) {
                            const float2 fA = __ffma2_rn(cR, lo2(cen[h]), pa[h][KF]);
                            const float2 fB = __ffma2_rn(cR, hi2(cen[h]), pb[h][KF]);
                            const float4 cc = uq[h][KF];
                            const float4 prev = *reinterpret_cast<const float4 *>(aux + h * S::WA);
                            const float4 kap = *reinterpret_cast<const float4 *>(aux + S::A_BYTES / 4 + h * S::WA);
                            const float2 oA =
                                __ffma2_rn(lo2(kap), fA, __ffma2_rn(neg1, lo2(prev), __fmul2_rn(two, lo2(cc))));
                            const float2 oB =
                                __ffma2_rn(hi2(kap), fB, __ffma2_rn(neg1, hi2(prev), __fmul2_rn(two, hi2(cc))));
                            float4 nxt = make_float4(oA.x, oA.y, oB.x, oB.y);
                            if (src_a_here && sya == h && za == p.src.z) add_src(nxt, sxa, src_a);
                            *reinterpret_cast<float4 *>(dst_s1 + h * S::WA) = nxt;
                            const int gy = gya + h;
                            if (store_plane && a_in_tile_x && gy >= y0 && gy < y0 + TY && gy < p.ny && gxa < p.nx)
                                *reinterpret_cast<float4 *>(out1 + (int64_t)gy * p.pitch + (int64_t)za * p.plane +
                                                            gxa) = nxt;
                        }
                    }
#pragma unroll
                    for (int h = 0; h < S::AROWS; ++h) {     // slot K held plane i - R - 1
                        uq[h][K] = cen[h];
                        pa[h][K] = nA[h];
                        pb[h][K] = nB[h];
                    }
                }
            }
            // ---- stage B: u^{n+1} plane a = i - 2R - 1 (z = z0 - R + a), from s1 ----
            const int a = i - 2 * R - 1;
            const int jb = a - 2 * R;                           // stage B output completed now
            if (has_b && a >= 0 && a < nouta) {
                const float *q0 = s1 + (a & 1) * (S::S1_BYTES / 4) + own_s1;
                const float4 cen = *reinterpret_cast<const float4 *>(q0);
                float2 nA = make_float2(0.f, 0.f), nB = nA;
                if (a >= R && a < R + nout) {                   // partial sums of output a - R
                    xy_terms(q0, S::WA, nA, nB);
#pragma unroll
                    for (int r = 1; r <= R; ++r) {
                        const float4 zm = vq[(KB + S::RING - r) % S::RING];
                        const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                        nA = __ffma2_rn(cr, lo2(zm), nA);
                        nB = __ffma2_rn(cr, hi2(zm), nB);
                    }
                }
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 cr = make_float2(wf<R>(r), wf<R>(r));
                    qa[(KB + S::RING - r) % S::RING] = __ffma2_rn(cr, lo2(cen), qa[(KB + S::RING - r) % S::RING]);
                    qb[(KB + S::RING - r) % S::RING] = __ffma2_rn(cr, hi2(cen), qb[(KB + S::RING - r) % S::RING]);
                }
                if (jb >= 0 && jb < nout) {
                    constexpr int KFB = (KB + 1) % S::RING;
                    if (!mbar_wait(&full_b[jb % S::SB], (jb / S::SB) & 1, p.err, wait_limit)) *abort_flag = 1;
                    const float *aux = reinterpret_cast<const float *>(sb + (jb % S::SB) * S::B_STAGE) + own_b;
                    const float2 cR = make_float2(wf<R>(R), wf<R>(R));
                    const float2 fA = __ffma2_rn(cR, lo2(cen), qa[KFB]);
                    const float2 fB = __ffma2_rn(cR, hi2(cen), qb[KFB]);
                    const float4 cc = vq[KFB];                  // u^{n+1}
                    const float4 un = *reinterpret_cast<const float4 *>(aux);
                    const float4 kap = *reinterpret_cast<const float4 *>(aux + S::B_BYTES / 4);
                    const float2 oA = __ffma2_rn(lo2(kap), fA, __ffma2_rn(neg1, lo2(un), __fmul2_rn(two, lo2(cc))));
                    const float2 oB = __ffma2_rn(hi2(kap), fB, __ffma2_rn(neg1, hi2(un), __fmul2_rn(two, hi2(cc))));
                    float4 nxt = make_float4(oA.x, oA.y, oB.x, oB.y);
                    const int zb = z0 + jb;
                    if (src_b_here && zb == p.src.z) add_src(nxt, p.src.x - gxb, src_b);
                    if (gxb < p.nx && gyb < p.ny)
                        *reinterpret_cast<float4 *>(out2 + (int64_t)gyb * p.pitch + (int64_t)zb * p.plane + gxb) =
                            nxt;
                }
                vq[KB] = cen;
                qa[KB] = nA;
                qb[KB] = nB;
            }
            __syncthreads();
            done = i + 1;
            if (*abort_flag) {
                i0 = niter;                                     // block-uniform exit
                return;
            }
            if (tid == 0) {
                if (i + S::SU < nin) issue_u(i + S::SU);
                const int ja = i - 2 * R;
                if (ja >= 0 && ja + S::SA < nouta) issue_a(ja + S::SA);
                if (jb >= 0 && jb + S::SB < nout) issue_b(jb + S::SB);
            }
        };
        Unroll<0, S::RING>::run(body);
    }
    if (*abort_flag && tid == 0) {
        // let the copies already issued land before shared memory is released
        // (bounded): after iteration done - 1, u^n planes done .. and the aux
        // boxes from the first unconsumed one up to the last issued one
        const int i = done - 1;
        for (int t = done; t < min(nin, done + S::SU - 1); ++t)
            mbar_wait(&full_u[t % S::SU], (t / S::SU) & 1, p.err, 100000000ull);
        const int ca = i >= 2 * R ? i - 2 * R + 1 : 0;
        const int ia = min(nouta, i >= 2 * R ? i - 2 * R + S::SA : S::SA);
        for (int j = ca; j < ia; ++j) mbar_wait(&full_a[j % S::SA], (j / S::SA) & 1, p.err, 100000000ull);
        const int jbl = i - 4 * R - 1;
        const int cb = jbl >= 0 ? jbl + 1 : 0;
        const int ib = min(nout, jbl >= 0 ? jbl + S::SB : S::SB);
        for (int j = cb; j < ib; ++j) mbar_wait(&full_b[j % S::SB], (j / S::SB) & 1, p.err, 100000000ull);
    }
}

}  // namespace stencil
