// K1: 2.5D-blocked sweep, one time step per launch.
//
// The GPU form of the paper's loop tiling (Sec. 3, Fig. 1b): instead of a
// cache blocksize (i, j, k) each thread block owns a TX x TY tile of the xy
// plane and marches through a chunk of z planes.  Per plane:
//   * one TMA box of u^n, (TX + 2 HX) x (TY + 2R), lands in a shared-memory
//     ring of SU stages (out-of-range coordinates are zero-filled by the TMA
//     unit, which is exactly the ghost-zero Dirichlet boundary);
//   * TMA boxes of u^{n-1} and kappa (TX x TY) land in a ring of SA stages;
//   * each thread owns 4 consecutive x points of one row and keeps their u
//     values for planes o-R..o+R in registers (the z queue), reads its x and
//     y neighbours of plane o from shared memory as 16-byte vectors, and
//     writes u^{n+1} over u^{n-1} with one 16-byte store.
// One elected thread issues every copy; mbarrier phases (expect_tx) signal
// arrival; a block barrier per plane frees the stages for reuse.  Every
// mbarrier wait is bounded (ERR_TIMEOUT instead of a hang).
#pragma once

#include "common.cuh"

namespace stencil {

template <int R, int TX, int TY>
struct TiledShape {
    static constexpr int HX = ((R + 3) / 4) * 4;        // x halo rounded to 16 bytes
    static constexpr int BW = TX + 2 * HX;              // u box width
    static constexpr int BH = TY + 2 * R;               // u box height
    static constexpr int TPR = TX / 4;                  // threads per row
    static constexpr int NT = TPR * TY;                 // threads per block
    static constexpr int SU = R + 3;                    // u stages: R+1 live planes + 2 in flight
    static constexpr int SA = 3;                        // u_prev / kappa stages
    static constexpr int U_ELEMS = ((BW * BH * 4 + 127) / 128) * 32;   // stage size in floats (128 B aligned)
    static constexpr int A_ELEMS = TX * TY;
    static constexpr uint32_t U_BYTES = BW * BH * 4;
    static constexpr uint32_t A_BYTES = TX * TY * 4;
    static constexpr int BAR_OFF = (SU * U_ELEMS + 2 * SA * A_ELEMS) * 4;
    static constexpr int FLAG_OFF = BAR_OFF + (SU + SA) * 8;
    static constexpr int SMEM = FLAG_OFF + 16;
    static_assert(TX % 32 == 0 && TX >= 32 && BW <= 256 && BH <= 256, "TMA box limits");
    static_assert(NT <= 1024 && NT >= 32, "block size");
};

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
    uint64_t *bar_u = reinterpret_cast<uint64_t *>(smem + S::BAR_OFF);
    uint64_t *bar_a = bar_u + S::SU;
    int &abort_flag = *reinterpret_cast<int *>(smem + S::FLAG_OFF);

    const int tid = threadIdx.x;
    const int tx4 = tid % S::TPR;
    const int ty = tid / S::TPR;
    const int bx = blockIdx.x % p.tiles_x;
    const int by = blockIdx.x / p.tiles_x;
    const int x0 = bx * TX;
    const int y0 = by * TY;
    const int z0 = blockIdx.y * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    if (z0 >= z1) return;                     // uniform over the block
    const int nout = z1 - z0;                 // output planes
    const int nin = nout + 2 * R;             // planes through the queue: z0-R .. z1+R-1
    const int pz0 = z0 - R;

    if (tid == 0) {
        for (int i = 0; i < S::SU; ++i) mbar_init(&bar_u[i], 1);
        for (int i = 0; i < S::SA; ++i) mbar_init(&bar_a[i], 1);
        fence_barrier_init();
        abort_flag = 0;
    }
    __syncthreads();

    int issued_u = 0, issued_a = 0;           // copies issued so far (thread 0 only)
    if (tid == 0) {
        const int nu = min(S::SU, nin);
        issued_u = nu;
        for (int i = 0; i < nu; ++i) {
            mbar_arrive_expect_tx(&bar_u[i], S::U_BYTES);
            tma_load_3d(su + i * S::U_ELEMS, &map_u, &bar_u[i], x0 - S::HX, y0 - R, pz0 + i);
        }
        const int na = min(S::SA, nout);
        issued_a = na;
        for (int j = 0; j < na; ++j) {
            mbar_arrive_expect_tx(&bar_a[j], 2 * S::A_BYTES);
            tma_load_3d(sp + j * S::A_ELEMS, &map_up, &bar_a[j], x0, y0, z0 + j);
            tma_load_3d(sk + j * S::A_ELEMS, &map_k, &bar_a[j], x0, y0, z0 + j);
        }
    }

    const int gx = x0 + 4 * tx4;
    const int gy = y0 + ty;
    const bool store_ok = (gx < p.nx) && (gy < p.ny);
    const int own = (R + ty) * S::BW + S::HX + 4 * tx4;     // offset of own 4 points in a u stage
    const int own_a = ty * TX + 4 * tx4;
    float *dst_row = p.up + (int64_t)gy * p.pitch + gx;

    float4 q[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) q[j] = make_float4(0.f, 0.f, 0.f, 0.f);

    int i = 0;
    for (; i < nin; ++i) {
        const int stage = i % S::SU;
        if (!mbar_wait(&bar_u[stage], (i / S::SU) & 1, p.err)) abort_flag = 1;
        q[2 * R] = *reinterpret_cast<const float4 *>(su + stage * S::U_ELEMS + own);

        if (i >= 2 * R) {
            const int ja = i - 2 * R;                 // output plane index within the chunk
            const int o = z0 + ja;
            const int sa = ja % S::SA;
            if (!mbar_wait(&bar_a[sa], (ja / S::SA) & 1, p.err)) abort_flag = 1;
            const float *pl = su + ((i - R) % S::SU) * S::U_ELEMS + own;
            const float4 c = q[R];
            float4 acc;
            acc.x = 3.0f * wf<R>(0) * c.x;
            acc.y = 3.0f * wf<R>(0) * c.y;
            acc.z = 3.0f * wf<R>(0) * c.z;
            acc.w = 3.0f * wf<R>(0) * c.w;
            // x neighbours: the 16-byte groups left and right of the own group
            const float4 l1 = *reinterpret_cast<const float4 *>(pl - 4);
            const float4 r1 = *reinterpret_cast<const float4 *>(pl + 4);
            float xl[8], xr[8];    // xl[k] = u[x - 1 - k] for point 0; xr[k] = u[x + 4 + k]
            xl[0] = l1.w; xl[1] = l1.z; xl[2] = l1.y; xl[3] = l1.x;
            xr[0] = r1.x; xr[1] = r1.y; xr[2] = r1.z; xr[3] = r1.w;
            if constexpr (R > 4) {
                const float4 l2 = *reinterpret_cast<const float4 *>(pl - 8);
                const float4 r2 = *reinterpret_cast<const float4 *>(pl + 8);
                xl[4] = l2.w; xl[5] = l2.z; xl[6] = l2.y; xl[7] = l2.x;
                xr[4] = r2.x; xr[5] = r2.y; xr[6] = r2.z; xr[7] = r2.w;
            } else {
#pragma unroll
                for (int k = 4; k < 8; ++k) { xl[k] = 0.f; xr[k] = 0.f; }
            }
            // the row of 12 (R=4) / 20 (R=5) values around the own 4 points:
            // row[m] = u[x - 8 + m], m = 0..19; own points are m = 8..11
            float row[20];
#pragma unroll
            for (int k = 0; k < 8; ++k) row[7 - k] = xl[k];
            row[8] = c.x; row[9] = c.y; row[10] = c.z; row[11] = c.w;
#pragma unroll
            for (int k = 0; k < 8; ++k) row[12 + k] = xr[k];
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const float4 ym = *reinterpret_cast<const float4 *>(pl - r * S::BW);
                const float4 yp = *reinterpret_cast<const float4 *>(pl + r * S::BW);
                const float4 zm = q[R - r];
                const float4 zp = q[R + r];
                float s0 = row[8 - r] + row[8 + r];
                float s1 = row[9 - r] + row[9 + r];
                float s2 = row[10 - r] + row[10 + r];
                float s3 = row[11 - r] + row[11 + r];
                s0 += ym.x + yp.x; s1 += ym.y + yp.y; s2 += ym.z + yp.z; s3 += ym.w + yp.w;
                s0 += zm.x + zp.x; s1 += zm.y + zp.y; s2 += zm.z + zp.z; s3 += zm.w + zp.w;
                acc.x = fmaf(wf<R>(r), s0, acc.x);
                acc.y = fmaf(wf<R>(r), s1, acc.y);
                acc.z = fmaf(wf<R>(r), s2, acc.z);
                acc.w = fmaf(wf<R>(r), s3, acc.w);
            }
            const float4 prev = *reinterpret_cast<const float4 *>(sp + sa * S::A_ELEMS + own_a);
            const float4 kap = *reinterpret_cast<const float4 *>(sk + sa * S::A_ELEMS + own_a);
            float4 nxt;
            nxt.x = fmaf(kap.x, acc.x, 2.0f * c.x - prev.x);
            nxt.y = fmaf(kap.y, acc.y, 2.0f * c.y - prev.y);
            nxt.z = fmaf(kap.z, acc.z, 2.0f * c.z - prev.z);
            nxt.w = fmaf(kap.w, acc.w, 2.0f * c.w - prev.w);
            if (p.src.on && o == p.src.z && gy == p.src.y && (unsigned)(p.src.x - gx) < 4u) {
                const double t = (double)current_step(p) * p.src.dt;
                const float add = (float)(p.src.scale * ricker(p.src.f, p.src.t0, t));
                const int k = p.src.x - gx;
                if (k == 0) nxt.x += add;
                else if (k == 1) nxt.y += add;
                else if (k == 2) nxt.z += add;
                else nxt.w += add;
            }
            if (store_ok) *reinterpret_cast<float4 *>(dst_row + (int64_t)o * p.plane) = nxt;
        }
#pragma unroll
        for (int j = 0; j < 2 * R; ++j) q[j] = q[j + 1];

        __syncthreads();                    // stages of planes i-R (xy) and i (queue) are free
        if (abort_flag) break;              // uniform: read after the barrier
        if (tid == 0) {
            const int nu = i - R + S::SU;   // plane i-R leaves; its stage takes plane i-R+SU
            if (i >= R && nu < nin) {
                const int st = nu % S::SU;
                issued_u = nu + 1;
                mbar_arrive_expect_tx(&bar_u[st], S::U_BYTES);
                tma_load_3d(su + st * S::U_ELEMS, &map_u, &bar_u[st], x0 - S::HX, y0 - R, pz0 + nu);
            }
            if (i >= 2 * R) {
                const int na = i - 2 * R + S::SA;
                if (na < nout) {
                    const int st = na % S::SA;
                    issued_a = na + 1;
                    mbar_arrive_expect_tx(&bar_a[st], 2 * S::A_BYTES);
                    tma_load_3d(sp + st * S::A_ELEMS, &map_up, &bar_a[st], x0, y0, z0 + na);
                    tma_load_3d(sk + st * S::A_ELEMS, &map_k, &bar_a[st], x0, y0, z0 + na);
                }
            }
        }
    }
    // After an abandoned wait, let the copies already issued land (bounded)
    // before the block's shared memory is released.
    if (abort_flag && tid == 0) {
        for (int j = i + 1; j < issued_u; ++j)
            mbar_wait(&bar_u[j % S::SU], (j / S::SU) & 1, p.err, 100000000ull);
        for (int j = max(0, i - 2 * R + 1); j < issued_a; ++j)
            mbar_wait(&bar_a[j % S::SA], (j / S::SA) & 1, p.err, 100000000ull);
    }
}

}  // namespace stencil
