// Plans that advance two time steps per launch (STENCIL_KERNEL_TWO_STEP).
//
// The kernel reads u^{n-1} and u^n and writes u^{n+1} and u^{n+2} into two
// other buffers, because neighbouring thread blocks still read both inputs
// around their own tiles.  The plan therefore holds four FP32 level buffers
// B = (buf[0], buf[1], tbuf[0], tbuf[1]) in two pairs; the current levels
// are one pair, (u^{n-1}, u^n) = (B[2q], B[2q+1]) with q = t2_pair, and a
// two-step launch writes the other pair.  An odd step count ends with one
// launch of the one-step tiled kernel, which writes u^{n+1} over u^{n-1} in
// place: the pair then holds its levels the other way round (t2_swapped),
// and the next two-step launch returns to the normal order.  The state is
// advanced on the host as launches are enqueued, as the one-step plans flip
// `cur`.
#include <algorithm>

#include "plan_impl.h"

namespace stencil {

void *Plan::level_buf(int which) const
{
    if (tile.kernel != STENCIL_KERNEL_TWO_STEP) return buf[cur ^ which];
    const int q = 2 * t2_pair;
    const int now = t2_swapped ? q : q + 1;
    return t2_buf(which == 0 ? now : now ^ 1);
}

int Plan::build_maps_two_step()
{
    TwoStepInfo info;
    if (!two_step_config(R, tile.tx, tile.ty, &info))
        return fail(STENCIL_EUNSUPPORTED, "two-step tile %dx%d not built for radius %d", tile.tx, tile.ty, R);
    TiledInfo plain;
    if (!tiled_config(R, STENCIL_FP32, 64, 16, &plain))
        return fail(STENCIL_EUNSUPPORTED, "tiled kernel 64x16 not built for radius %d", R);
    const int tx = tile.tx, ty = tile.ty;
    for (int k = 0; k < 4; ++k) {
        const void *b = t2_buf(k);
        int rc = encode_map(&t2_u_halo[k], b, nx, ny, nz, pitch, 4, tx + 2 * info.ex + 2 * info.hx, ty + 4 * R);
        if (!rc) rc = encode_map(&t2_up_region[k], b, nx, ny, nz, pitch, 4, tx + 2 * info.ex, ty + 2 * R);
        if (!rc) rc = encode_map(&t2_u_core[k], b, nx, ny, nz, pitch, 4, tx, ty);
        if (!rc) rc = encode_map(&t2_plain_halo[k], b, nx, ny, nz, pitch, 4, 64 + 2 * plain.hx, 16 + 2 * R);
        if (!rc) rc = encode_map(&t2_plain_core[k], b, nx, ny, nz, pitch, 4, 64, 16);
        if (rc) return rc;
    }
    int rc = encode_map(&t2_k_region, kappa, nx, ny, nz, pitch, 4, tx + 2 * info.ex, ty + 2 * R);
    if (!rc) rc = encode_map(&t2_k_core, kappa, nx, ny, nz, pitch, 4, tx, ty);
    if (!rc) rc = encode_map(&map_kcore, kappa, nx, ny, nz, pitch, 4, 64, 16);
    return rc;
}

cudaError_t Plan::launch_two_step_pair(int step_off, cudaStream_t s)
{
    const int q = 2 * t2_pair;
    const int now = t2_swapped ? q : q + 1, before = now ^ 1;
    const int o = 2 * (1 - t2_pair);                 // the other pair receives u^{n+1}, u^{n+2}
    TwoStepMaps m;
    m.u_halo = t2_u_halo[now];
    m.up_region = t2_up_region[before];
    m.k_region = t2_k_region;
    m.u_core = t2_u_core[now];
    m.k_core = t2_k_core;
    SweepParams prm = params(0, step_off);
    prm.u = t2_buf(now);
    prm.up = t2_buf(before);
    prm.zchunk = tile.zchunk > 0 ? tile.zchunk : nz;
    const cudaError_t e =
        launch_two_step(R, m, prm, static_cast<float *>(t2_buf(o)), static_cast<float *>(t2_buf(o + 1)), s);
    t2_pair ^= 1;
    t2_swapped = false;
    cur = o + 1;
    return e;
}

cudaError_t Plan::launch_two_step_single(int step_off, cudaStream_t s)
{
    const int q = 2 * t2_pair;
    const int now = t2_swapped ? q : q + 1, before = now ^ 1;
    TiledMaps m;
    m.u_halo = t2_plain_halo[now];
    m.up_core = t2_plain_core[before];
    m.k_core = map_kcore;
    SweepParams prm = params(0, step_off);
    prm.u = t2_buf(now);
    prm.up = t2_buf(before);                         // u^{n+1} is written over u^{n-1}
    prm.zchunk = t2_plain_zchunk > 0 ? t2_plain_zchunk : nz;
    const cudaError_t e = launch_tiled(R, STENCIL_FP32, 64, 16, m, prm, s);
    t2_swapped = !t2_swapped;
    cur = before;
    return e;
}

int Plan::capture_graphs_two_step()
{
    drop_graphs();
    const int pair0 = t2_pair, cur0 = cur;
    const bool sw0 = t2_swapped;
    int rc = STENCIL_OK;
    for (int par = 0; par < 2 && rc == STENCIL_OK; ++par) {
        t2_pair = par;
        t2_swapped = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = fail_cuda(e, "cudaStreamBeginCapture");
            break;
        }
        cudaError_t le = cudaSuccess;
        for (int i = 0; i < graph_len && le == cudaSuccess; i += 2) le = launch_two_step_pair(i, stream);
        if (le == cudaSuccess) le = launch_advance(d_step, graph_len, stream);
        e = cudaStreamEndCapture(stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            rc = fail_cuda(le, "launch during graph capture");
            break;
        }
        if (e != cudaSuccess) {
            rc = fail_cuda(e, "cudaStreamEndCapture");
            break;
        }
        e = cudaGraphInstantiate(&graph_exec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) rc = fail_cuda(e, "cudaGraphInstantiate");
    }
    t2_pair = pair0;
    t2_swapped = sw0;
    cur = cur0;
    if (rc) drop_graphs();
    return rc;
}

int Plan::enqueue_two_step(int nsteps)
{
    int left = nsteps;
    // graphs start from a pair in the normal order: a swapped pair takes one
    // eager two-step launch first
    if (t2_swapped && left >= 2) {
        cudaError_t e = launch_two_step_pair(0, stream);
        if (e == cudaSuccess) e = launch_advance(d_step, 2, stream);
        if (e != cudaSuccess) return fail_cuda(e, "two-step launch");
        left -= 2;
    }
    if (graph_len >= 2 && left >= graph_len && !t2_swapped) {
        if (!graph_exec[0]) {
            int rc = capture_graphs_two_step();
            if (rc) return rc;
        }
        while (left >= graph_len) {
            cudaError_t e = cudaGraphLaunch(graph_exec[t2_pair], stream);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGraphLaunch");
            t2_pair ^= (graph_len / 2) & 1;
            cur = 2 * t2_pair + 1;
            left -= graph_len;
        }
    }
    while (left > 0) {
        const int k = std::min(left, 64);
        int off = 0;
        cudaError_t e = cudaSuccess;
        for (; off + 2 <= k && e == cudaSuccess; off += 2) e = launch_two_step_pair(off, stream);
        if (off < k && e == cudaSuccess) e = launch_two_step_single(off, stream);
        if (e == cudaSuccess) e = launch_advance(d_step, k, stream);
        if (e != cudaSuccess) return fail_cuda(e, "two-step launch");
        left -= k;
    }
    steps_done += nsteps;
    return STENCIL_OK;
}

}  // namespace stencil
