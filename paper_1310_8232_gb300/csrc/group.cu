// Grouped multi-shot execution and the stencil_batch_* entry points.
#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "group.h"

namespace stencil {

cudaError_t Group::alloc(void **p, size_t bytes)
{
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMalloc(p, bytes);
}

void Group::free_dev(void *p)
{
    if (!p) return;
    if (pool) cudaFreeAsync(p, stream);
    else cudaFree(p);
}

void Group::release()
{
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    free_dev(d_shots);
    free_dev(d_items);
    free_dev(d_rtm);
    d_shots = nullptr;
    d_items = nullptr;
    d_rtm = nullptr;
    cap_shots = cap_items = 0;
}

int group_zchunk(int R, int storage, int tx, int ty, const std::vector<Plan *> &plans, double share)
{
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int slots = std::max(1, (int)(share * sms * std::max(1, tiled_blocks_per_sm(R, storage, tx, ty))));
    TiledInfo info{};
    tiled_config(R, storage, tx, ty, &info);
    // the single-plan choice's candidates up to 128: small grids want short
    // z-marches (latency), big groups fewer warm-up planes
    static const int cand[] = {8, 12, 16, 24, 32, 48, 64, 96, 128};
    int best = 32;
    double best_t = -1;
    for (int zc : cand) {
        if (info.zmax && zc > info.zmax) break;
        // greedy list schedule of all shots' blocks, chunk-major
        std::vector<double> slot(slots, 0.0);
        std::make_heap(slot.begin(), slot.end(), std::greater<double>());
        double makespan = 0;
        int maxnz = 0;
        for (const Plan *p : plans) maxnz = std::max(maxnz, p->nz);
        for (int z0 = 0; z0 < maxnz; z0 += zc)
            for (const Plan *p : plans) {
                if (z0 >= p->nz) continue;
                const int tiles = ((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty);
                const double cost = std::min(zc, p->nz - z0) + 0.5 * 2 * R;
                for (int t = 0; t < tiles; ++t) {
                    std::pop_heap(slot.begin(), slot.end(), std::greater<double>());
                    slot.back() += cost;
                    makespan = std::max(makespan, slot.back());
                    std::push_heap(slot.begin(), slot.end(), std::greater<double>());
                }
            }
        if (best_t < 0 || makespan < best_t) {
            best_t = makespan;
            best = zc;
        }
    }
    return best;
}

int Group::build(const std::vector<Plan *> &plans, const std::vector<int64_t> &n_end)
{
    if (graph) {
        cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    n_shots = (int)plans.size();
    h_shots.assign(n_shots, GroupShot{});
    absorb = false;
    for (const Plan *p : plans) absorb = absorb || p->absorb_folded();
    h_items.clear();
    h_rtm.clear();
    int maxnz = 0;
    for (int i = 0; i < n_shots; ++i) {
        const Plan *p = plans[i];
        if (p->R != R || p->storage != storage || p->tile.kernel != STENCIL_KERNEL_TILED || p->tile.tx != tx ||
            p->tile.ty != ty)
            return fail(STENCIL_EINVAL, "shot %d does not match the group's radius, storage or tile", i);
        GroupShot &g = h_shots[i];
        g.halo[0] = p->maps_halo[0];
        g.halo[1] = p->maps_halo[1];
        g.core[0] = p->maps_core[0];
        g.core[1] = p->maps_core[1];
        g.kcore = p->map_kcore;
        g.prm = p->params(0, 0);            // with the layer's width and table if it has one
        g.prm.zchunk = zchunk;
        g.prm.energy_on = 0;        // grouped launches run the plain sweep
        g.prm.fault_tx = 0;
        g.buf[0] = p->buf[0];
        g.buf[1] = p->buf[1];
        g.n_end = n_end[i];
        g.parity_base = (int)(((p->cur - p->steps_done) % 2 + 2) % 2);
        g.rtm = p->rtm;
        if (p->rtm.phase != 0) h_rtm.push_back(i);
        maxnz = std::max(maxnz, p->nz);
    }
    for (int z0 = 0; z0 < maxnz; z0 += zchunk)           // chunk-major over all shots
        for (int i = 0; i < n_shots; ++i) {
            const Plan *p = plans[i];
            if (z0 >= p->nz) continue;
            const int z1 = std::min(z0 + zchunk, p->nz);
            const int tiles_x = (p->nx + tx - 1) / tx, tiles_y = (p->ny + ty - 1) / ty;
            for (int by = 0; by < tiles_y; ++by)
                for (int bx = 0; bx < tiles_x; ++bx) h_items.push_back(GroupItem{i, bx, by, z0, z1});
        }
    n_items = (int)h_items.size();
    cudaError_t e;
    if (n_shots > cap_shots) {
        free_dev(d_shots);
        free_dev(d_rtm);
        d_shots = nullptr;
        d_rtm = nullptr;
        cap_shots = std::max(n_shots, 2 * cap_shots);
        if ((e = alloc(reinterpret_cast<void **>(&d_shots), sizeof(GroupShot) * cap_shots)) != cudaSuccess ||
            (e = alloc(reinterpret_cast<void **>(&d_rtm), sizeof(int) * cap_shots)) != cudaSuccess) {
            cap_shots = 0;
            return fail_cuda(e, "cudaMalloc(group shots)");
        }
    }
    n_rtm = (int)h_rtm.size();
    if (n_items > cap_items) {
        free_dev(d_items);
        d_items = nullptr;
        cap_items = std::max(n_items, 2 * cap_items);
        if ((e = alloc(reinterpret_cast<void **>(&d_items), sizeof(GroupItem) * cap_items)) != cudaSuccess) {
            cap_items = 0;
            return fail_cuda(e, "cudaMalloc(group items)");
        }
    }
    if (n_shots &&
        (e = cudaMemcpyAsync(d_shots, h_shots.data(), sizeof(GroupShot) * n_shots, cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess)
        return fail_cuda(e, "group shots upload");
    if (n_items &&
        (e = cudaMemcpyAsync(d_items, h_items.data(), sizeof(GroupItem) * n_items, cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess)
        return fail_cuda(e, "group items upload");
    if (n_rtm &&
        (e = cudaMemcpyAsync(d_rtm, h_rtm.data(), sizeof(int) * n_rtm, cudaMemcpyHostToDevice, stream)) !=
            cudaSuccess)
        return fail_cuda(e, "group migration list upload");
    // the host vectors must outlive the copies
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return fail_cuda(e, "group upload");
    return STENCIL_OK;
}

int Group::step(int k)
{
    TraceRange tr("grouped steps");
    if (n_shots == 0 || k <= 0) return STENCIL_OK;
    cudaError_t e;
    auto enqueue = [&](int steps) -> cudaError_t {
        for (int i = 0; i < steps; ++i) {
            cudaError_t r = launch_grouped(R, storage, tx, ty, d_shots, d_items, n_items, i, absorb, stream);
            if (r == cudaSuccess && n_rtm) r = launch_group_rtm(d_shots, d_rtm, n_rtm, i, stream);
            if (r != cudaSuccess) return r;
        }
        return launch_group_advance(d_shots, n_shots, steps, stream);
    };
    int left = k;
    if (graph_len > 0 && left >= graph_len) {
        if (!graph) {
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return fail_cuda(e, "cudaStreamBeginCapture");
            cudaError_t le = enqueue(graph_len);
            e = cudaStreamEndCapture(stream, &g);
            if (le != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return fail_cuda(le, "grouped launch during capture");
            }
            if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
        }
        while (left >= graph_len) {
            if ((e = cudaGraphLaunch(graph, stream)) != cudaSuccess) return fail_cuda(e, "cudaGraphLaunch");
            left -= graph_len;
        }
    }
    while (left > 0) {
        const int chunk = std::min(left, 64);
        if ((e = enqueue(chunk)) != cudaSuccess) return fail_cuda(e, "grouped launch");
        left -= chunk;
    }
    return STENCIL_OK;
}

// ---- stencil_batch_* ---------------------------------------------------------------
struct Batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Plan *> plans;
    std::vector<int64_t> n_end;
    Group group;
    bool built = false;

    void release()
    {
        if (stream) cudaStreamSynchronize(stream);
        group.release();
        for (Plan *p : plans) {
            p->release();
            delete p;
        }
        plans.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
};

}  // namespace stencil

using namespace stencil;

extern "C" {

int stencil_batch_create(const stencil_desc *descs, int32_t n, int32_t graph_steps, stencil_batch_t *out)
{
    if (!descs || !out || n < 1) return fail(STENCIL_EINVAL, "need at least one descriptor");
    if (graph_steps < 0 || (graph_steps & 1)) return fail(STENCIL_EINVAL, "graph_steps must be 0 or even");
    *out = nullptr;
    Batch *b = new Batch();
    auto bail = [&](int code) {
        b->release();
        delete b;
        return code;
    };
    cudaGetDevice(&b->dev);
    cudaError_t e;
    if (descs[0].cuda_stream) {
        b->stream = static_cast<cudaStream_t>(descs[0].cuda_stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(fail_cuda(e, "cudaStreamCreate"));
        b->own_stream = true;
    }
    const int R = descs[0].radius, storage = descs[0].storage;
    stencil_tile tile = descs[0].tile;
    if (tile.kernel == STENCIL_KERNEL_AUTO) {
        tile.kernel = STENCIL_KERNEL_TILED;
        tile.tx = 64;
        tile.ty = 16;
    }
    if (tile.kernel != STENCIL_KERNEL_TILED) return bail(fail(STENCIL_EUNSUPPORTED, "batches run the tiled kernel"));
    for (int i = 0; i < n; ++i) {
        if (descs[i].radius != R || descs[i].storage != storage)
            return bail(fail(STENCIL_EINVAL, "shot %d: every shot of a batch has the same radius and storage", i));
        stencil_desc d = descs[i];
        d.cuda_stream = b->stream;
        d.tune_mode = STENCIL_TUNE_NONE;
        d.graph_steps = 0;
        d.tile = tile;
        d.tile.zchunk = -1;
        Plan *p = nullptr;
        int rc = plan_create(&d, &p);
        if (rc) return bail(rc);
        b->plans.push_back(p);
    }
    b->group.R = R;
    b->group.storage = storage;
    b->group.tx = tile.tx;
    b->group.ty = tile.ty;
    b->group.stream = b->stream;
    b->group.graph_len = graph_steps;
    b->group.zchunk = group_zchunk(R, storage, tile.tx, tile.ty, b->plans);
    TiledInfo info{};
    tiled_config(R, storage, tile.tx, tile.ty, &info);
    if (info.zmax) b->group.zchunk = std::min(b->group.zchunk, info.zmax);
    b->n_end.assign(n, 0);
    *out = reinterpret_cast<stencil_batch_t>(b);
    return STENCIL_OK;
}

int stencil_batch_run(stencil_batch_t h, int32_t nsteps)
{
    if (!h) return fail(STENCIL_EINVAL, "null batch");
    if (nsteps < 0) return fail(STENCIL_EINVAL, "nsteps < 0");
    Batch *b = reinterpret_cast<Batch *>(h);
    cudaSetDevice(b->dev);
    // every shot's target: its current level + nsteps; the descriptors are
    // rebuilt only when the targets change
    bool changed = !b->built;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        const int64_t tgt = b->plans[i]->steps_done + nsteps;
        if (tgt != b->n_end[i]) changed = true;
        b->n_end[i] = tgt;
    }
    if (changed) {
        // n_end lives in the descriptors: refresh them in place (same
        // addresses, so a captured graph stays valid)
        Group &g = b->group;
        cudaGraphExec_t keep = g.graph;
        const void *shots_before = g.d_shots, *items_before = g.d_items;
        g.graph = nullptr;
        int rc = g.build(b->plans, b->n_end);
        if (keep) {
            if (g.d_shots == shots_before && g.d_items == items_before) g.graph = keep;
            else cudaGraphExecDestroy(keep);
        }
        if (rc) return rc;
        b->built = true;
    }
    int rc = b->group.step(nsteps);
    if (rc) return rc;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        Plan *p = b->plans[i];
        const int pb = b->group.h_shots[i].parity_base;
        p->steps_done = b->n_end[i];
        p->cur = (int)((p->steps_done + pb) & 1);
    }
    return STENCIL_OK;
}

int stencil_batch_sync(stencil_batch_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null batch");
    Batch *b = reinterpret_cast<Batch *>(h);
    cudaSetDevice(b->dev);
    for (Plan *p : b->plans) {
        int rc = p->check_device_error();
        if (rc) return rc;
    }
    return STENCIL_OK;
}

int stencil_batch_size(stencil_batch_t h, int32_t *n)
{
    if (!h || !n) return fail(STENCIL_EINVAL, "null argument");
    *n = (int32_t)reinterpret_cast<Batch *>(h)->plans.size();
    return STENCIL_OK;
}

int stencil_batch_plan(stencil_batch_t h, int32_t shot, stencil_plan_t *plan)
{
    if (!h || !plan) return fail(STENCIL_EINVAL, "null argument");
    Batch *b = reinterpret_cast<Batch *>(h);
    if (shot < 0 || shot >= (int)b->plans.size()) return fail(STENCIL_EINVAL, "shot index out of range");
    *plan = reinterpret_cast<stencil_plan_t>(b->plans[shot]);
    return STENCIL_OK;
}

int stencil_batch_zchunk(stencil_batch_t h, int32_t *zchunk)
{
    if (!h || !zchunk) return fail(STENCIL_EINVAL, "null argument");
    *zchunk = reinterpret_cast<Batch *>(h)->group.zchunk;
    return STENCIL_OK;
}

int stencil_batch_destroy(stencil_batch_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null batch");
    Batch *b = reinterpret_cast<Batch *>(h);
    cudaSetDevice(b->dev);
    b->release();
    delete b;
    return STENCIL_OK;
}

}  // extern "C"
