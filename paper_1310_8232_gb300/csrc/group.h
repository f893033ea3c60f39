// Grouped execution of many plans (shots) in one launch per time step: the
// engine behind stencil_batch_* and the shot server.
#pragma once

#include <vector>

#include "plan_impl.h"

namespace stencil {

struct Group {
    int R = 5, storage = 0, tx = 64, ty = 16, zchunk = 32;
    bool absorb = false;            // some shot has an absorbing layer: the absorbing variant
    cudaStream_t stream = nullptr;
    // set: the device tables come from this stream-ordered pool on `stream`
    // (no device-wide synchronisation when they grow, as cudaFree would do)
    cudaMemPool_t pool = nullptr;
    GroupShot *d_shots = nullptr;
    GroupItem *d_items = nullptr;
    int *d_rtm = nullptr;           // indices of the shots with migration work (GroupRtm)
    int cap_shots = 0, cap_items = 0;
    int n_shots = 0, n_items = 0, n_rtm = 0;
    std::vector<GroupShot> h_shots;
    std::vector<GroupItem> h_items;
    std::vector<int> h_rtm;
    int graph_len = 0;
    cudaGraphExec_t graph = nullptr;

    ~Group() { release(); }
    void release();
    cudaError_t alloc(void **p, size_t bytes);
    void free_dev(void *p);
    // Describe `plans` (same radius, storage and tile shape) to the device;
    // shot i stops when its counter reaches n_end[i].  Enqueued on stream.
    int build(const std::vector<Plan *> &plans, const std::vector<int64_t> &n_end);
    // Enqueue k steps of every shot (k grouped launches + one counter advance),
    // through a captured graph of graph_len steps where k allows.
    int step(int k);
};

// A common z-chunk for the blocks of several grids sharing the GPU; `share`
// is the fraction of the GPU's block slots the group can expect (1 when it
// runs alone, less when other groups run beside it).
int group_zchunk(int R, int storage, int tx, int ty, const std::vector<Plan *> &plans, double share = 1.0);

}  // namespace stencil
