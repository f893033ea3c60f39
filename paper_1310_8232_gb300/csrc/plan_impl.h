// The plan object behind stencil_plan_t, shared by the runtime translation units.
#pragma once

#include <vector>
#include <cmath>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "stencil.h"

namespace stencil {

int fail(int code, const char *fmt, ...);
int fail_cuda(cudaError_t e, const char *what);
double cfl_limit(int R);
int64_t row_pitch(int nx, int esize);
int encode_map(CUtensorMap *m, const void *base, int nx, int ny, int nz, int64_t pitch, int esize, int bw, int bh);
// the same with an explicit plane stride (elements), for a view of some rows
// of every plane
int encode_map_strided(CUtensorMap *m, const void *base, int nx, int ny, int nz, int64_t pitch, int64_t plane,
                       int esize, int bw, int bh);
// Grids of at most this many points get the naive kernel by default (FP32).
constexpr int64_t NAIVE_MAX_POINTS = 1 << 20;
stencil_tile default_tile(int R, int storage, int nx, int ny, int nz);
int choose_zchunk(int R, int storage, int tx, int ty, int nx, int ny, int nz);
int choose_zchunk_two_step(int R, int nx, int ny, int nz);
int check_tile(int R, int storage, const stencil_tile &t);
extern thread_local std::string g_last_error;

// NVTX range for the lifetime of a scope (host-side phases: plan set-up,
// step enqueue, tile selection, engine iterations); free when no profiler
// is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Row-by-row copy between pitched layouts; one flat copy when both sides
// are dense (a 2D copy of many short rows is much slower than a flat one).
inline cudaError_t memcpy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t row_bytes,
                               size_t rows, cudaMemcpyKind kind, cudaStream_t s)
{
    if (dpitch == row_bytes && spitch == row_bytes) return cudaMemcpyAsync(dst, src, row_bytes * rows, kind, s);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row_bytes, rows, kind, s);
}

struct Plan {
    int dev = 0;
    cudaMemPool_t pool = nullptr;         // set: stream-ordered allocations from this pool
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int R = 5;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dt = 0;
    int64_t pitch = 0;                    // row pitch in elements (wavefields and kappa)
    int64_t field_elems = 0;
    int storage = STENCIL_FP32;
    int esize = 4;                        // bytes per wavefield element
    // FP32: buf[cur] = u^n, buf[cur ^ 1] = u^{n-1} (overwritten by u^{n+1});
    // 16-bit: buf[cur] = u^n, buf[cur ^ 1] receives u^{n+1}, and dbuf holds
    // d^n = u^n - u^{n-1} (rewritten in place by each step)
    void *buf[2] = {nullptr, nullptr};
    void *dbuf = nullptr;
    // two-step kernel: two more FP32 levels; the levels live in one pair of
    // the four buffers B = (buf[0], buf[1], tbuf[0], tbuf[1]), pair t2_pair:
    // u^{n-1} = B[2 t2_pair], u^n = B[2 t2_pair + 1] (swapped when t2_swapped)
    void *tbuf[2] = {nullptr, nullptr};
    int t2_pair = 0;
    bool t2_swapped = false;
    int t2_plain_zchunk = 0;              // z-chunk of the one-step launches (64 x 16 tile)
    bool user_owned = false;              // buf and kappa belong to the caller (not freed)
    float *kappa = nullptr;
    float *staging[2] = {nullptr, nullptr};   // 16-bit storage: FP32 copies for state transfer
    // 16-bit storage: [4][nz] per-plane scales and max |.| by level mod 4, of u and of d
    float *d_scale = nullptr;
    unsigned *d_amax = nullptr;
    float *d_scale_d = nullptr;
    unsigned *d_amax_d = nullptr;
    float growth = 0, src_bound = 0;      // kappa_max * 3W; |source amplitude|
    int cur = 0;
    void *d_scratch = nullptr;
    int64_t *d_step = nullptr;
    int *d_err = nullptr;
    unsigned *d_vmax = nullptr;
    unsigned long long *d_bad = nullptr;
    double *d_partials = nullptr;
    double *d_result = nullptr;
    int64_t device_bytes = 0;
    int64_t steps_done = 0;
    double vmax = 0, cfl = 0, cfl_lim = 0;
    bool velocity_ok = false;
    double src_amp = 0;
    Source src{};
    stencil_tile tile{};
    CUtensorMap maps_halo[2];
    CUtensorMap maps_core[2];
    CUtensorMap map_kcore;
    // two-step kernel: its boxes of each of the four buffers, kappa's, and the
    // one-step kernel's (64 x 16 tile) for an odd last step
    CUtensorMap t2_u_halo[4], t2_up_region[4], t2_u_core[4], t2_plain_halo[4], t2_plain_core[4];
    CUtensorMap t2_k_region, t2_k_core;
    int graph_len = 0;
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    // recording (receiver traces, per-step energy); off when rec_mem is null
    void *rec_mem = nullptr;
    float *rec = nullptr;
    double *rec_energy = nullptr, *rec_part = nullptr;
    unsigned *rec_count = nullptr;
    int64_t rec_n0 = 0;
    int rec_cap = 0, rec_z = -1, rec_y = -1, rec_energy_on = 0;
    // absorbing layer and plane injection
    int absorb_w = 0;
    float absorb_eta = 0.0f;
    int64_t absorb_shell = 0;
    float *absorb_save = nullptr;
    float2 *absorb_tab = nullptr;         // device (g_d, h_d), d = 0..W, after the saved values
    std::vector<float2> absorb_tab_host;
    // failure-path testing (stencil_debug_wait_fault)
    uint32_t fault_tx = 0, wait_ns = 0;
    const float *inj = nullptr;
    int64_t inj_n0 = 0;
    int inj_steps = 0, inj_reverse = 0, inj_z = -1, inj_y = -1;
    float inj_scale = 0.0f;
    // tile selection results
    // a served migration's per-step work in grouped launches (phase 0: none)
    GroupRtm rtm{};
    int tune_mode = 0;
    double min_time_ms = NAN, actual_time_ms = NAN, full_time_ms = NAN, quality = NAN, selection_ms = NAN;
    int n_candidates = 0;

    cudaError_t dev_alloc(void **ptr, size_t bytes);
    void dev_free(void *ptr);
    char *bptr(int b, int64_t off_elems) const { return static_cast<char *>(buf[b]) + off_elems * esize; }
    // what the sweep reads beside kappa, point by point, when u^n is in
    // buf[parity]: u^{n-1} (FP32) or d^n (16-bit)
    char *aux_ptr(int parity, int64_t off_elems) const
    {
        return storage == STENCIL_FP32 ? bptr(parity ^ 1, off_elems)
                                       : static_cast<char *>(dbuf) + off_elems * esize;
    }
    int ensure_staging();
    // FP32 view of level n - which (the field itself for FP32 storage, an
    // unpacked copy in staging[which] for 16-bit storage); enqueued on stream
    int fp32_level(int which, const float **out);
    // the buffer holding u^{n - which} (which = 0, 1)
    void *level_buf(int which) const;
    int build_maps();
    // two-step kernel (plan_two_step.cu)
    void *t2_buf(int k) const { return k < 2 ? buf[k] : tbuf[k - 2]; }
    int build_maps_two_step();
    cudaError_t launch_two_step_pair(int step_off, cudaStream_t s);
    cudaError_t launch_two_step_single(int step_off, cudaStream_t s);
    int enqueue_two_step(int nsteps);
    int capture_graphs_two_step();
    int load_velocity(const float *v, int on_device);
    SweepParams params(int parity, int step_off) const;
    cudaError_t launch_one(int parity, int step_off, cudaStream_t s) const;
    StepOps step_ops(int step_off) const;
    bool has_step_ops() const;
    // the absorbing layer runs inside the sweep (tiled kernel, FP32 storage)
    bool absorb_folded() const;
    int enqueue_eager(int nsteps);
    int enqueue(int nsteps);
    int capture_graphs();
    void drop_graphs();
    int check_device_error();
    void release();
};

// Build a plan; with a pool, every device allocation of the plan is
// stream-ordered from it (no device-wide synchronisation on free).
int plan_create(const stencil_desc *d, Plan **out, cudaMemPool_t pool = nullptr);

// Tile selection (Sec. 3.2-3.3 on GPU tile parameters); sets p->tile.
int tune_plan(Plan *p, const stencil_desc *d);

}  // namespace stencil
