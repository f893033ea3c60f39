// Shot server: continuous batching of independent shots on one GPU.
//
// Requests (a problem description, a step count and a host output buffer)
// arrive at any time through shot_submit.  One engine thread admits queued
// shots in arrival order while a slot is free and the projected device bytes
// fit under the memory budget, and keeps every admitted shot's wavefields
// resident.  Resident shots are split by size (points per time step) into
// lanes; each lane advances its shots together, chunk_steps time steps per
// chunk, with the grouped kernel (one launch per step over all its shots'
// tiles) on a stream of its own, the lanes of smaller shots on streams of
// higher priority.  A lane starts its next chunk as soon as its previous one
// has finished (and queues it behind the running one when no shot can join
// or leave in between), independently of the other lanes, so a small shot is not
// held to the step rate of the largest resident one, and the block scheduler
// serves the small shots' blocks first while the large shots fill the rest
// of the GPU.  New shots' plans are made on an admission stream while the
// lanes run; a shot joins its lane when the lane's current chunk ends.
// Shots that reach their step count retire: the final field is copied to the
// caller's buffer and the shot's memory is freed by a second thread on its
// own stream, and the slot goes to the next request.  Device memory comes
// from a server-owned stream-ordered pool, so neither admission nor
// retirement synchronises the whole device.  shot_poll reports state and
// timing without blocking.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "group.h"

namespace stencil {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    stencil_desc desc{};
    std::vector<float> velocity;      // host copy (desc.velocity points here unless on device)
    int32_t nsteps = 0;
    float *out_host = nullptr;
    int state = SHOT_QUEUED;
    int status = STENCIL_OK;
    double t_submit = -1, t_admit = -1, t_done = -1;
    int64_t steps_done = 0;
    int64_t bytes = 0;
    Plan *plan = nullptr;
    // a served migration (shot_submit_rtm): phase 0 forward, 1 backward
    bool rtm = false;
    shot_rtm_cfg rtm_cfg{};
    float *image_host = nullptr, *traces_host = nullptr;
    int phase = 0;
    float *d_rtm = nullptr;           // traces | snapshots | image, one pool allocation
};

// Device bytes of a migration's traces, snapshots and image (dense FP32).
int64_t rtm_bytes(const stencil_desc &d, int32_t nsteps, const shot_rtm_cfg &c)
{
    const int64_t pts = (int64_t)d.nx * d.ny * d.nz;
    const int64_t rows = c.receiver_y < 0 ? d.ny : 1;
    return 4 * ((int64_t)nsteps * rows * d.nx + (int64_t)(nsteps / c.snap_every) * pts + pts);
}

int64_t projected_bytes(const stencil_desc &d)
{
    const int esize = d.storage == STENCIL_FP32 ? 4 : 2;
    const int64_t elems = row_pitch(d.nx, esize) * d.ny * d.nz;
    // two wavefield levels and kappa; 16-bit storage adds the difference
    // field, its FP32 staging for the final read-back and the scale tables
    int64_t b = elems * (2 * esize + 4) + 64 * 1024 + 32LL * d.nz;
    if (d.storage != STENCIL_FP32) b += elems * esize + 2 * elems * 4 + 64LL * d.nz;
    return b;
}

}  // namespace

// Shots of one size class, stepped together on one stream.
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t done[2] = {nullptr, nullptr}; // recorded after each chunk (ring of the chunks in flight)
    Group group;
    std::vector<Request *> resident;          // in the lane's group
    std::vector<Request *> joining;           // admitted, join at the next chunk
    bool rebuild = false;
    int head = 0, n_flight = 0;               // oldest chunk in flight, chunks in flight (0 .. 2)
    int step_rc[2] = {STENCIL_OK, STENCIL_OK};
};

// Lane of a shot: lane k holds shots of [2^(21+2(k-1)), 2^(21+2k)) points
// (below 2 M points in lane 0; the last lane takes everything above).
static int lane_of(const stencil_desc &d, int lanes)
{
    const int64_t points = (int64_t)d.nx * d.ny * d.nz;
    int k = 0;
    for (int64_t t = int64_t(1) << 21; k < lanes - 1 && points >= t; t <<= 2) ++k;
    return k;
}

struct Server {
    shot_server_cfg cfg{};
    int dev = 0;
    cudaStream_t retire_stream = nullptr;
    cudaStream_t admit_stream = nullptr;      // plan creation, overlapping the engine's steps
    cudaMemPool_t pool = nullptr;
    int64_t budget = 0;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_ticket = 1;
    bool stopping = false;
    shot_server_stats stats{};

    std::vector<std::unique_ptr<Lane>> lanes; // engine thread only (after creation)
    uint64_t wake_seq = 0;                    // bumped (under mu) when a lane's chunk ends
    std::thread engine;
    int engine_error = STENCIL_OK;

    // retirement: read-back and free on the retire thread
    std::deque<std::pair<Request *, int>> retire_q;
    bool retire_stop = false;
    std::thread retirer;
    static constexpr size_t BOUNCE_BYTES = 32u << 20;
    float *bounce[2] = {nullptr, nullptr};    // pinned host halves for read-back
    cudaEvent_t bounce_ev[2] = {nullptr, nullptr};
    int read_back(Plan *p, float *out);

    ~Server();
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    int launch_lane(Lane &L);                 // (re)describe the lane if needed, enqueue its next chunk
    void end_chunk(Lane &L, int rc);          // account the finished chunk, retire finished shots
    void retire_loop();
    void retire(Request *r, int status);      // hand a shot to the retire thread
    void finish(Request *r, int status);      // retire thread: read back, free, report
};

// Everything the server holds on the device or host (the engine and retire
// threads have ended, or never started); safe on a partly created server.
Server::~Server()
{
    cudaSetDevice(dev);
    for (auto &L : lanes) {
        if (L->stream) cudaStreamSynchronize(L->stream);
        L->group.release();
        for (cudaEvent_t ev : L->done)
            if (ev) cudaEventDestroy(ev);
        if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
    }
    for (cudaStream_t st : {retire_stream, admit_stream}) {
        if (!st) continue;
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (int k = 0; k < 2; ++k) {
        if (bounce[k]) cudaFreeHost(bounce[k]);
        if (bounce_ev[k]) cudaEventDestroy(bounce_ev[k]);
    }
    if (pool) cudaMemPoolDestroy(pool);
}

void Server::retire(Request *r, int status)
{
    std::lock_guard<std::mutex> lock(mu);
    retire_q.emplace_back(r, status);
    cv.notify_all();
}

void Server::retire_loop()
{
    cudaSetDevice(dev);
    for (;;) {
        std::pair<Request *, int> job;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv.wait(lock, [&] { return retire_stop || !retire_q.empty(); });
            if (retire_q.empty()) return;       // stop requested and nothing left
            job = retire_q.front();
            retire_q.pop_front();
        }
        finish(job.first, job.second);
    }
}

// Host copy of n bytes split over a few threads (one core copies ~14 GB/s,
// far below the device-to-host link).
static void parallel_copy(void *dst, const void *src, size_t n)
{
    constexpr size_t SLICE = 8u << 20;
    const int parts = (int)std::min<size_t>(4, std::max<size_t>(1, n / SLICE));
    if (parts == 1) {
        std::memcpy(dst, src, n);
        return;
    }
    const size_t per = (n / parts + 63) & ~size_t(63);
    std::vector<std::thread> helpers;
    for (int k = 1; k < parts; ++k) {
        const size_t o = std::min(n, per * k), len = std::min(n, o + per) - o;
        helpers.emplace_back([=] { std::memcpy(static_cast<char *>(dst) + o, static_cast<const char *>(src) + o, len); });
    }
    std::memcpy(dst, src, std::min(n, per));
    for (auto &t : helpers) t.join();
}

// u^N of a finished shot into the caller's dense buffer.  A page-locked
// buffer takes one device-to-host copy.  Any other goes through the pinned
// bounce halves (the device-to-pinned copy of chunk k overlaps the host copy
// of chunk k-1): a device-to-host copy straight into pageable memory that
// the process has not touched yet faults its pages in one by one on the
// driver's side, and measured an order of magnitude slower under load.
int Server::read_back(Plan *p, float *out)
{
    const float *src = nullptr;
    int rc = p->fp32_level(0, &src);
    if (rc) return rc;
    const size_t row_bytes = (size_t)p->nx * sizeof(float);
    const int64_t rows = (int64_t)p->ny * p->nz;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeHost) {
        cudaError_t e = memcpy_rows(out, row_bytes, src, p->pitch * sizeof(float), row_bytes, (size_t)rows,
                                    cudaMemcpyDeviceToHost, retire_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(retire_stream);
        return e == cudaSuccess ? STENCIL_OK : fail_cuda(e, "read-back");
    }
    cudaGetLastError();                         // an unregistered pointer is not an error here
    const int64_t per = std::max<int64_t>(1, (int64_t)(BOUNCE_BYTES / row_bytes));
    int64_t prev_r0 = -1, prev_n = 0;
    int k = 0;
    for (int64_t r0 = 0; r0 < rows; r0 += per, ++k) {
        const int64_t n = std::min(per, rows - r0);
        cudaError_t e = memcpy_rows(bounce[k & 1], row_bytes, src + r0 * p->pitch, p->pitch * sizeof(float),
                                    row_bytes, (size_t)n, cudaMemcpyDeviceToHost, retire_stream);
        if (e == cudaSuccess) e = cudaEventRecord(bounce_ev[k & 1], retire_stream);
        if (e != cudaSuccess) return fail_cuda(e, "read-back");
        if (prev_r0 >= 0) {
            if ((e = cudaEventSynchronize(bounce_ev[(k - 1) & 1])) != cudaSuccess) return fail_cuda(e, "read-back");
            parallel_copy(out + prev_r0 * p->nx, bounce[(k - 1) & 1], (size_t)prev_n * row_bytes);
        }
        prev_r0 = r0;
        prev_n = n;
    }
    if (prev_r0 >= 0) {
        cudaError_t e = cudaEventSynchronize(bounce_ev[(k - 1) & 1]);
        if (e != cudaSuccess) return fail_cuda(e, "read-back");
        parallel_copy(out + prev_r0 * p->nx, bounce[(k - 1) & 1], (size_t)prev_n * row_bytes);
    }
    return STENCIL_OK;
}

void Server::finish(Request *r, int status)
{
    TraceRange tr("retire shot");
    const auto f0 = Clock::now();
    int rc = status;
    if (r->plan) {
        // the engine has synchronised its stream after the shot's last step;
        // from here on the shot's plan works on the retire stream
        r->plan->stream = retire_stream;
        r->plan->own_stream = false;
        if (rc == STENCIL_OK && r->out_host) rc = read_back(r->plan, r->out_host);
        if (r->d_rtm) {
            // a migration: the image (and the traces) are dense on the device
            const stencil_desc &d = r->desc;
            const int64_t pts = (int64_t)d.nx * d.ny * d.nz;
            const int64_t tr = (int64_t)r->nsteps * (r->rtm_cfg.receiver_y < 0 ? d.ny : 1) * d.nx;
            const float *image = r->d_rtm + tr + (int64_t)(r->nsteps / r->rtm_cfg.snap_every) * pts;
            cudaError_t e = cudaSuccess;
            if (rc == STENCIL_OK && r->image_host)
                e = cudaMemcpyAsync(r->image_host, image, sizeof(float) * pts, cudaMemcpyDeviceToHost, retire_stream);
            if (rc == STENCIL_OK && e == cudaSuccess && r->traces_host)
                e = cudaMemcpyAsync(r->traces_host, r->d_rtm, sizeof(float) * tr, cudaMemcpyDeviceToHost,
                                    retire_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(retire_stream);
            if (e != cudaSuccess && rc == STENCIL_OK) rc = fail_cuda(e, "migration read-back");
            cudaFreeAsync(r->d_rtm, retire_stream);
            r->d_rtm = nullptr;
        }
        r->plan->release();
        delete r->plan;
        r->plan = nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    stats.retire_s += std::chrono::duration<double>(Clock::now() - f0).count();
    r->state = rc == STENCIL_OK ? SHOT_DONE : SHOT_FAILED;
    r->status = rc;
    r->t_done = now();
    stats.bytes_in_use -= r->bytes;
    stats.running -= 1;
    if (rc == STENCIL_OK) {
        stats.done += 1;
        stats.point_updates += (int64_t)r->desc.nx * r->desc.ny * r->desc.nz * r->nsteps * (r->rtm ? 2 : 1);
    } else {
        stats.failed += 1;
    }
    cv.notify_all();
}

static void CUDART_CB wake_engine(void *arg)
{
    // host callback at the end of a lane's chunk: no CUDA calls here
    Server *s = static_cast<Server *>(arg);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->wake_seq += 1;
    }
    s->cv.notify_all();
}

int Server::launch_lane(Lane &L)
{
    if (L.rebuild) {
        const auto b0 = Clock::now();
        std::vector<Plan *> plans;
        std::vector<int64_t> n_end;
        for (Request *r : L.resident) {
            plans.push_back(r->plan);
            n_end.push_back(r->nsteps);
        }
        // the lanes with shots share the GPU's block slots
        int active = 0;
        for (auto &lp : lanes) active += !lp->resident.empty() || !lp->joining.empty();
        L.group.zchunk = group_zchunk(L.group.R, L.group.storage, L.group.tx, L.group.ty, plans,
                                      1.0 / std::max(1, active));
        TiledInfo info{};
        tiled_config(L.group.R, L.group.storage, L.group.tx, L.group.ty, &info);
        if (info.zmax) L.group.zchunk = std::min(L.group.zchunk, info.zmax);
        const int rc = L.group.build(plans, n_end);
        {
            std::lock_guard<std::mutex> lock(mu);
            stats.build_s += std::chrono::duration<double>(Clock::now() - b0).count();
        }
        if (rc) return rc;
        L.rebuild = false;
    }
    const int k = (L.head + L.n_flight) & 1;
    L.step_rc[k] = L.group.step(cfg.chunk_steps);
    cudaError_t e = cudaEventRecord(L.done[k], L.stream);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(L.stream, wake_engine, this);
    if (e != cudaSuccess && L.step_rc[k] == STENCIL_OK) L.step_rc[k] = fail_cuda(e, "lane chunk");
    L.n_flight += 1;
    return STENCIL_OK;
}

void Server::end_chunk(Lane &L, int rc)
{
    if (rc != STENCIL_OK && L.n_flight > 1) {
        // the chunk queued behind the failed one still uses the shots' memory
        cudaStreamSynchronize(L.stream);
        L.n_flight = 1;
    }
    std::vector<Request *> keep;
    for (size_t i = 0; i < L.resident.size(); ++i) {
        Request *r = L.resident[i];
        Plan *p = r->plan;
        const int pb = L.group.h_shots[i].parity_base;
        p->steps_done = std::min<int64_t>(p->steps_done + cfg.chunk_steps, r->nsteps);
        p->cur = (int)((p->steps_done + pb) & 1);
        {
            std::lock_guard<std::mutex> lock(mu);
            r->steps_done = (int64_t)r->phase * r->nsteps + p->steps_done;
        }
        if (rc != STENCIL_OK) {
            retire(r, rc);
            L.rebuild = true;
        } else if (p->steps_done >= r->nsteps && r->rtm && r->phase == 0) {
            // a migration's forward phase is done: the same plan goes back
            // in time from zero fields without its point source (no chunk of
            // this lane is in flight behind this one, see run())
            const size_t fbytes = (size_t)p->field_elems * p->esize;
            cudaError_t e = cudaMemsetAsync(p->buf[0], 0, fbytes, L.stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->buf[1], 0, fbytes, L.stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(p->d_step, 0, sizeof(int64_t), L.stream);
            if (e != cudaSuccess) {
                retire(r, fail_cuda(e, "migration backward set-up"));
            } else {
                r->phase = 1;
                p->src.on = 0;
                p->rtm.phase = 2;
                p->steps_done = 0;
                p->cur = 0;
                keep.push_back(r);
            }
            L.rebuild = true;
        } else if (p->steps_done >= r->nsteps) {
            retire(r, p->check_device_error());
            L.rebuild = true;
        } else {
            keep.push_back(r);
        }
    }
    L.resident.swap(keep);
    L.head ^= 1;
    L.n_flight -= 1;
    std::lock_guard<std::mutex> lock(mu);
    stats.iterations += 1;
}

void Server::run()
{
    cudaSetDevice(dev);
    int in_flight = 0;                        // lanes with a chunk on the GPU
    Clock::time_point busy_t0{};
    uint64_t seen_wake = 0;
    for (;;) {
        // ---- every idle lane with shots starts its next chunk; a lane whose
        //      membership cannot change before its running chunk ends queues
        //      the chunk after it too, so the GPU does not wait for the host
        for (auto &lp : lanes) {
            Lane &L = *lp;
            if (L.n_flight == 0) {
                if (!L.joining.empty()) {
                    for (Request *r : L.joining) L.resident.push_back(r);
                    L.joining.clear();
                    L.rebuild = true;
                }
                if (L.resident.empty()) continue;
                const int rc = launch_lane(L);
                if (rc) {
                    engine_error = rc;
                    for (Request *r : L.resident) retire(r, rc);
                    L.resident.clear();
                    continue;
                }
            }
            if (L.n_flight == 1 && L.joining.empty() && !L.rebuild && L.step_rc[L.head] == STENCIL_OK) {
                bool finishing = false;              // a shot ends within the running chunk
                for (Request *r : L.resident) finishing |= r->plan->steps_done + cfg.chunk_steps >= r->nsteps;
                if (!finishing) launch_lane(L);
            }
        }

        {
            int busy_now = 0;
            for (auto &lp : lanes) busy_now += lp->n_flight > 0;
            if (in_flight == 0 && busy_now > 0) busy_t0 = Clock::now();
            in_flight = busy_now;
        }

        // ---- admission (plans made on the admission stream) ----------------
        int slots_used = 0;
        for (auto &lp : lanes) slots_used += (int)(lp->resident.size() + lp->joining.size());
        std::vector<Request *> admit;
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stopping) {
                for (Request *r : queue) {
                    r->state = SHOT_FAILED;
                    r->status = STENCIL_ECANCELLED;
                    r->t_done = now();
                    stats.queued -= 1;
                    stats.failed += 1;
                }
                queue.clear();
                if (slots_used == 0 && in_flight == 0) {
                    cv.notify_all();
                    return;
                }
            }
            while (!queue.empty() && slots_used + (int)admit.size() < cfg.max_slots &&
                   stats.bytes_in_use + queue.front()->bytes <= budget) {
                Request *r = queue.front();
                queue.pop_front();
                stats.bytes_in_use += r->bytes;
                stats.queued -= 1;
                stats.running += 1;
                r->state = SHOT_RUNNING;
                admit.push_back(r);
            }
        }
        TraceRange tr_it("engine iteration");
        for (Request *r : admit) {
            const auto a0 = Clock::now();
            stencil_desc d = r->desc;
            d.cuda_stream = admit_stream;
            d.tune_mode = STENCIL_TUNE_NONE;
            d.graph_steps = 0;
            d.storage = cfg.storage;
            d.radius = cfg.radius;
            d.tile = stencil_tile{STENCIL_KERNEL_TILED, lanes[0]->group.tx, lanes[0]->group.ty, -1};
            Plan *p = nullptr;
            const int arc = plan_create(&d, &p, pool);   // synchronous on the admission stream
            {
                std::lock_guard<std::mutex> lock(mu);
                r->t_admit = now();
                stats.admitted += 1;
                stats.admit_s += std::chrono::duration<double>(Clock::now() - a0).count();
            }
            if (arc) {
                retire(r, arc);
                continue;
            }
            if (r->rtm) {
                // the migration's traces, snapshots and image (zeroed), from the pool
                const stencil_desc &dd = r->desc;
                const int64_t pts = (int64_t)dd.nx * dd.ny * dd.nz;
                const int64_t tr = (int64_t)r->nsteps * (r->rtm_cfg.receiver_y < 0 ? dd.ny : 1) * dd.nx;
                const int64_t ns = r->nsteps / r->rtm_cfg.snap_every;
                cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r->d_rtm),
                                                        rtm_bytes(dd, r->nsteps, r->rtm_cfg), pool, admit_stream);
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(r->d_rtm + tr + ns * pts, 0, sizeof(float) * pts, admit_stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(admit_stream);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    r->plan = p;
                    retire(r, fail(STENCIL_ENOMEM, "migration buffers: %s", cudaGetErrorString(e)));
                    continue;
                }
                p->rtm.phase = 1;
                p->rtm.z = r->rtm_cfg.receiver_z;
                p->rtm.y = r->rtm_cfg.receiver_y;
                p->rtm.T = r->nsteps;
                p->rtm.k = r->rtm_cfg.snap_every;
                p->rtm.image_scale = r->rtm_cfg.image_scale;
                p->rtm.traces = r->d_rtm;
                p->rtm.snaps = r->d_rtm + tr;
                p->rtm.image = r->d_rtm + tr + ns * pts;
            }
            Lane &L = *lanes[lane_of(r->desc, (int)lanes.size())];
            p->stream = L.stream;               // the lane's stream from here on
            r->plan = p;
            r->velocity.clear();
            r->velocity.shrink_to_fit();
            L.joining.push_back(r);
        }

        // ---- lanes whose chunk has ended: account and retire ---------------
        bool ended = false;
        for (auto &lp : lanes) {
            Lane &L = *lp;
            while (L.n_flight > 0) {
                const cudaError_t e = cudaEventQuery(L.done[L.head]);
                if (e == cudaErrorNotReady) break;
                int rc = L.step_rc[L.head];
                if (rc == STENCIL_OK && e != cudaSuccess) rc = fail_cuda(e, "lane chunk");
                end_chunk(L, rc);
                ended = true;
            }
        }
        int busy_now = 0;
        for (auto &lp : lanes) busy_now += lp->n_flight > 0;
        if (in_flight > 0 && busy_now == 0) {
            std::lock_guard<std::mutex> lock(mu);
            stats.busy_s += std::chrono::duration<double>(Clock::now() - busy_t0).count();
        }
        in_flight = busy_now;
        if (ended || !admit.empty()) continue;   // idle lanes may start at once

        // ---- nothing to do until a chunk ends, a shot arrives or memory frees
        int joining = 0;
        for (auto &lp : lanes) joining += lp->n_flight ? 0 : (int)lp->joining.size();
        if (joining) continue;
        std::unique_lock<std::mutex> lock(mu);
        cv.wait_for(lock, std::chrono::milliseconds(in_flight ? 2 : 20), [&] {
            return (stopping && in_flight == 0) || wake_seq != seen_wake ||
                   (!queue.empty() && slots_used < cfg.max_slots &&
                    stats.bytes_in_use + queue.front()->bytes <= budget);
        });
        seen_wake = wake_seq;
    }
}

}  // namespace stencil


using namespace stencil;

extern "C" {

void shot_server_cfg_init(shot_server_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->hbm_budget_frac = 0.8;
    c->max_slots = 64;
    c->chunk_steps = 20;
    c->radius = 5;
    c->storage = STENCIL_FP32;
    c->tile.kernel = STENCIL_KERNEL_AUTO;
    c->lanes = 3;
}

int shot_server_create(const shot_server_cfg *cfg, shot_server_t *out)
{
    if (!cfg || !out) return fail(STENCIL_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->radius != 4 && cfg->radius != 5) return fail(STENCIL_EINVAL, "radius must be 4 or 5");
    if (cfg->max_slots < 1 || cfg->chunk_steps < 1) return fail(STENCIL_EINVAL, "max_slots, chunk_steps >= 1");
    if (cfg->lanes < 1 || cfg->lanes > 6) return fail(STENCIL_EINVAL, "lanes must be 1 .. 6");
    if (!(cfg->hbm_budget_frac > 0) && cfg->hbm_budget_bytes <= 0)
        return fail(STENCIL_EINVAL, "need a memory budget");
    if (cfg->storage != STENCIL_FP32 && cfg->storage != STENCIL_FP16 && cfg->storage != STENCIL_BF16)
        return fail(STENCIL_EINVAL, "bad storage");
    auto s = std::make_unique<Server>();
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STENCIL_ENODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return fail_cuda(e, "cudaMemGetInfo");
    // a share of the memory free now, not of the device's total: on a GPU
    // that other work also uses, the budget stays within what exists
    s->budget = cfg->hbm_budget_bytes > 0 ? cfg->hbm_budget_bytes
                                          : (int64_t)(cfg->hbm_budget_frac * (double)free_b);
    stencil_tile t = cfg->tile;
    if (t.kernel == STENCIL_KERNEL_AUTO) t = stencil_tile{STENCIL_KERNEL_TILED, 64, 16, 0};
    if (t.kernel != STENCIL_KERNEL_TILED) return fail(STENCIL_EUNSUPPORTED, "the server runs the tiled kernel");
    TiledInfo info;
    if (!tiled_config(cfg->radius, cfg->storage, t.tx, t.ty, &info))
        return fail(STENCIL_EUNSUPPORTED, "tile %dx%d not built", t.tx, t.ty);
    // lanes: one on the caller's stream, else cfg->lanes on streams of
    // decreasing priority (lane 0, the smallest shots, highest)
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    const int nl = cfg->cuda_stream ? 1 : cfg->lanes;
    for (int k = 0; k < nl; ++k) {
        auto L = std::make_unique<Lane>();
        if (cfg->cuda_stream) {
            L->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
        } else {
            const int prio = std::min(prio_least, prio_greatest + k);
            if ((e = cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, prio)) != cudaSuccess)
                return fail_cuda(e, "cudaStreamCreateWithPriority");
            L->own_stream = true;
        }
        if ((e = cudaEventCreateWithFlags(&L->done[0], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&L->done[1], cudaEventDisableTiming)) != cudaSuccess) {
            if (L->done[0]) cudaEventDestroy(L->done[0]);
            if (L->own_stream) cudaStreamDestroy(L->stream);
            return fail_cuda(e, "cudaEventCreate");
        }
        L->group.R = cfg->radius;
        L->group.storage = cfg->storage;
        L->group.tx = t.tx;
        L->group.ty = t.ty;
        L->group.stream = L->stream;
        L->group.graph_len = 0;
        s->lanes.push_back(std::move(L));
    }
    if ((e = cudaStreamCreateWithFlags(&s->retire_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return fail_cuda(e, "cudaStreamCreate(retire)");
    // admission sits on the path of every new shot: highest priority
    if ((e = cudaStreamCreateWithPriority(&s->admit_stream, cudaStreamNonBlocking, prio_greatest)) != cudaSuccess)
        return fail_cuda(e, "cudaStreamCreate(admission)");
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->dev;
    if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return fail_cuda(e, "cudaMemPoolCreate");
    for (int k = 0; k < 2; ++k)
        if ((e = cudaMallocHost(reinterpret_cast<void **>(&s->bounce[k]), Server::BOUNCE_BYTES)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->bounce_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return fail_cuda(e, "pinned read-back buffers");
    uint64_t keep = (uint64_t)s->budget;                 // keep freed memory for the next shots
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (auto &L : s->lanes) L->group.pool = s->pool;    // group tables without device-wide syncs
    s->stats.budget_bytes = s->budget;
    s->t0 = Clock::now();
    Server *raw = s.get();
    s->engine = std::thread([raw] { raw->run(); });
    s->retirer = std::thread([raw] { raw->retire_loop(); });
    *out = reinterpret_cast<shot_server_t>(s.release());
    return STENCIL_OK;
}

static int submit(shot_server_t h, const stencil_desc *d, int32_t nsteps, float *out_host, const shot_rtm_cfg *rtm,
                  float *image_host, float *traces_host, uint64_t *ticket);

int shot_submit(shot_server_t h, const stencil_desc *d, int32_t nsteps, float *out_host, uint64_t *ticket)
{
    return submit(h, d, nsteps, out_host, nullptr, nullptr, nullptr, ticket);
}

void shot_rtm_cfg_init(shot_rtm_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->receiver_y = -1;
    c->snap_every = 10;
    c->image_scale = 1.0f;
}

int shot_submit_rtm(shot_server_t h, const stencil_desc *d, int32_t nsteps, const shot_rtm_cfg *cfg,
                    float *image_host, float *traces_host, uint64_t *ticket)
{
    if (!h || !d || !cfg || !image_host || !ticket) return fail(STENCIL_EINVAL, "null argument");
    Server *s = reinterpret_cast<Server *>(h);
    if (s->cfg.storage != STENCIL_FP32) return fail(STENCIL_EUNSUPPORTED, "migrations need an FP32 server");
    if (nsteps < 1 || cfg->snap_every < 1 || nsteps % cfg->snap_every)
        return fail(STENCIL_EINVAL, "nsteps must be a positive multiple of snap_every");
    if (cfg->receiver_z < 0 || cfg->receiver_z >= d->nz || cfg->receiver_y < -1 || cfg->receiver_y >= d->ny)
        return fail(STENCIL_EINVAL, "receiver outside the grid");
    if (!std::isfinite(cfg->image_scale)) return fail(STENCIL_EINVAL, "image_scale must be finite");
    return submit(h, d, nsteps, nullptr, cfg, image_host, traces_host, ticket);
}

static int submit(shot_server_t h, const stencil_desc *d, int32_t nsteps, float *out_host, const shot_rtm_cfg *rtm,
                  float *image_host, float *traces_host, uint64_t *ticket)
{
    if (!h || !d || !ticket) return fail(STENCIL_EINVAL, "null argument");
    if (nsteps < 0) return fail(STENCIL_EINVAL, "nsteps < 0");
    Server *s = reinterpret_cast<Server *>(h);
    if (d->radius != s->cfg.radius) return fail(STENCIL_EINVAL, "radius differs from the server's");
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || !d->velocity) return fail(STENCIL_EINVAL, "bad descriptor");
    if (d->absorb_width > 0 && d->absorb_eta > 0.0 && s->cfg.storage != STENCIL_FP32)
        return fail(STENCIL_EUNSUPPORTED, "an absorbing layer needs FP32 storage");
    if (d->user_buffers[0] || d->user_buffers[1] || d->user_buffers[2])
        return fail(STENCIL_EINVAL, "the shot server allocates its own buffers (user_buffers must be NULL)");
    auto r = std::make_unique<Request>();
    r->desc = *d;
    r->desc.storage = s->cfg.storage;
    r->nsteps = nsteps;
    r->out_host = out_host;
    r->bytes = projected_bytes(r->desc);
    if (rtm) {
        r->rtm = true;
        r->rtm_cfg = *rtm;
        r->image_host = image_host;
        r->traces_host = traces_host;
        r->bytes += rtm_bytes(r->desc, nsteps, *rtm);
    }
    if (!d->velocity_on_device) {
        // a page-locked model is read in place at admission (one direct
        // copy); any other is copied now, so the caller may free it at once
        cudaPointerAttributes attr{};
        const bool pinned = cudaPointerGetAttributes(&attr, d->velocity) == cudaSuccess &&
                            attr.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (!pinned) {
            const size_t n = (size_t)d->nx * d->ny * d->nz;
            r->velocity.assign(d->velocity, d->velocity + n);
            r->desc.velocity = r->velocity.data();
        }
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stopping) return fail(STENCIL_ECANCELLED, "the server is shutting down");
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    *ticket = r->ticket;
    s->stats.submitted += 1;
    if (r->bytes > s->budget) {
        r->state = SHOT_FAILED;
        r->status = STENCIL_EBUDGET;
        r->t_done = r->t_submit;
        s->stats.failed += 1;
        s->all[r->ticket] = std::move(r);
        return fail(STENCIL_EBUDGET, "shot needs more device memory than the whole budget");
    }
    s->stats.queued += 1;
    s->queue.push_back(r.get());
    s->all[r->ticket] = std::move(r);
    s->cv.notify_all();
    return STENCIL_OK;
}

int shot_poll(shot_server_t h, uint64_t ticket, int32_t *state, shot_timing *t)
{
    if (!h) return fail(STENCIL_EINVAL, "null server");
    Server *s = reinterpret_cast<Server *>(h);
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(STENCIL_EUNKNOWN_TICKET, "no shot with ticket %llu", (unsigned long long)ticket);
    const Request *r = it->second.get();
    if (state) *state = r->state;
    if (t) {
        t->t_submit = r->t_submit;
        t->t_admit = r->t_admit;
        t->t_done = r->t_done;
        t->steps_done = r->steps_done;
        t->status = r->status;
        t->pad = 0;
    }
    return STENCIL_OK;
}

int shot_wait(shot_server_t h, uint64_t ticket, double timeout_s, int32_t *state)
{
    if (!h) return fail(STENCIL_EINVAL, "null server");
    Server *s = reinterpret_cast<Server *>(h);
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(STENCIL_EUNKNOWN_TICKET, "no shot with ticket %llu", (unsigned long long)ticket);
    Request *r = it->second.get();
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    const bool finished = s->cv.wait_until(lock, until, [&] { return r->state == SHOT_DONE || r->state == SHOT_FAILED; });
    if (state) *state = r->state;
    if (!finished) return fail(STENCIL_ENOTREADY, "shot %llu not finished", (unsigned long long)ticket);
    return STENCIL_OK;
}

int shot_server_get_stats(shot_server_t h, shot_server_stats *out)
{
    if (!h || !out) return fail(STENCIL_EINVAL, "null argument");
    Server *s = reinterpret_cast<Server *>(h);
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    return STENCIL_OK;
}

int shot_server_destroy(shot_server_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null server");
    Server *s = reinterpret_cast<Server *>(h);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    if (s->engine.joinable()) s->engine.join();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->retire_stop = true;
    }
    s->cv.notify_all();
    if (s->retirer.joinable()) s->retirer.join();
    const int err = s->engine_error;
    delete s;                               // releases the streams, buffers and pool
    return err;
}

}  // extern "C"
