// Host runtime behind the C-ABI of include/stencil.h: plan lifecycle, step
// enqueueing (eager or through captured CUDA graphs), state transfer, FP64
// validation reductions.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <functional>

#include "internal.h"
#include "plan_impl.h"
#include "stencil.h"

namespace stencil {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int fail_cuda(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(STENCIL_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(STENCIL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

double cfl_limit(int R)
{
    double W;
    if (R == 4) {
        W = std::fabs(wd<4>(0));
        for (int r = 1; r <= 4; ++r) W += 2.0 * std::fabs(wd<4>(r));
    } else if (R == 5) {
        W = std::fabs(wd<5>(0));
        for (int r = 1; r <= 5; ++r) W += 2.0 * std::fabs(wd<5>(r));
    } else {
        return -1.0;
    }
    return 2.0 / std::sqrt(3.0 * W);
}

int64_t row_pitch(int nx, int esize)
{
    const int64_t per = 128 / esize;       // 128-byte rows for the wavefields
    return ((int64_t)nx + per - 1) / per * per;
}

// ---- storage dispatch of the tiled kernel --------------------------------------
bool tiled_config(int R, int storage, int tx, int ty, TiledInfo *info)
{
    TiledInfo tmp;
    if (!info) info = &tmp;
    if (storage == STENCIL_FP32) return tiled_config_f32(R, tx, ty, info);
    if (storage == STENCIL_FP16) return tiled_config_f16(R, tx, ty, info);
    if (storage == STENCIL_BF16) return tiled_config_bf16(R, tx, ty, info);
    return false;
}

int tiled_blocks_per_sm(int R, int storage, int tx, int ty)
{
    if (storage == STENCIL_FP32) return tiled_blocks_per_sm_f32(R, tx, ty);
    if (storage == STENCIL_FP16) return tiled_blocks_per_sm_f16(R, tx, ty);
    if (storage == STENCIL_BF16) return tiled_blocks_per_sm_bf16(R, tx, ty);
    return 0;
}

cudaError_t launch_grouped(int R, int storage, int tx, int ty, const GroupShot *shots, const GroupItem *items,
                           int n_items, int step_off, bool absorb, cudaStream_t s)
{
    if (storage == STENCIL_FP32) return launch_grouped_f32(R, tx, ty, shots, items, n_items, step_off, absorb, s);
    if (storage == STENCIL_FP16) return launch_grouped_f16(R, tx, ty, shots, items, n_items, step_off, absorb, s);
    if (storage == STENCIL_BF16) return launch_grouped_bf16(R, tx, ty, shots, items, n_items, step_off, absorb, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tiled(int R, int storage, int tx, int ty, const TiledMaps &m, const SweepParams &p,
                         cudaStream_t s)
{
    if (storage == STENCIL_FP32) return launch_tiled_f32(R, tx, ty, m, p, s);
    if (storage == STENCIL_FP16) return launch_tiled_f16(R, tx, ty, m, p, s);
    if (storage == STENCIL_BF16) return launch_tiled_bf16(R, tx, ty, m, p, s);
    return cudaErrorInvalidValue;
}

// ---- TMA descriptors --------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int encode_map(CUtensorMap *m, const void *base, int nx, int ny, int nz, int64_t pitch, int esize, int bw,
               int bh)
{
    return encode_map_strided(m, base, nx, ny, nz, pitch, pitch * ny, esize, bw, bh);
}

int encode_map_strided(CUtensorMap *m, const void *base, int nx, int ny, int nz, int64_t pitch, int64_t plane,
                       int esize, int bw, int bh)
{
    auto fn = encode_fn();
    if (!fn) return fail(STENCIL_ECUDA, "cuTensorMapEncodeTiled not available from the driver");
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * esize), (cuuint64_t)(plane * esize)};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(STENCIL_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return STENCIL_OK;
}

// Small device-to-host reads go through a pinned per-thread buffer: a copy
// into pageable memory waits for any other thread's pageable copy in
// flight (the driver stages them), which would stall e.g. plan set-up
// behind a large read-back on another thread.
static void *pinned_scratch()
{
    thread_local void *buf = nullptr;
    if (!buf && cudaMallocHost(&buf, 256) != cudaSuccess) buf = nullptr;
    return buf;
}

// Read `bytes` (<= 256) of device memory into host `dst` through the pinned
// scratch; synchronises `s`.
static cudaError_t read_small(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    void *pin = pinned_scratch();
    if (!pin) {
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
        return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    cudaError_t e = cudaMemcpyAsync(pin, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) std::memcpy(dst, pin, bytes);
    return e;
}

// ---- plan internals -----------------------------------------------------------
int Plan::build_maps()
{
    if (tile.kernel == STENCIL_KERNEL_TWO_STEP) return build_maps_two_step();
    if (tile.kernel != STENCIL_KERNEL_TILED) return STENCIL_OK;
    TiledInfo info;
    if (!tiled_config(R, storage, tile.tx, tile.ty, &info))
        return fail(STENCIL_EUNSUPPORTED, "tile %dx%d not built for radius %d", tile.tx, tile.ty, R);
    // maps_core[b] is the point-wise operand read when u^n is in buf[b ^ 1]:
    // u^{n-1} = buf[b] (FP32), or the one d buffer (16-bit)
    for (int b = 0; b < 2; ++b) {
        int rc = encode_map(&maps_halo[b], buf[b], nx, ny, nz, pitch, esize, tile.tx + 2 * info.hx,
                            tile.ty + 2 * R);
        if (rc) return rc;
        rc = encode_map(&maps_core[b], aux_ptr(b ^ 1, 0), nx, ny, nz, pitch, esize, tile.tx, tile.ty);
        if (rc) return rc;
    }
    return encode_map(&map_kcore, kappa, nx, ny, nz, pitch, 4, tile.tx, tile.ty);
}

SweepParams Plan::params(int parity, int step_off) const
{
    SweepParams s{};
    s.nx = nx;
    s.ny = ny;
    s.nz = nz;
    s.pitch = pitch;
    s.plane = pitch * ny;
    s.u = buf[parity];
    s.up = buf[parity ^ 1];
    s.dv = dbuf;
    s.kappa = kappa;
    s.zchunk = tile.zchunk > 0 ? tile.zchunk : nz;
    s.tiles_x = 0;
    s.src = src;
    s.step_base = d_step;
    s.step_off = step_off;
    s.err = d_err;
    s.scale = d_scale;
    s.amax = d_amax;
    s.scale_d = d_scale_d;
    s.amax_d = d_amax_d;
    s.growth = growth;
    s.src_bound = src_bound;
    s.energy = rec_energy;
    s.energy_part = rec_part;
    s.energy_count = rec_count;
    s.rec_n0 = rec_n0;
    s.rec_cap = rec_cap;
    s.energy_on = rec_mem ? rec_energy_on : 0;
    if (absorb_folded()) {
        // the tiled FP32 sweep applies the layer itself, then the source
        s.absorb_w = absorb_w;
        s.absorb_tab = absorb_tab;
    } else if (absorb_w > 0) {
        s.src.on = 0;                       // added after the layer's own pass
    }
    s.wait_ns = wait_ns;
    s.fault_tx = fault_tx;
    return s;
}

StepOps Plan::step_ops(int step_off) const
{
    StepOps o{};
    o.nx = nx;
    o.ny = ny;
    o.nz = nz;
    o.pitch = pitch;
    o.plane = pitch * ny;
    o.step_base = d_step;
    o.step_off = step_off;
    o.absorb_w = absorb_folded() ? 0 : absorb_w;
    o.absorb_tab = absorb_tab;
    o.shell_points = absorb_shell;
    o.save = absorb_save;
    o.src = src;
    o.inj = inj;
    o.inj_n0 = inj_n0;
    o.inj_steps = inj_steps;
    o.inj_reverse = inj_reverse;
    o.inj_z = inj ? inj_z : -1;
    o.inj_y = inj_y;
    o.inj_scale = inj_scale;
    o.rec = rec;
    o.scale = storage == STENCIL_FP32 ? nullptr : d_scale;
    o.rec_n0 = rec_n0;
    o.rec_cap = rec_cap;
    o.rec_z = rec ? rec_z : -1;
    o.rec_y = rec_y;
    return o;
}

bool Plan::absorb_folded() const
{
    return absorb_w > 0 && tile.kernel == STENCIL_KERNEL_TILED && storage == STENCIL_FP32;
}

bool Plan::has_step_ops() const
{
    return (absorb_w > 0 && !absorb_folded()) || inj != nullptr || rec != nullptr;
}

// One time step: [layer save] sweep [layer apply, source, injection, record]
cudaError_t Plan::launch_one(int parity, int step_off, cudaStream_t s) const
{
    const SweepParams prm = params(parity, step_off);
    const bool ops = has_step_ops();
    StepOps o{};
    cudaError_t e = cudaSuccess;
    if (ops) {
        o = step_ops(step_off);
        e = launch_step_pre(o, buf[parity ^ 1], s);
        if (e != cudaSuccess) return e;
    }
    if (tile.kernel == STENCIL_KERNEL_NAIVE) {
        e = launch_naive(R, prm, s);
    } else {
        TiledMaps m;
        m.u_halo = maps_halo[parity];
        m.up_core = maps_core[parity ^ 1];
        m.k_core = map_kcore;
        e = launch_tiled(R, storage, tile.tx, tile.ty, m, prm, s);
    }
    if (e == cudaSuccess && ops) e = launch_step_post(o, buf[parity ^ 1], storage, s);
    return e;
}

int Plan::enqueue_eager(int nsteps)
{
    int done = 0;
    while (done < nsteps) {
        const int k = std::min(nsteps - done, 64);
        for (int i = 0; i < k; ++i) {
            cudaError_t e = launch_one(cur, i, stream);
            if (e != cudaSuccess) return fail_cuda(e, "sweep launch");
            cur ^= 1;
        }
        cudaError_t e = launch_advance(d_step, k, stream);
        if (e != cudaSuccess) return fail_cuda(e, "step counter");
        done += k;
    }
    return STENCIL_OK;
}

int Plan::capture_graphs()
{
    drop_graphs();
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamBeginCapture");
        int c = par;
        cudaError_t le = cudaSuccess;
        for (int i = 0; i < graph_len && le == cudaSuccess; ++i) {
            le = launch_one(c, i, stream);
            c ^= 1;
        }
        if (le == cudaSuccess) le = launch_advance(d_step, graph_len, stream);
        e = cudaStreamEndCapture(stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail_cuda(le, "launch during graph capture");
        }
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&graph_exec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
    }
    return STENCIL_OK;
}

void Plan::drop_graphs()
{
    for (auto &g : graph_exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

int Plan::enqueue(int nsteps)
{
    if (nsteps < 0) return fail(STENCIL_EINVAL, "nsteps < 0");
    if (!velocity_ok) return fail(STENCIL_EINVAL, "the plan has no valid velocity model");
    if (tile.kernel == STENCIL_KERNEL_TWO_STEP) return enqueue_two_step(nsteps);
    int left = nsteps;
    if (graph_len > 0 && left >= graph_len) {
        if (!graph_exec[0]) {
            int rc = capture_graphs();
            if (rc) return rc;
        }
        while (left >= graph_len) {
            cudaError_t e = cudaGraphLaunch(graph_exec[cur], stream);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGraphLaunch");
            left -= graph_len;   // graph_len is even: parity unchanged
        }
    }
    int rc = enqueue_eager(left);
    if (rc) return rc;
    steps_done += nsteps;
    return STENCIL_OK;
}

int Plan::check_device_error()
{
    int h = 0;
    cudaError_t e = read_small(&h, d_err, sizeof(int), stream);
    if (e != cudaSuccess) return fail_cuda(e, "stream synchronize");
    if (h) {
        cudaMemsetAsync(d_err, 0, sizeof(int), stream);
        cudaStreamSynchronize(stream);
        if (h & ERR_TIMEOUT) return fail(STENCIL_ETIMEOUT, "a device-side wait timed out");
        return fail(STENCIL_ECUDA, "device error word 0x%x", h);
    }
    return STENCIL_OK;
}

void Plan::release()
{
    if (stream) cudaStreamSynchronize(stream);
    drop_graphs();
    if (rec_mem) dev_free(rec_mem);
    rec_mem = nullptr;
    if (absorb_save) dev_free(absorb_save);
    absorb_save = nullptr;
    if (!user_owned) {
        for (auto &b : buf)
            if (b) dev_free(b);
        if (kappa) dev_free(kappa);
    }
    if (dbuf) dev_free(dbuf);
    dbuf = nullptr;
    for (auto &b : tbuf)
        if (b) dev_free(b);
    tbuf[0] = tbuf[1] = nullptr;
    for (auto &b : staging)
        if (b) dev_free(b);
    staging[0] = staging[1] = nullptr;
    if (d_scratch) dev_free(d_scratch);
    if (pool && stream) cudaStreamSynchronize(stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
    buf[0] = buf[1] = nullptr;
    kappa = nullptr;
    d_scratch = nullptr;
    stream = nullptr;
}

// v (dense, host or device) -> pitched kappa buffer, then kappa = v^2 dt^2 /
// dx^2 in place (K4), vmax and the count of invalid values read back; checks
// the CFL bound.  Synchronous on the plan's stream.
int Plan::load_velocity(const float *v, int on_device)
{
    cudaStream_t s = stream;
    cudaError_t e = memcpy_rows(kappa, pitch * sizeof(float), v, (size_t)nx * sizeof(float),
                                      (size_t)nx * sizeof(float), (size_t)ny * nz,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "velocity copy");
    if ((e = cudaMemsetAsync(d_vmax, 0, sizeof(unsigned), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return fail_cuda(e, "cudaMemsetAsync");
    e = launch_coef_init(kappa, nx, ny, nz, pitch, (dt * dt) / (dx * dx), d_vmax, d_bad, s);
    if (e != cudaSuccess) return fail_cuda(e, "coef_init");
    unsigned vmax_bits = 0;
    unsigned long long nbad = 0;
    // d_vmax and d_bad are adjacent in the scratch block (offsets 16 and 24)
    unsigned char both[16];
    e = read_small(both, d_vmax, sizeof both, s);
    if (e != cudaSuccess) return fail_cuda(e, "velocity setup");
    std::memcpy(&vmax_bits, both, sizeof vmax_bits);
    std::memcpy(&nbad, both + 8, sizeof nbad);
    velocity_ok = false;
    if (nbad) return fail(STENCIL_EINVAL, "%llu velocities are not finite and > 0", nbad);
    float vm;
    std::memcpy(&vm, &vmax_bits, sizeof vm);
    vmax = vm;
    cfl_lim = cfl_limit(R);
    cfl = (double)vm * dt / dx;
    if (cfl > cfl_lim * (1.0 + 1e-12))
        return fail(STENCIL_ECFL, "vmax*dt/dx = %.6g exceeds the stability bound %.6g", cfl, cfl_lim);
    // |kappa Lambda(u)| <= kappa_max * sum |weights| * max |u| over the star;
    // sum |weights| over the 3D star = 3W with 3W = 4 / cfl_limit^2 (the
    // 16-bit storage's scale bound on the step's change of d)
    const double kmax = cfl * cfl;
    growth = (float)(kmax * 4.0 / (cfl_lim * cfl_lim) * (1.0 + 1e-6));
    velocity_ok = true;
    return STENCIL_OK;
}

cudaError_t Plan::dev_alloc(void **ptr, size_t bytes)
{
    if (pool) return cudaMallocFromPoolAsync(ptr, bytes, pool, stream);
    return cudaMalloc(ptr, bytes);
}

void Plan::dev_free(void *ptr)
{
    if (pool) cudaFreeAsync(ptr, stream);
    else cudaFree(ptr);
}

int Plan::ensure_staging()
{
    for (auto &b : staging)
        if (!b) {
            cudaError_t e = dev_alloc(reinterpret_cast<void **>(&b), (size_t)field_elems * sizeof(float));
            if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc(staging)");
            e = cudaMemsetAsync(b, 0, (size_t)field_elems * sizeof(float), stream);
            if (e != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync(staging)");
            device_bytes += field_elems * (int64_t)sizeof(float);
        }
    return STENCIL_OK;
}

int Plan::fp32_level(int which, const float **out)
{
    if (storage == STENCIL_FP32) {
        *out = static_cast<const float *>(level_buf(which));
        return STENCIL_OK;
    }
    int rc = ensure_staging();
    if (rc) return rc;
    // u^n from buf[cur]; u^{n-1} = u^n - d^n
    const int slot = (int)(((steps_done % 4) + 4) % 4);
    cudaError_t e =
        which == 0
            ? launch_unpack16(storage, buf[cur], staging[0], nx, ny, nz, pitch, d_scale + (int64_t)slot * nz, stream)
            : launch_unpack16_prev(storage, buf[cur], dbuf, staging[1], nx, ny, nz, pitch,
                                   d_scale + (int64_t)slot * nz, d_scale_d + (int64_t)slot * nz, stream);
    if (e != cudaSuccess) return fail_cuda(e, "unpack");
    *out = staging[which];
    return STENCIL_OK;
}

// Predicted makespan of one sweep with z-chunk zc: blocks (chunk-major,
// as the hardware hands them out) go to the earliest-free of `slots`
// resident block slots; a block costs its output planes plus a weight for
// the 2R warm-up planes, which only stream u.
static double predicted_makespan(int R, int tiles, int nz, int zc, int slots)
{
    const double warm = 0.5 * 2 * R;
    std::vector<double> slot(std::max(1, slots), 0.0);
    std::make_heap(slot.begin(), slot.end(), std::greater<double>());
    double makespan = 0;
    for (int z0 = 0; z0 < nz; z0 += zc) {
        const double cost = std::min(zc, nz - z0) + warm;
        for (int t = 0; t < tiles; ++t) {
            std::pop_heap(slot.begin(), slot.end(), std::greater<double>());
            slot.back() += cost;
            makespan = std::max(makespan, slot.back());
            std::push_heap(slot.begin(), slot.end(), std::greater<double>());
        }
    }
    return makespan;
}

int choose_zchunk(int R, int storage, int tx, int ty, int nx, int ny, int nz)
{
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int bps = std::max(1, tiled_blocks_per_sm(R, storage, tx, ty));
    TiledInfo info{};
    tiled_config(R, storage, tx, ty, &info);
    const int zmax = info.zmax > 0 ? info.zmax : nz;        // 16-bit kernels bound the chunk
    const int tiles = ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
    static const int cand[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
    int best = 0;
    double best_t = 0;
    if (nz <= zmax) {
        best = nz;
        best_t = predicted_makespan(R, tiles, nz, nz, sms * bps);
    }
    for (int zc : cand) {
        if (zc >= nz || zc > zmax) break;
        const double t = predicted_makespan(R, tiles, nz, zc, sms * bps);
        if (best == 0 || t < best_t * (1.0 - 1e-9)) {
            best_t = t;
            best = zc;
        }
    }
    return best > 0 ? best : std::min(nz, zmax);
}

// The two-step kernel's z-chunk: the same block-scheduler model over its
// one block per SM, each block also streaming the 4R extra planes of its two
// stages (their stage A work weighs about as much as an output plane's).
int choose_zchunk_two_step(int R, int nx, int ny, int nz)
{
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int bps = std::max(1, two_step_blocks_per_sm(R));
    const int ty = two_step_tile_y(R);
    const int tiles = ((nx + 63) / 64) * ((ny + ty - 1) / ty);
    static const int cand[] = {16, 24, 32, 48, 64, 96, 128, 192, 256};
    int best = nz;
    double best_t = predicted_makespan(2 * R, tiles, nz, nz, sms * bps);
    for (int zc : cand) {
        if (zc >= nz) break;
        const double t = predicted_makespan(2 * R, tiles, nz, zc, sms * bps);
        if (t < best_t) {
            best_t = t;
            best = zc;
        }
    }
    return best;
}

stencil_tile default_tile(int R, int storage, int nx, int ny, int nz)
{
    stencil_tile t;
    if (storage == STENCIL_FP32 && (int64_t)nx * ny * nz <= NAIVE_MAX_POINTS) {
        // small grids are latency-bound: one pass of one thread per point
        // beats a z-march whose blocks cannot fill the GPU
        t.kernel = STENCIL_KERNEL_NAIVE;
        t.tx = t.ty = 0;
        t.zchunk = 0;
        return t;
    }
    t.kernel = STENCIL_KERNEL_TILED;
    t.tx = 64;
    t.ty = 16;
    t.zchunk = choose_zchunk(R, storage, t.tx, t.ty, nx, ny, nz);
    return t;
}

int validate_desc(const stencil_desc *d)
{
    if (!d) return fail(STENCIL_EINVAL, "null descriptor");
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return fail(STENCIL_EINVAL, "grid dims must be >= 1");
    if (d->ny > 65535 || d->nz > 65535 || d->nx > (1 << 24))
        return fail(STENCIL_EINVAL, "grid dims too large");
    if (d->radius != 4 && d->radius != 5) return fail(STENCIL_EINVAL, "radius must be 4 or 5");
    if (!(d->dx > 0) || !std::isfinite(d->dx)) return fail(STENCIL_EINVAL, "dx must be > 0");
    if (!(d->dt > 0) || !std::isfinite(d->dt)) return fail(STENCIL_EINVAL, "dt must be > 0");
    if (!d->velocity) return fail(STENCIL_EINVAL, "null velocity");
    if (d->src_amp != 0.0) {
        if (d->src_x < 0 || d->src_x >= d->nx || d->src_y < 0 || d->src_y >= d->ny || d->src_z < 0 ||
            d->src_z >= d->nz)
            return fail(STENCIL_EINVAL, "source outside the grid");
        if (!(d->src_freq_hz > 0)) return fail(STENCIL_EINVAL, "source frequency must be > 0");
    }
    if (d->storage != STENCIL_FP32 && d->storage != STENCIL_FP16 && d->storage != STENCIL_BF16)
        return fail(STENCIL_EINVAL, "storage must be FP32, FP16 or BF16");
    if (d->graph_steps < 0 || (d->graph_steps & 1))
        return fail(STENCIL_EINVAL, "graph_steps must be 0 or a positive even number");
    if (d->tune_mode < STENCIL_TUNE_NONE || d->tune_mode > STENCIL_TUNE_EXHAUSTIVE)
        return fail(STENCIL_EINVAL, "bad tune_mode");
    if (d->absorb_width < 0 || d->absorb_width > ABSORB_MAX_W || !(d->absorb_eta >= 0.0) ||
        !std::isfinite(d->absorb_eta))
        return fail(STENCIL_EINVAL, "absorb_width must be in [0, %d] and absorb_eta finite and >= 0", ABSORB_MAX_W);
    const int n_user = (d->user_buffers[0] != nullptr) + (d->user_buffers[1] != nullptr) +
                       (d->user_buffers[2] != nullptr);
    if (n_user) {
        if (n_user != 3) return fail(STENCIL_EINVAL, "user_buffers: give all three or none");
        if (d->storage != STENCIL_FP32)
            return fail(STENCIL_EUNSUPPORTED, "user_buffers need FP32 storage");
        if (d->nx % 4) return fail(STENCIL_EINVAL, "user_buffers need nx a multiple of 4 (16-byte rows)");
        for (void *b : d->user_buffers)
            if (reinterpret_cast<uintptr_t>(b) % 16) return fail(STENCIL_EINVAL, "user_buffers must be 16-byte aligned");
        if (d->user_buffers[0] == d->user_buffers[1] || d->user_buffers[0] == d->user_buffers[2] ||
            d->user_buffers[1] == d->user_buffers[2])
            return fail(STENCIL_EINVAL, "user_buffers must be three different buffers");
    }
    return STENCIL_OK;
}

int check_tile(int R, int storage, const stencil_tile &t)
{
    if (t.kernel == STENCIL_KERNEL_NAIVE) {
        if (storage != STENCIL_FP32) return fail(STENCIL_EUNSUPPORTED, "the naive kernel stores FP32 only");
        return STENCIL_OK;
    }
    if (t.kernel == STENCIL_KERNEL_TWO_STEP) {
        if (storage != STENCIL_FP32) return fail(STENCIL_EUNSUPPORTED, "the two-step kernel stores FP32 only");
        if (t.zchunk < 0) return fail(STENCIL_EINVAL, "zchunk must be >= 0");
        TwoStepInfo info;
        if (!two_step_config(R, t.tx, t.ty, &info))
            return fail(STENCIL_EUNSUPPORTED, "two-step tile %dx%d not built for radius %d", t.tx, t.ty, R);
        return STENCIL_OK;
    }
    if (t.kernel != STENCIL_KERNEL_TILED) return fail(STENCIL_EINVAL, "bad kernel id %d", t.kernel);
    if (t.zchunk < 0) return fail(STENCIL_EINVAL, "zchunk must be >= 0");
    TiledInfo info;
    if (!tiled_config(R, storage, t.tx, t.ty, &info))
        return fail(STENCIL_EUNSUPPORTED, "tile %dx%d not available for radius %d and storage %d", t.tx, t.ty, R,
                    storage);
    if (info.zmax && t.zchunk > info.zmax)
        return fail(STENCIL_EINVAL, "zchunk %d above %d for 16-bit storage", t.zchunk, info.zmax);
    return STENCIL_OK;
}

int plan_create(const stencil_desc *d, Plan **out, cudaMemPool_t pool)
{
    TraceRange tr("plan_create");
    int rc = validate_desc(d);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STENCIL_ENODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    Plan *p = new Plan();
    p->dev = dev;
    p->pool = pool;
    p->R = d->radius;
    p->nx = d->nx;
    p->ny = d->ny;
    p->nz = d->nz;
    p->dx = d->dx;
    p->dt = d->dt;
    p->storage = d->storage;
    p->esize = d->storage == STENCIL_FP32 ? 4 : 2;
    p->user_owned = d->user_buffers[0] != nullptr;
    // caller-owned buffers are dense; the plan's own rows are padded to 128 B
    p->pitch = p->user_owned ? d->nx : row_pitch(d->nx, p->esize);
    p->field_elems = p->pitch * d->ny * d->nz;
    p->graph_len = d->graph_steps;
    p->tune_mode = d->tune_mode;
    p->absorb_w = d->absorb_eta > 0.0 ? d->absorb_width : 0;
    p->absorb_eta = (float)d->absorb_eta;
    if (p->absorb_w > 0 && d->storage != STENCIL_FP32) {
        delete p;
        return fail(STENCIL_EUNSUPPORTED, "the absorbing layer needs FP32 storage");
    }
    const bool two_step = d->tile.kernel == STENCIL_KERNEL_TWO_STEP && d->tune_mode == STENCIL_TUNE_NONE;
    if (d->tile.kernel == STENCIL_KERNEL_TWO_STEP &&
        (d->tune_mode != STENCIL_TUNE_NONE || p->absorb_w > 0 || p->user_owned || d->storage != STENCIL_FP32)) {
        delete p;
        return fail(STENCIL_EUNSUPPORTED,
                    "the two-step kernel runs FP32 plans without tuning, absorbing layer or caller-owned buffers");
    }
    auto bail = [&](int code) {
        p->release();
        delete p;
        return code;
    };
    if (d->cuda_stream) {
        p->stream = static_cast<cudaStream_t>(d->cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail_cuda(e, "cudaStreamCreate"));
        p->own_stream = true;
    }
    const size_t fbytes = (size_t)p->field_elems * p->esize;
    const size_t kbytes = (size_t)p->field_elems * sizeof(float);
    if (p->user_owned) {
        p->buf[0] = d->user_buffers[0];
        p->buf[1] = d->user_buffers[1];
        p->kappa = static_cast<float *>(d->user_buffers[2]);
    } else {
        for (auto &b : p->buf) {
            e = p->dev_alloc(&b, fbytes);
            if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(field)"));
        }
        e = p->dev_alloc(reinterpret_cast<void **>(&p->kappa), kbytes);
        if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(kappa)"));
    }
    if (p->storage != STENCIL_FP32) {
        e = p->dev_alloc(&p->dbuf, fbytes);
        if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(difference field)"));
    }
    if (two_step)
        for (auto &b : p->tbuf) {
            e = p->dev_alloc(&b, fbytes);
            if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(two-step levels)"));
            if ((e = cudaMemsetAsync(b, 0, fbytes, p->stream)) != cudaSuccess)
                return bail(fail_cuda(e, "cudaMemsetAsync"));
        }
    // scratch: step counter, error word, v range, reduction partials and
    // result, and (16-bit storage) the per-level per-plane scale and amax
    // tables of u and d, 4 x [4][nz] x 4 bytes
    const size_t red_bytes = 256 + sizeof(double) * (2 * RED_BLOCKS + 8);
    const size_t tab_bytes = p->storage == STENCIL_FP32 ? 0 : (size_t)16 * 4 * d->nz;
    const size_t scratch = red_bytes + tab_bytes;
    e = p->dev_alloc(&p->d_scratch, scratch);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(scratch)"));
    unsigned char *sc = static_cast<unsigned char *>(p->d_scratch);
    p->d_step = reinterpret_cast<int64_t *>(sc);
    p->d_err = reinterpret_cast<int *>(sc + 8);
    p->d_vmax = reinterpret_cast<unsigned *>(sc + 16);
    p->d_bad = reinterpret_cast<unsigned long long *>(sc + 24);
    p->d_result = reinterpret_cast<double *>(sc + 64);
    p->d_partials = reinterpret_cast<double *>(sc + 256);
    if (tab_bytes) {
        const size_t tab = 4 * 4 * (size_t)d->nz;
        p->d_scale = reinterpret_cast<float *>(sc + red_bytes);
        p->d_amax = reinterpret_cast<unsigned *>(sc + red_bytes + tab);
        p->d_scale_d = reinterpret_cast<float *>(sc + red_bytes + 2 * tab);
        p->d_amax_d = reinterpret_cast<unsigned *>(sc + red_bytes + 3 * tab);
    }
    p->device_bytes = (p->user_owned ? 0 : 2 * (int64_t)fbytes + (int64_t)kbytes) + (int64_t)scratch +
                      (p->dbuf ? (int64_t)fbytes : 0) + (two_step ? 2 * (int64_t)fbytes : 0);
    if (p->absorb_w > 0) {
        // u^{n-1} of the layer's points, saved before each sweep
        p->absorb_shell = shell_points(d->nx, d->ny, d->nz, p->absorb_w);
        // ... and the damping factors by distance to the nearest face:
        // g_d = 1/(1+eta_d), h_d = eta_d/(1+eta_d), eta_d = eta_max ((W-d)/W)^2
        // (FP64, rounded once), entry W = (1, 0)
        const size_t save_bytes = ((sizeof(float) * (size_t)p->absorb_shell + 15) / 16) * 16;
        const size_t tab_n = (size_t)p->absorb_w + 1;
        e = p->dev_alloc(reinterpret_cast<void **>(&p->absorb_save), save_bytes + sizeof(float2) * tab_n);
        if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(absorbing layer)"));
        p->absorb_tab = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(p->absorb_save) + save_bytes);
        p->absorb_tab_host.resize(tab_n);
        for (int dd = 0; dd <= p->absorb_w; ++dd) {
            const double a = (double)(p->absorb_w - dd) / p->absorb_w;
            const double eta = d->absorb_eta * a * a;
            p->absorb_tab_host[dd] = make_float2((float)(1.0 / (1.0 + eta)), (float)(eta / (1.0 + eta)));
        }
        e = cudaMemcpyAsync(p->absorb_tab, p->absorb_tab_host.data(), sizeof(float2) * tab_n,
                            cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) return bail(fail_cuda(e, "absorbing layer table"));
        p->device_bytes += (int64_t)(save_bytes + sizeof(float2) * tab_n);
    }

    cudaStream_t s = p->stream;
    if ((e = cudaMemsetAsync(p->d_scratch, 0, scratch, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->buf[0], 0, fbytes, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->buf[1], 0, fbytes, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->kappa, 0, kbytes, s)) != cudaSuccess ||
        (p->dbuf && (e = cudaMemsetAsync(p->dbuf, 0, fbytes, s)) != cudaSuccess))
        return bail(fail_cuda(e, "cudaMemsetAsync"));
    float v_src = 0.0f;
    if (d->src_amp != 0.0) {
        const float *vs = d->velocity + ((int64_t)d->src_z * d->ny + d->src_y) * d->nx + d->src_x;
        if (d->velocity_on_device) e = read_small(&v_src, vs, sizeof(float), s);
        else v_src = *vs;
        if (e != cudaSuccess) return bail(fail_cuda(e, "source velocity read"));
    }
    p->src_amp = d->src_amp;
    rc = p->load_velocity(d->velocity, d->velocity_on_device);
    if (rc) return bail(rc);

    p->src.on = d->src_amp != 0.0;
    p->src.x = d->src_x;
    p->src.y = d->src_y;
    p->src.z = d->src_z;
    p->src.f = d->src_freq_hz;
    p->src.t0 = d->src_t0 < 0 ? 1.0 / d->src_freq_hz : d->src_t0;
    p->src.dt = d->dt;
    p->src.scale = d->src_amp * (double)v_src * (double)v_src * d->dt * d->dt;
    p->src_bound = (float)(std::fabs(p->src.scale) * (1.0 + 1e-6));

    // tile
    stencil_tile t = d->tile;
    if (t.kernel == STENCIL_KERNEL_TWO_STEP) {
        // fixed tile; the odd last step of a run uses the tiled kernel's 64 x 16
        t.tx = 64;
        t.ty = two_step_tile_y(d->radius);
        if (t.zchunk < 0) t.zchunk = choose_zchunk_two_step(d->radius, d->nx, d->ny, d->nz);
        p->t2_plain_zchunk = choose_zchunk(d->radius, STENCIL_FP32, 64, 16, d->nx, d->ny, d->nz);
    }
    if (t.kernel == STENCIL_KERNEL_AUTO) t = default_tile(d->radius, d->storage, d->nx, d->ny, d->nz);
    else if (t.kernel == STENCIL_KERNEL_TILED && t.zchunk < 0)
        t.zchunk = choose_zchunk(d->radius, d->storage, t.tx, t.ty, d->nx, d->ny, d->nz);
    if (t.zchunk == 0) t.zchunk = d->nz;
    rc = check_tile(p->R, p->storage, t);
    if (rc) return bail(rc);
    p->tile = t;
    rc = p->build_maps();
    if (rc) return bail(rc);
    if (d->tune_mode != STENCIL_TUNE_NONE) {
        rc = tune_plan(p, d);
        if (rc) return bail(rc);
    }
    *out = p;
    return STENCIL_OK;
}

}  // namespace stencil

using namespace stencil;

extern "C" {

void stencil_desc_init(stencil_desc *d)
{
    if (!d) return;
    std::memset(d, 0, sizeof *d);
    d->radius = 5;
    d->dx = 10.0;
    d->src_freq_hz = 15.0;
    d->src_t0 = -1.0;
    d->src_amp = 1.0;
    d->storage = STENCIL_FP32;
    d->tune_mode = STENCIL_TUNE_NONE;
    d->tile.kernel = STENCIL_KERNEL_AUTO;
    d->tune.parts = 5;
    d->tune.iterations = 8;
    d->tune.streams = 4;
    d->tune.groups = 2;
}

int stencil_plan(const stencil_desc *d, stencil_plan_t *out)
{
    if (!out) return fail(STENCIL_EINVAL, "null output handle");
    *out = nullptr;
    Plan *p = nullptr;
    int rc = plan_create(d, &p);
    if (rc) return rc;
    *out = reinterpret_cast<stencil_plan_t>(p);
    return STENCIL_OK;
}

int stencil_destroy(stencil_plan_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    p->release();
    delete p;
    return STENCIL_OK;
}

int stencil_step(stencil_plan_t h, int32_t nsteps)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    TraceRange tr("stencil_step");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    return p->enqueue(nsteps);
}

static int copy_out(Plan *p, int which, float *out, int on_device)
{
    const float *src = nullptr;
    int rc = p->fp32_level(which, &src);
    if (rc) return rc;
    cudaError_t e = memcpy_rows(out, (size_t)p->nx * sizeof(float), src, p->pitch * sizeof(float),
                                      (size_t)p->nx * sizeof(float), (size_t)p->ny * p->nz,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "field copy out");
    return STENCIL_OK;
}

int stencil_run(stencil_plan_t h, int32_t nsteps, float *out_u, int32_t out_on_device)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    TraceRange tr("stencil_run");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    int rc = p->enqueue(nsteps);
    if (rc) return rc;
    if (out_u) {
        rc = copy_out(p, 0, out_u, out_on_device);
        if (rc) return rc;
    }
    return p->check_device_error();
}

int stencil_sync(stencil_plan_t h)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    return p->check_device_error();
}

int stencil_get_field(stencil_plan_t h, int32_t which, float *out, int32_t out_on_device)
{
    if (!h || !out) return fail(STENCIL_EINVAL, "null argument");
    if (which != 0 && which != 1) return fail(STENCIL_EINVAL, "which must be 0 or 1");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    int rc = copy_out(p, which, out, out_on_device);
    if (rc) return rc;
    return p->check_device_error();
}

int stencil_set_fields(stencil_plan_t h, const float *u, const float *u_prev, int32_t on_device, int64_t step)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    if (step < 0) return fail(STENCIL_EINVAL, "step must be >= 0");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    const float *src[2] = {u, u_prev};
    if (p->storage == STENCIL_FP32 && !u && !u_prev) {
        // both levels zero: one launch clears them and sets the counter
        cudaError_t e = launch_clear_levels(static_cast<float *>(p->level_buf(0)), static_cast<float *>(p->level_buf(1)),
                                            p->field_elems, p->d_step, step, p->stream);
        if (e != cudaSuccess) return fail_cuda(e, "field reset");
        p->steps_done = step;
        return STENCIL_OK;
    }
    if (p->storage != STENCIL_FP32) {
        int rc = p->ensure_staging();
        if (rc) return rc;
    }
    // FP32: straight into the two level buffers.  16-bit: both levels staged
    // in FP32 (zeros where not given), then u^n and d^n = u^n - u^{n-1}
    // packed with the scales of level `step`.
    for (int k = 0; k < 2; ++k) {
        float *dst = p->storage == STENCIL_FP32 ? static_cast<float *>(p->level_buf(k)) : p->staging[k];
        cudaError_t e;
        if (!src[k])
            e = cudaMemsetAsync(dst, 0, (size_t)p->field_elems * sizeof(float), p->stream);
        else
            e = memcpy_rows(dst, p->pitch * sizeof(float), src[k], (size_t)p->nx * sizeof(float),
                            (size_t)p->nx * sizeof(float), (size_t)p->ny * p->nz,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) return fail_cuda(e, "field copy in");
    }
    if (p->storage != STENCIL_FP32) {
        const int64_t slot = step % 4;
        cudaError_t e = launch_pack16(p->storage, p->staging[0], nullptr, p->buf[p->cur], p->nx, p->ny, p->nz,
                                      p->pitch, p->d_scale + slot * p->nz, p->d_amax + slot * p->nz, p->stream);
        if (e == cudaSuccess)
            e = launch_pack16(p->storage, p->staging[0], p->staging[1], p->dbuf, p->nx, p->ny, p->nz, p->pitch,
                              p->d_scale_d + slot * p->nz, p->d_amax_d + slot * p->nz, p->stream);
        if (e != cudaSuccess) return fail_cuda(e, "field pack");
        // the maxima of the levels the next two steps write start from zero
        for (int64_t level = step + 1; level <= step + 2 && e == cudaSuccess; ++level) {
            const int64_t sl = level % 4;
            e = cudaMemsetAsync(p->d_amax + sl * p->nz, 0, sizeof(unsigned) * p->nz, p->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(p->d_amax_d + sl * p->nz, 0, sizeof(unsigned) * p->nz, p->stream);
        }
        if (e != cudaSuccess) return fail_cuda(e, "amax reset");
    }
    cudaError_t e = launch_set_step(p->d_step, step, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "step counter");
    p->steps_done = step;
    // a copy from host memory is complete before the caller gets its arrays
    // back; without one the call only enqueues (errors surface at the next
    // synchronising call)
    if (!on_device && (u || u_prev)) return p->check_device_error();
    return STENCIL_OK;
}

int stencil_set_velocity(stencil_plan_t h, const float *velocity, int32_t on_device)
{
    if (!h || !velocity) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    float v_src = 0.0f;
    if (p->src.on) {
        const float *vs = velocity + ((int64_t)p->src.z * p->ny + p->src.y) * p->nx + p->src.x;
        cudaError_t e = cudaSuccess;
        if (on_device) e = read_small(&v_src, vs, sizeof(float), p->stream);
        else v_src = *vs;
        if (e != cudaSuccess) return fail_cuda(e, "source velocity read");
    }
    const double old_scale = p->src.scale;
    const float old_bound = p->src_bound, old_growth = p->growth;
    int rc = p->load_velocity(velocity, on_device);
    if (rc) return rc;
    p->src.scale = p->src_amp * (double)v_src * (double)v_src * p->dt * p->dt;
    p->src_bound = (float)(std::fabs(p->src.scale) * (1.0 + 1e-6));
    // captured launches carry the source scale and the growth bound by value:
    // recapture only when a new model changes them (kappa is read in place)
    if (p->src.scale != old_scale || p->src_bound != old_bound || p->growth != old_growth) p->drop_graphs();
    return STENCIL_OK;
}

int stencil_get_stats(stencil_plan_t h, stencil_stats *s)
{
    if (!h || !s) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    std::memset(s, 0, sizeof *s);
    s->steps_done = p->steps_done;
    s->tile = p->tile;
    s->vmax = p->vmax;
    s->cfl = p->cfl;
    s->cfl_limit = p->cfl_lim;
    s->pitch = p->pitch;
    s->field_bytes = p->field_elems * (int64_t)p->esize;
    s->device_bytes = p->device_bytes;
    s->min_time_ms = p->min_time_ms;
    s->actual_time_ms = p->actual_time_ms;
    s->full_time_ms = p->full_time_ms;
    s->quality = p->quality;
    s->selection_ms = p->selection_ms;
    s->n_candidates = p->n_candidates;
    s->tune_mode = p->tune_mode;
    s->current_buffer = p->cur;
    s->user_buffers = p->user_owned ? 1 : 0;
    return STENCIL_OK;
}

int stencil_energy(stencil_plan_t h, double *out)
{
    if (!h || !out) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    const float *u1 = nullptr, *u0 = nullptr;
    int rc = p->fp32_level(0, &u1);
    if (!rc) rc = p->fp32_level(1, &u0);
    if (rc) return rc;
    cudaError_t e = launch_energy(p->R, u1, u0, p->kappa, p->nx, p->ny, p->nz, p->pitch, p->d_partials,
                                  p->d_result, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "energy");
    e = read_small(out, p->d_result, sizeof(double), p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "energy copy");
    return p->check_device_error();
}

int stencil_rel_l2(stencil_plan_t h, const double *ref, double *out)
{
    if (!h || !ref || !out) return fail(STENCIL_EINVAL, "null argument");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    const float *u1 = nullptr;
    int rc0 = p->fp32_level(0, &u1);
    if (rc0) return rc0;
    cudaError_t e = launch_sqdiff(u1, ref, p->nx, p->ny, p->nz, p->pitch, p->d_partials, p->d_result, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "rel_l2");
    double h2[2];
    e = read_small(h2, p->d_result, sizeof h2, p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "rel_l2 copy");
    int rc = p->check_device_error();
    if (rc) return rc;
    *out = h2[1] > 0 ? std::sqrt(h2[0] / h2[1]) : (h2[0] == 0 ? 0.0 : INFINITY);
    return STENCIL_OK;
}

double stencil_cfl_limit(int32_t radius) { return cfl_limit(radius); }

int stencil_tile_info(int32_t radius, int32_t storage, int32_t tx, int32_t ty, int32_t *smem_bytes,
                      int32_t *threads)
{
    TiledInfo info;
    if (!tiled_config(radius, storage, tx, ty, &info)) return 0;
    if (smem_bytes) *smem_bytes = info.smem;
    if (threads) *threads = info.threads;
    return 1;
}

int stencil_debug_wait_fault(stencil_plan_t h, int32_t enable, uint32_t wait_ns)
{
    if (!h) return fail(STENCIL_EINVAL, "null plan");
    Plan *p = reinterpret_cast<Plan *>(h);
    cudaSetDevice(p->dev);
    if (p->tile.kernel != STENCIL_KERNEL_TILED && p->tile.kernel != STENCIL_KERNEL_TWO_STEP)
        return fail(STENCIL_EUNSUPPORTED, "the hook needs the tiled or two-step kernel");
    int rc = p->check_device_error();
    if (rc) return rc;
    p->fault_tx = enable ? 16u : 0u;
    p->wait_ns = wait_ns;
    p->drop_graphs();               // captured launches carry the parameters by value
    return STENCIL_OK;
}

const char *stencil_last_error(void) { return g_last_error.c_str(); }

const char *stencil_version(void) { return "libstencil 0.1.0 (sm_103a)"; }

}  // extern "C"
