// Tile selection: the paper's two-phase blocksize-selection methodology
// (Sec. 3.2-3.3) re-run on the GPU tile parameters (tx, ty, zchunk), plus
// an exhaustive search and the library's own tuner.
//
// Mapping of the paper's roles onto one GPU:
//   * "process on a core"  -> a CUDA stream sweeping its own slab of rows
//     (a y-range of every plane, the grid's full depth: C streams share L2
//     and HBM the way the cores of a node share cache and memory bus, and
//     each meets the real run's z extent, so the z-chunk is judged in the
//     setting it will run in);
//   * "node"               -> a group; the nC candidates are split over N
//     groups, which run one after another;
//   * nI iterations        -> nI sweeps of the slab, timed with CUDA events
//     on the stream.
// Selection phase gives MinTime, verification phase (all streams run the
// chosen tile together) gives ActualTime; quality = (Actual - Min) / Min.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan_impl.h"

namespace stencil {

// ---- candidate generation (Sec. 3.7) --------------------------------------
// b_l = <1, S/(P-1)+1, 2S/(P-1)+1, ..., (P-1)S/(P-1)+1>, read with integer
// division and the last value clamped to S (the printed example for
// S = 200, P = 5 is <1, 51, 101, 151, 200>); duplicates dropped.
std::vector<int> candidates_1d(int S, int P)
{
    std::vector<int> out;
    if (S < 1 || P < 2) return out;
    out.push_back(1);
    for (int m = 1; m < P; ++m) {
        const int b = std::min<long long>(S, (long long)m * S / (P - 1) + 1);
        if (std::find(out.begin(), out.end(), b) == out.end()) out.push_back(b);
    }
    return out;
}

// P-part subset of an admissible value list: the 1-based positions given by
// candidates_1d(len, P).
static std::vector<int> pick_axis(const std::vector<int> &vals, int P)
{
    std::vector<int> out;
    for (int pos : candidates_1d((int)vals.size(), P)) out.push_back(vals[pos - 1]);
    return out;
}

// ---- stage reductions (Sec. 3.3, Eqs. 1-3) ------------------------------------
struct Pick {
    int group = -1, stream = -1, cand = -1;
    double t = 0;
};

// t[(g*C + c)*K + k]: time of group g's k-th candidate on stream c.
// target 0 = min (MMMB), 1 = max (MWMB), 2 = closest to the mean (MAMB).
// Ties go to the lowest index at every stage.
Pick three_stage(const double *t, int G, int C, int K, int target)
{
    Pick best;
    for (int g = 0; g < G; ++g) {
        std::vector<int> bk(C);
        std::vector<double> bt(C);
        for (int c = 0; c < C; ++c) {            // stage 1: per-stream best
            const double *row = t + ((size_t)g * C + c) * K;
            int k = 0;
            for (int j = 1; j < K; ++j)
                if (row[j] < row[k]) k = j;
            bk[c] = k;
            bt[c] = row[k];
        }
        int cs = 0;                               // stage 2: one stream of the group
        if (target == 0) {
            for (int c = 1; c < C; ++c)
                if (bt[c] < bt[cs]) cs = c;
        } else if (target == 1) {
            for (int c = 1; c < C; ++c)
                if (bt[c] > bt[cs]) cs = c;
        } else {
            double mean = 0;
            for (int c = 0; c < C; ++c) mean += bt[c];
            mean /= C;
            for (int c = 1; c < C; ++c)
                if (std::fabs(bt[c] - mean) < std::fabs(bt[cs] - mean)) cs = c;
        }
        if (best.group < 0 || bt[cs] < best.t) {  // stage 3: min over groups
            best.group = g;
            best.stream = cs;
            best.cand = bk[cs];
            best.t = bt[cs];
        }
    }
    return best;
}

// OB: t[c*K + k] = stream c's k-th own candidate; global minimum.
Pick original_block(const double *t, int C, int K)
{
    Pick best;
    for (int c = 0; c < C; ++c)
        for (int k = 0; k < K; ++k)
            if (best.stream < 0 || t[(size_t)c * K + k] < best.t) {
                best.stream = c;
                best.cand = k;
                best.t = t[(size_t)c * K + k];
            }
    best.group = 0;
    return best;
}

// ---- candidate tiles ----------------------------------------------------------
struct Cand {
    int tx, ty, zc;
};

static const int TX_VALUES[] = {32, 64, 128};
static const int TY_VALUES[] = {4, 8, 16, 32};

// z-chunks 8, 12, 16, 24, 32, 48, ... (powers of two and 1.5x them) below
// top, then top = min(nz, zmax) (zmax: the 16-bit kernels' bound)
static std::vector<int> zchunk_values(int nz, int zmax)
{
    const int top = zmax > 0 ? std::min(nz, zmax) : nz;
    std::vector<int> z;
    for (int v = 8; v < top; v *= 2) {
        z.push_back(v);
        if (v + v / 2 < top) z.push_back(v + v / 2);
    }
    z.push_back(top);
    return z;
}

static bool feasible(int R, int storage, int tx, int ty, int *zmax = nullptr)
{
    TiledInfo info;
    if (!tiled_config(R, storage, tx, ty, &info)) return false;
    if (zmax) *zmax = info.zmax;
    return true;
}

// Every tile the library can run for this grid, (tx, ty, zc) in that order.
static std::vector<Cand> admissible(int R, int storage, int nz)
{
    std::vector<Cand> out;
    int zmax = 0;
    for (int tx : TX_VALUES)
        for (int ty : TY_VALUES)
            if (feasible(R, storage, tx, ty, &zmax))
                for (int zc : zchunk_values(nz, zmax)) out.push_back({tx, ty, zc});
    return out;
}

// The P-part candidate set of Sec. 3.7, one axis list per tile parameter.
static std::vector<Cand> candidate_set(int R, int storage, int nz, int P)
{
    std::vector<int> txs(std::begin(TX_VALUES), std::end(TX_VALUES));
    std::vector<int> tys(std::begin(TY_VALUES), std::end(TY_VALUES));
    std::vector<Cand> out;
    int zmax = 0;
    for (int tx : pick_axis(txs, P))
        for (int ty : pick_axis(tys, P))
            if (feasible(R, storage, tx, ty, &zmax))
                for (int zc : pick_axis(zchunk_values(nz, zmax), P)) out.push_back({tx, ty, zc});
    return out;
}

// ---- timing engine ----------------------------------------------------------------
// A view of the plan's buffers restricted to rows [y0, y0 + nys) of every
// plane (all nz planes), with the tensor maps of one candidate tile.  Views
// of different row slabs never touch each other's memory, so several streams
// can sweep them at once; each sweeps the grid's full depth, so a candidate
// z-chunk meets the same number of planes (and warm-up planes per chunk) as
// in the real run.
struct View {
    int y0 = 0, nys = 0;
    Cand c{};
    TiledMaps maps[2];   // by parity
};

static int make_view(const Plan *p, const Cand &c, int y0, int nys, View *v)
{
    TiledInfo info;
    if (!tiled_config(p->R, p->storage, c.tx, c.ty, &info))
        return fail(STENCIL_EUNSUPPORTED, "tile %dx%d unavailable", c.tx, c.ty);
    v->y0 = y0;
    v->nys = nys;
    v->c = c;
    const int64_t off = (int64_t)y0 * p->pitch, plane = p->pitch * p->ny;
    for (int par = 0; par < 2; ++par) {
        int rc = encode_map_strided(&v->maps[par].u_halo, p->bptr(par, off), p->nx, nys, p->nz, p->pitch, plane,
                                    p->esize, c.tx + 2 * info.hx, c.ty + 2 * p->R);
        if (!rc)
            rc = encode_map_strided(&v->maps[par].up_core, p->aux_ptr(par, off), p->nx, nys, p->nz, p->pitch, plane,
                                    p->esize, c.tx, c.ty);
        if (!rc)
            rc = encode_map_strided(&v->maps[par].k_core, p->kappa + off, p->nx, nys, p->nz, p->pitch, plane, 4,
                                    c.tx, c.ty);
        if (rc) return rc;
    }
    return STENCIL_OK;
}

static cudaError_t sweep_view(const Plan *p, const View &v, int parity, cudaStream_t s)
{
    const int64_t off = (int64_t)v.y0 * p->pitch;
    SweepParams prm = p->params(parity, 0);
    prm.ny = v.nys;                 // rows of the view; plane stride stays the grid's
    prm.u = p->bptr(parity, off);
    prm.up = p->bptr(parity ^ 1, off);
    if (p->storage != STENCIL_FP32) prm.dv = p->aux_ptr(parity, off);
    prm.kappa = p->kappa + off;
    prm.zchunk = std::min(v.c.zc, p->nz);
    prm.src.on = 0;
    prm.energy_on = 0;              // selection sweeps time the plain sweep
    prm.fault_tx = 0;
    return launch_tiled(p->R, p->storage, v.c.tx, v.c.ty, v.maps[parity], prm, s);
}

struct Streams {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> e0, e1;
    ~Streams()
    {
        for (auto x : e0) cudaEventDestroy(x);
        for (auto x : e1) cudaEventDestroy(x);
        for (auto x : s) cudaStreamDestroy(x);
    }
    int init(int C)
    {
        s.resize(C);
        e0.resize(C);
        e1.resize(C);
        for (int c = 0; c < C; ++c) {
            cudaError_t e = cudaStreamCreateWithFlags(&s[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreate(&e0[c]);
            if (e == cudaSuccess) e = cudaEventCreate(&e1[c]);
            if (e != cudaSuccess) return fail_cuda(e, "tuner stream setup");
        }
        return STENCIL_OK;
    }
};

// Each stream c sweeps views[c] nI times; all streams run at once (launches
// interleaved step by step).  ms[c] = stream c's elapsed time.
static int time_together(const Plan *p, Streams &S, const std::vector<View> &views, int nI, double *ms)
{
    const int C = (int)views.size();
    auto sync_all = [&]() {
        cudaError_t r = cudaStreamSynchronize(p->stream);
        for (int c = 0; c < C && r == cudaSuccess; ++c) r = cudaStreamSynchronize(S.s[c]);
        return r;
    };
    cudaError_t e = sync_all();
    if (e != cudaSuccess) return fail_cuda(e, "tuner sync");
    for (int c = 0; c < C; ++c)    // untimed warm-up launch (module load, first-touch)
        if ((e = sweep_view(p, views[c], 0, S.s[c])) != cudaSuccess) return fail_cuda(e, "tuner warm-up");
    if ((e = sync_all()) != cudaSuccess) return fail_cuda(e, "tuner sync");
    for (int c = 0; c < C; ++c) cudaEventRecord(S.e0[c], S.s[c]);
    for (int i = 0; i < nI; ++i)
        for (int c = 0; c < C; ++c)
            if ((e = sweep_view(p, views[c], i & 1, S.s[c])) != cudaSuccess) return fail_cuda(e, "tuner sweep");
    for (int c = 0; c < C; ++c) cudaEventRecord(S.e1[c], S.s[c]);
    if ((e = sync_all()) != cudaSuccess) return fail_cuda(e, "tuner sync");
    for (int c = 0; c < C; ++c) {
        float f = 0;
        cudaEventElapsedTime(&f, S.e0[c], S.e1[c]);
        ms[c] = f;
    }
    return STENCIL_OK;
}

// Slab c of C: rows [c*ny/C, (c+1)*ny/C) of every plane.
static void slab(int ny, int C, int c, int *y0, int *n)
{
    const int a = (int)((int64_t)c * ny / C), b = (int)((int64_t)(c + 1) * ny / C);
    *y0 = a;
    *n = b - a;
}

static int time_full(const Plan *p, Streams &S, const Cand &c, int nI, double *ms)
{
    std::vector<View> v(1);
    int rc = make_view(p, c, 0, p->ny, &v[0]);
    if (rc) return rc;
    Streams one;
    if ((rc = one.init(1))) return rc;
    (void)S;
    return time_together(p, one, v, nI, ms);
}

int tune_plan(Plan *p, const stencil_desc *d)
{
    TraceRange tr("tile selection");
    const auto t_start = std::chrono::steady_clock::now();
    const int mode = d->tune_mode;
    const int P = d->tune.parts > 1 ? d->tune.parts : 5;
    const int nI = d->tune.iterations > 0 ? d->tune.iterations : 8;
    int C = d->tune.streams > 0 ? d->tune.streams : 4;
    int G = d->tune.groups > 0 ? d->tune.groups : 2;
    C = std::max(1, std::min(C, p->ny));
    Streams S;
    int rc = S.init(C);
    if (rc) return rc;

    std::vector<Cand> cands = (mode == STENCIL_TUNE_EXHAUSTIVE || mode == STENCIL_TUNE_OWN)
                                  ? admissible(p->R, p->storage, p->nz)
                                  : candidate_set(p->R, p->storage, p->nz, P);
    if (cands.empty()) return fail(STENCIL_EUNSUPPORTED, "no feasible tile");
    Cand chosen{};
    double min_ms = 0, actual_ms = 0;
    bool concurrent_verify = true;

    if (mode == STENCIL_TUNE_MWMB || mode == STENCIL_TUNE_MMMB || mode == STENCIL_TUNE_MAMB) {
        const int target = mode == STENCIL_TUNE_MMMB ? 0 : mode == STENCIL_TUNE_MWMB ? 1 : 2;
        // nC candidates split into N groups of ceil(nC/N) (the last ones
        // shorter; missing entries are +inf and never chosen)
        const int nC = (int)cands.size();
        G = std::max(1, std::min(G, nC));
        const int K = (nC + G - 1) / G;
        std::vector<double> t((size_t)G * C * K, INFINITY);
        for (int g = 0; g < G; ++g)
            for (int k = 0; k < K && (size_t)g * K + k < cands.size(); ++k) {
                const Cand &c = cands[(size_t)g * K + k];
                std::vector<View> views(C);
                for (int s = 0; s < C; ++s) {
                    int y0, n;
                    slab(p->ny, C, s, &y0, &n);
                    if ((rc = make_view(p, c, y0, n, &views[s]))) return rc;
                }
                std::vector<double> ms(C);
                if ((rc = time_together(p, S, views, nI, ms.data()))) return rc;
                for (int s = 0; s < C; ++s) t[((size_t)g * C + s) * K + k] = ms[s];
            }
        Pick pk = three_stage(t.data(), G, C, K, target);
        chosen = cands[(size_t)pk.group * K + pk.cand];
        min_ms = pk.t;
        p->n_candidates = nC;
    } else if (mode == STENCIL_TUNE_OB) {
        // nC/nP candidates per stream, distinct across streams (the last
        // stream's list shorter: it repeats its own last candidate)
        const int nC = (int)cands.size();
        const int K = (nC + C - 1) / C;
        std::vector<double> t((size_t)C * K, INFINITY);
        for (int k = 0; k < K; ++k) {
            std::vector<View> views(C);
            for (int s = 0; s < C; ++s) {
                int y0, n;
                slab(p->ny, C, s, &y0, &n);
                const Cand &c = cands[std::min<size_t>((size_t)s * K + k, cands.size() - 1)];
                if ((rc = make_view(p, c, y0, n, &views[s]))) return rc;
            }
            std::vector<double> ms(C);
            if ((rc = time_together(p, S, views, nI, ms.data()))) return rc;
            for (int s = 0; s < C; ++s)
                if ((size_t)s * K + k < cands.size()) t[(size_t)s * K + k] = ms[s];
        }
        Pick pk = original_block(t.data(), C, K);
        chosen = cands[(size_t)pk.stream * K + pk.cand];
        min_ms = pk.t;
        p->n_candidates = nC;
    } else {
        // EXHAUSTIVE: every admissible tile on the full grid.  OWN: the same
        // space, pruned: best (tx, ty) at the default zchunk, then every
        // zchunk for that (tx, ty).
        std::vector<Cand> run;
        if (mode == STENCIL_TUNE_EXHAUSTIVE) {
            run = cands;
        } else {
            for (int tx : TX_VALUES)
                for (int ty : TY_VALUES)
                    if (feasible(p->R, p->storage, tx, ty))
                        run.push_back({tx, ty, choose_zchunk(p->R, p->storage, tx, ty, p->nx, p->ny, p->nz)});
        }
        double best = 0;
        for (const Cand &c : run) {
            double ms;
            if ((rc = time_full(p, S, c, nI, &ms))) return rc;
            if (p->n_candidates++ == 0 || ms < best) {
                best = ms;
                chosen = c;
            }
        }
        if (mode == STENCIL_TUNE_OWN) {
            int zmax = 0;
            feasible(p->R, p->storage, chosen.tx, chosen.ty, &zmax);
            for (int zc : zchunk_values(p->nz, zmax)) {
                const Cand c{chosen.tx, chosen.ty, zc};
                double ms;
                if ((rc = time_full(p, S, c, nI, &ms))) return rc;
                ++p->n_candidates;
                if (ms < best) {
                    best = ms;
                    chosen = c;
                }
            }
        }
        min_ms = best;
        concurrent_verify = false;
    }

    // verification phase
    if (concurrent_verify) {
        std::vector<View> views(C);
        for (int s = 0; s < C; ++s) {
            int y0, n;
            slab(p->ny, C, s, &y0, &n);
            if ((rc = make_view(p, chosen, y0, n, &views[s]))) return rc;
        }
        std::vector<double> ms(C);
        if ((rc = time_together(p, S, views, nI, ms.data()))) return rc;
        actual_ms = *std::max_element(ms.begin(), ms.end());
    } else {
        if ((rc = time_full(p, S, chosen, nI, &actual_ms))) return rc;
    }
    double full_ms = 0;
    if ((rc = time_full(p, S, chosen, nI, &full_ms))) return rc;

    // adopt the tile; the timing runs scribbled on the fields: clear them
    p->tile.kernel = STENCIL_KERNEL_TILED;
    p->tile.tx = chosen.tx;
    p->tile.ty = chosen.ty;
    p->tile.zchunk = chosen.zc;
    p->drop_graphs();
    if ((rc = p->build_maps())) return rc;
    const size_t fbytes = (size_t)p->field_elems * p->esize;
    cudaError_t e = cudaMemsetAsync(p->buf[0], 0, fbytes, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->buf[1], 0, fbytes, p->stream);
    if (e == cudaSuccess && p->dbuf) e = cudaMemsetAsync(p->dbuf, 0, fbytes, p->stream);
    // the four [4][nz] scale and max tables of u and d are contiguous
    if (e == cudaSuccess && p->d_scale) e = cudaMemsetAsync(p->d_scale, 0, sizeof(float) * 16 * p->nz, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail_cuda(e, "clear after tuning");
    p->min_time_ms = min_ms;
    p->actual_time_ms = actual_ms;
    p->full_time_ms = full_ms;
    p->quality = (actual_ms - min_ms) / min_ms;
    p->selection_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return p->check_device_error();
}

}  // namespace stencil

using namespace stencil;

extern "C" {

int stencil_candidates_1d(int32_t S, int32_t P, int32_t *out, int32_t cap, int32_t *n)
{
    if (!out || !n || cap < 0) return fail(STENCIL_EINVAL, "null argument");
    if (S < 1 || P < 2) return fail(STENCIL_EINVAL, "need S >= 1 and P >= 2");
    std::vector<int> v = candidates_1d(S, P);
    *n = (int32_t)v.size();
    if ((int)v.size() > cap) return fail(STENCIL_EINVAL, "output too small (%d needed)", (int)v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
    return STENCIL_OK;
}

int stencil_select(const double *times, int32_t groups, int32_t streams, int32_t cands, int32_t target,
                   int32_t *group, int32_t *stream, int32_t *cand, double *time)
{
    if (!times || !group || !stream || !cand || !time) return fail(STENCIL_EINVAL, "null argument");
    if (groups < 1 || streams < 1 || cands < 1) return fail(STENCIL_EINVAL, "counts must be >= 1");
    if (target < 0 || target > 2) return fail(STENCIL_EINVAL, "target must be 0 (min), 1 (max) or 2 (avg)");
    Pick pk = three_stage(times, groups, streams, cands, target);
    *group = pk.group;
    *stream = pk.stream;
    *cand = pk.cand;
    *time = pk.t;
    return STENCIL_OK;
}

int stencil_select_ob(const double *times, int32_t streams, int32_t cands, int32_t *stream, int32_t *cand,
                      double *time)
{
    if (!times || !stream || !cand || !time) return fail(STENCIL_EINVAL, "null argument");
    if (streams < 1 || cands < 1) return fail(STENCIL_EINVAL, "counts must be >= 1");
    Pick pk = original_block(times, streams, cands);
    *stream = pk.stream;
    *cand = pk.cand;
    *time = pk.t;
    return STENCIL_OK;
}

}  // extern "C"
