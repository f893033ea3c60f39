/*
 * The paper's method on the host cores -- a CPU BASELINE, NOT A CHECKER.
 *
 * Only bench.py's host-method leg and the test suite call this file; the
 * product path never links or runs it, and it shares no code with the CUDA
 * library.  It is what the paper itself runs, transplanted to this host:
 *
 *   - the "3D model" step of Sec. 2 (order-2R star Laplacian, leapfrog in
 *     time, point source), in FP32, traversed in blocks of bi x bj x bk
 *     points (the loop tiling of Sec. 3, Fig. 1b), blocks shared out over
 *     the host's cores with OpenMP;
 *   - the blocksize picked by MWMB (Sec. 3.2-3.3): every core sweeps its own
 *     instance of a slab of the grid (nx x ny x nz/T), as the paper's
 *     processes each own a problem, with every candidate block in the same
 *     order, nI times each, all cores at once (so they contend for the
 *     shared caches and memory as in the real run); stage 1 keeps each
 *     core's fastest candidate, stage 2 the slowest of those (Eq. 2; the host
 *     is one node, so stage 3 has one entry); the verification phase times
 *     the chosen block on all cores again (ActualTime), and quality =
 *     (ActualTime - MinTime) / MinTime (Sec. 3.6);
 *   - candidates per axis by the P-part rule of Sec. 3.7 on the block
 *     extents: b[0] = 1, b[m] = min(S, floor(m S / (P-1)) + 1), duplicates
 *     dropped, for bi over nx, bj over ny and bk over the slab depth.
 *
 * Every point is evaluated with one fixed expression order whatever the
 * block, so any two blockings give the same bits.  Layout x fastest, then y,
 * then z; neighbours outside the grid read as zero; u^{n+1} is written over
 * u^{n-1} point by point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HM_MAX_R 8

typedef struct {
    int32_t nx, ny, nz, R;
    float c[HM_MAX_R + 1];       /* weights c_0 .. c_R (FP32) */
    const float *kappa;          /* v^2 dt^2 / dx^2 */
    int32_t sx, sy, sz;          /* source point, sx < 0: none */
    float src_scale;             /* amp v_s^2 dt^2 */
    double f, t0, dt;            /* Ricker */
} hm_grid;

static double hm_now(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

static inline float hm_at(const hm_grid *g, const float *u, long i, long j, long k)
{
    if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) return 0.0f;
    return u[(k * g->ny + j) * (long)g->nx + i];
}

/* Lambda(u) at one point in FP32: centre, then r ascending, each r summing
 * -x, +x, -y, +y, -z, +z left to right before the multiply by c_r. */
static inline float hm_lap_checked(const hm_grid *g, const float *u, long i, long j, long k)
{
    float acc = 3.0f * g->c[0] * hm_at(g, u, i, j, k);
    for (int r = 1; r <= g->R; ++r) {
        float s = hm_at(g, u, i - r, j, k);
        s += hm_at(g, u, i + r, j, k);
        s += hm_at(g, u, i, j - r, k);
        s += hm_at(g, u, i, j + r, k);
        s += hm_at(g, u, i, j, k - r);
        s += hm_at(g, u, i, j, k + r);
        acc += g->c[r] * s;
    }
    return acc;
}

/* One row segment [i0, i1) of row (j, k): the same expression; the part at
 * least R from the x faces reads its neighbours directly (and vectorises),
 * the rest through the checked reader. */
static void hm_row(const hm_grid *g, const float *u, float *up, long j, long k, long i0, long i1)
{
    const long nx = g->nx, ny = g->ny, R = g->R;
    const long sy = nx, sz = nx * ny;
    const int inner_jk = j >= R && j < ny - R && k >= R && k < g->nz - R;
    long a = i0, b = i1;
    if (inner_jk) {
        if (a < R) a = R < i1 ? R : i1;
        if (b > nx - R) b = nx - R > a ? nx - R : a;
    } else {
        a = b = i1;
    }
    const long row = (k * ny + j) * nx;
    for (long i = i0; i < a; ++i)
        up[row + i] = 2.0f * u[row + i] - up[row + i] + g->kappa[row + i] * hm_lap_checked(g, u, i, j, k);
    const float c0x3 = 3.0f * g->c[0];
    for (long i = a; i < b; ++i) {
        const float *p = u + row + i;
        float acc = c0x3 * p[0];
        for (int r = 1; r <= R; ++r) {
            float s = p[-r];
            s += p[r];
            s += p[-r * sy];
            s += p[r * sy];
            s += p[-r * sz];
            s += p[r * sz];
            acc += g->c[r] * s;
        }
        up[row + i] = 2.0f * u[row + i] - up[row + i] + g->kappa[row + i] * acc;
    }
    for (long i = b; i < i1; ++i)
        up[row + i] = 2.0f * u[row + i] - up[row + i] + g->kappa[row + i] * hm_lap_checked(g, u, i, j, k);
}

static double hm_ricker(double f, double t0, double t)
{
    const double pi = 3.14159265358979323846;
    const double a = pi * pi * f * f * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * exp(-a);
}

/* Blocks of one sweep, k-major (Fig. 1b), dealt to the threads in order. */
static void hm_sweep_once(const hm_grid *g, const float *u, float *up, int bi, int bj, int bk, int par)
{
    const long nbi = (g->nx + bi - 1) / bi, nbj = (g->ny + bj - 1) / bj, nbk = (g->nz + bk - 1) / bk;
    const long nb = nbi * nbj * nbk;
    #pragma omp parallel for schedule(static) if (par)
    for (long b = 0; b < nb; ++b) {
        const long kb = b / (nbi * nbj), jb = (b / nbi) % nbj, ib = b % nbi;
        const long k0 = kb * bk, k1 = k0 + bk < g->nz ? k0 + bk : g->nz;
        const long j0 = jb * bj, j1 = j0 + bj < g->ny ? j0 + bj : g->ny;
        const long i0 = ib * bi, i1 = i0 + bi < g->nx ? i0 + bi : g->nx;
        for (long k = k0; k < k1; ++k)
            for (long j = j0; j < j1; ++j) hm_row(g, u, up, j, k, i0, i1);
    }
}

/* `steps` leapfrog steps from step n0: on entry u = u^{n0}, up = u^{n0-1};
 * on exit u = u^{n0+steps}, up = u^{n0+steps-1} (the buffers swap roles
 * after each step; an odd count leaves them swapped, reported in *swapped).
 * par: 1 = blocks over all threads, 0 = this thread alone. */
static void hm_run_grid(const hm_grid *g, int steps, long n0, int bi, int bj, int bk, float *u, float *up,
                        int par, int *swapped)
{
    float *a = u, *b = up;
    const long plane = (long)g->nx * g->ny;
    for (int s = 0; s < steps; ++s) {
        hm_sweep_once(g, a, b, bi, bj, bk, par);        /* b <- u^{n+1} */
        if (g->sx >= 0) {
            const double w = hm_ricker(g->f, g->t0, (double)(n0 + s) * g->dt);
            b[(long)g->sz * plane + (long)g->sy * g->nx + g->sx] += (float)(g->src_scale * w);
        }
        float *t = a;
        a = b;
        b = t;
    }
    *swapped = (a != u);
}

static void hm_weights(int R, float *c)
{
    /* c_r = 2 (-1)^{r+1} (R!)^2 / (r^2 (R-r)! (R+r)!), c_0 = -2 sum c_r (in FP64, rounded once) */
    double fr = 1.0;
    for (int i = 2; i <= R; ++i) fr *= i;
    double sum = 0.0;
    for (int r = 1; r <= R; ++r) {
        double num = 2.0 * fr * fr * ((r % 2) ? 1.0 : -1.0), den = (double)r * r;
        for (int i = 2; i <= R - r; ++i) den *= i;
        for (int i = 2; i <= R + r; ++i) den *= i;
        c[r] = (float)(num / den);
        sum += num / den;
    }
    c[0] = (float)(-2.0 * sum);
}

/*
 * FP32 blocked run on the caller's arrays (x fastest): steps from n0, in
 * place on u (u^n) and up (u^{n-1}); returns the wall seconds.  bi/bj/bk <= 0
 * mean the whole extent.  nthreads <= 0: all.  Returns < 0 on bad arguments.
 */
double hm_run(int nx, int ny, int nz, int R, const float *kappa, int sx, int sy, int sz, float src_scale,
              double f, double t0, double dt, int steps, long n0, int bi, int bj, int bk, float *u, float *up,
              int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1 || R < 1 || R > HM_MAX_R || steps < 0 || !kappa || !u || !up) return -1.0;
    hm_grid g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.R = R;
    hm_weights(R, g.c);
    g.kappa = kappa;
    g.sx = sx; g.sy = sy; g.sz = sz;
    g.src_scale = src_scale; g.f = f; g.t0 = t0; g.dt = dt;
    if (bi <= 0 || bi > nx) bi = nx;
    if (bj <= 0 || bj > ny) bj = ny;
    if (bk <= 0 || bk > nz) bk = nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int swapped = 0;
    const double t = hm_now();
    hm_run_grid(&g, steps, n0, bi, bj, bk, u, up, 1, &swapped);
    const double el = hm_now() - t;
    if (swapped) {              /* results back into the caller's (u, up) */
        const size_t n = (size_t)nx * ny * nz;
        float *tmp = (float *)malloc(n * sizeof(float));
        if (!tmp) return -1.0;
        memcpy(tmp, u, n * sizeof(float));
        memcpy(u, up, n * sizeof(float));
        memcpy(up, tmp, n * sizeof(float));
        free(tmp);
    }
    return el;
}

/* Sec. 3.7: values of one block axis of extent S in P parts. */
int hm_candidates_1d(int S, int P, int *out)
{
    if (S < 1 || P < 2) return 0;
    int n = 0;
    out[n++] = 1;
    for (int m = 1; m < P; ++m) {
        long b = (long)m * S / (P - 1) + 1;
        if (b > S) b = S;
        int dup = 0;
        for (int q = 0; q < n; ++q) dup |= out[q] == (int)b;
        if (!dup) out[n++] = (int)b;
    }
    return n;
}

/*
 * MWMB on the host's T cores for an nx x ny x nz grid of the given velocity
 * model (kappa, x fastest): each core gets a private instance of the slab of
 * planes [t nz / T, (t+1) nz / T) (its kappa; fields zero but for a unit
 * spike, so the arithmetic is that of a live wave), candidates from the
 * P-part rule on (nx, ny, slab depth), nI sweeps timed per candidate.
 * Outputs: block[3] (bi, bj, bk), times[T * nC] (seconds per nI sweeps,
 * core-major) when not null and cap >= T * nC, *min_time (the stage-2
 * time), *actual_time (verification: every core runs the chosen block
 * again, the slowest core's time), *ncand.  Returns 0, or -1 on bad
 * arguments or memory.
 */
int hm_select_mwmb(int nx, int ny, int nz, int R, const float *kappa, int P, int nI, int nthreads, int *block,
                   double *times, long cap, double *min_time, double *actual_time, int *ncand)
{
    if (nx < 1 || ny < 1 || nz < 1 || R < 1 || R > HM_MAX_R || P < 2 || nI < 1 || !kappa || !block) return -1;
    int T = 1;
#ifdef _OPENMP
    T = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
    if (T > nz) T = nz;
    if (P > 64) return -1;
    const int nzs = nz / T;                      /* every core's slab depth (the first nzs*T planes) */
    int ci[64], cj[64], ck[64];
    const int ni = hm_candidates_1d(nx, P, ci), nj = hm_candidates_1d(ny, P, cj), nk = hm_candidates_1d(nzs, P, ck);
    const int nC = ni * nj * nk;
    const long plane = (long)nx * ny, slab = plane * nzs;
    float *mem = (float *)calloc((size_t)slab * 3 * T, sizeof(float));
    double *tt = (double *)malloc(sizeof(double) * (size_t)T * nC);
    if (!mem || !tt) { free(mem); free(tt); return -1; }
    #pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        float *k_t = mem + (size_t)slab * 3 * t, *u_t = k_t + slab, *p_t = u_t + slab;
        memcpy(k_t, kappa + (size_t)t * slab, sizeof(float) * (size_t)slab);
        hm_grid g;
        g.nx = nx; g.ny = ny; g.nz = nzs; g.R = R;
        hm_weights(R, g.c);
        g.kappa = k_t;
        g.sx = -1; g.sy = g.sz = 0; g.src_scale = 0.0f; g.f = g.t0 = g.dt = 0.0;
        for (int c = 0; c < nC; ++c) {
            const int bi = ci[c / (nj * nk)], bj = cj[(c / nk) % nj], bk = ck[c % nk];
            memset(u_t, 0, sizeof(float) * (size_t)slab * 2);
            u_t[(size_t)(nzs / 2) * plane + (size_t)(ny / 2) * nx + nx / 2] = 1.0f;
            int sw;
            #pragma omp barrier
            const double a = hm_now();
            hm_run_grid(&g, nI, 0, bi, bj, bk, u_t, p_t, 0, &sw);
            tt[(size_t)t * nC + c] = hm_now() - a;
        }
    }
    /* stage 1: each core's fastest candidate; stage 2 (MWMB, Eq. 2): the
     * slowest of those; ties to the lowest index */
    int worst = -1, pick = 0;
    double worst_t = 0.0;
    for (int t = 0; t < T; ++t) {
        int best = 0;
        for (int c = 1; c < nC; ++c)
            if (tt[(size_t)t * nC + c] < tt[(size_t)t * nC + best]) best = c;
        const double bt = tt[(size_t)t * nC + best];
        if (worst < 0 || bt > worst_t) {
            worst = t;
            worst_t = bt;
            pick = best;
        }
    }
    block[0] = ci[pick / (nj * nk)];
    block[1] = cj[(pick / nk) % nj];
    block[2] = ck[pick % nk];
    if (min_time) *min_time = worst_t;
    if (ncand) *ncand = nC;
    if (times && cap >= (long)T * nC) memcpy(times, tt, sizeof(double) * (size_t)T * nC);
    /* verification phase: all cores run the chosen block again */
    double act = 0.0;
    #pragma omp parallel num_threads(T) reduction(max : act)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        float *k_t = mem + (size_t)slab * 3 * t, *u_t = k_t + slab, *p_t = u_t + slab;
        hm_grid g;
        g.nx = nx; g.ny = ny; g.nz = nzs; g.R = R;
        hm_weights(R, g.c);
        g.kappa = k_t;
        g.sx = -1; g.sy = g.sz = 0; g.src_scale = 0.0f; g.f = g.t0 = g.dt = 0.0;
        memset(u_t, 0, sizeof(float) * (size_t)slab * 2);
        u_t[(size_t)(nzs / 2) * plane + (size_t)(ny / 2) * nx + nx / 2] = 1.0f;
        int sw;
        #pragma omp barrier
        const double a = hm_now();
        hm_run_grid(&g, nI, 0, block[0], block[1], block[2], u_t, p_t, 0, &sw);
        act = hm_now() - a;
    }
    if (actual_time) *actual_time = act;
    free(mem);
    free(tt);
    return 0;
}

int hm_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
