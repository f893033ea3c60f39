/*
 * FP64 CPU oracle for the acoustic leapfrog finite-difference sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header or table with
 * the CUDA library: the coefficients, the CFL bound, the wavelet and the
 * sweep are all written out again here from their definitions.
 *
 * What it computes (Sec. 2 of the paper, Fig. 1a and Algorithm 1 "RTM()"):
 * the "3D model" step of reverse-time migration, a finite-difference
 * solution of the acoustic wave equation that is 2nd order in time and of
 * order 2R in space (the paper fixes 10th order, i.e. R = 5, "five points in
 * each direction for each dimension"; R = 4 is also supported).  One time
 * step, for every grid point p,
 *
 *     u^{n+1}[p] = 2 u^n[p] - u^{n-1}[p] + kappa[p] * Lambda(u^n)[p]
 *     kappa[p]   = v[p]^2 dt^2 / dx^2
 *     Lambda(u)[p] = 3 c_0 u[p]
 *                  + sum_{r=1..R} c_r ( u[p-r ex] + u[p+r ex] + u[p-r ey]
 *                                     + u[p+r ey] + u[p-r ez] + u[p+r ez] )
 *
 * followed by the point-source injection u^{n+1}[s] += v_s^2 dt^2 w(n dt).
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - c_r are the exact central 2nd-derivative weights of order 2R (the paper
 *     prints none); closed form below;
 *   - neighbours outside [0,n) read as zero (homogeneous Dirichlet through
 *     ghost zeros) and every grid point is an unknown;
 *   - u^0 = u^{-1} = 0 unless the caller supplies a start state;
 *   - w is a Ricker wavelet, w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2)
 *     with tau = t - t0, added after the stencil at step n with t = n dt.
 *
 * Layout: x fastest, then y, then z (one axis contiguous in memory, Sec. 2).
 * Index p = (k*ny + j)*nx + i.
 *
 * The blocked traversal of Sec. 3 (loop tiling with a blocksize (bi,bj,bk),
 * Fig. 1b) changes only the order in which points are visited; every point's
 * expression is evaluated with the same operation order, so blocked and
 * unblocked sweeps agree bit for bit.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (contraction off so
 * x86 and Arm hosts round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_R 8

static int64_t gcd64(int64_t a, int64_t b)
{
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

static int64_t fact64(int n)
{
    int64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/*
 * Exact rational weights of the order-2R central second difference,
 *   c_r = 2 (-1)^{r+1} (R!)^2 / ( r^2 (R-r)! (R+r)! ),  r = 1..R
 *   c_0 = -2 sum_{r>=1} c_r
 * (the weights that make the stencil exact on polynomials of degree <= 2R+1).
 * num[r]/den[r], den > 0, fully reduced.  Returns 0, or -1 for R out of range.
 */
int oracle_fd_coeffs_rational(int R, int64_t *num, int64_t *den)
{
    if (R < 1 || R > 6) return -1;     /* 6!^2 * 12! still fits in int64 */
    int64_t rf2 = fact64(R) * fact64(R);
    int64_t s_num = 0, s_den = 1;       /* running sum of c_r, r >= 1 */
    for (int r = 1; r <= R; ++r) {
        int64_t n = 2 * rf2 * ((r % 2 == 1) ? 1 : -1);
        int64_t d = (int64_t)r * r * fact64(R - r) * fact64(R + r);
        int64_t g = gcd64(n, d);
        num[r] = n / g;
        den[r] = d / g;
        /* s += num[r]/den[r] */
        int64_t nn = s_num * den[r] + num[r] * s_den;
        int64_t dd = s_den * den[r];
        int64_t g2 = gcd64(nn, dd);
        if (g2 == 0) g2 = 1;
        s_num = nn / g2;
        s_den = dd / g2;
    }
    num[0] = -2 * s_num;
    den[0] = s_den;
    int64_t g0 = gcd64(num[0], den[0]);
    num[0] /= g0;
    den[0] /= g0;
    return 0;
}

/* c[0..R] as doubles: each is one correctly rounded division num/den. */
int oracle_fd_coeffs(int R, double *c)
{
    int64_t num[ORACLE_MAX_R + 1], den[ORACLE_MAX_R + 1];
    if (oracle_fd_coeffs_rational(R, num, den)) return -1;
    for (int r = 0; r <= R; ++r) c[r] = (double)num[r] / (double)den[r];
    return 0;
}

/*
 * Von Neumann stability bound on the Courant number v dt / dx for the 3D
 * leapfrog scheme.  The 1D symbol of the second difference,
 * c_0 + 2 sum c_r cos(r theta), has its largest magnitude W = |c_0| + 2 sum|c_r|
 * at theta = pi (the weights alternate in sign); stability of the 3D leapfrog
 * needs (v dt/dx)^2 * 3 W <= 4, i.e.  v dt/dx <= 2 / sqrt(3 W).
 */
double oracle_cfl_limit(int R)
{
    double c[ORACLE_MAX_R + 1];
    if (oracle_fd_coeffs(R, c)) return -1.0;
    double W = fabs(c[0]);
    for (int r = 1; r <= R; ++r) W += 2.0 * fabs(c[r]);
    return 2.0 / sqrt(3.0 * W);
}

/* Ricker wavelet of peak frequency f (Hz) centred on t0 (s). */
double oracle_ricker(double f, double t0, double t)
{
    const double pi = 3.14159265358979323846;
    double tau = t - t0;
    double a = pi * pi * f * f * tau * tau;
    return (1.0 - 2.0 * a) * exp(-a);
}

typedef struct {
    int nx, ny, nz, R;
    double c[ORACLE_MAX_R + 1];
} grid_t;

/* u at (i,j,k), zero outside the grid (ghost zeros). */
static inline double at(const grid_t *g, const double *u, long i, long j, long k)
{
    if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) return 0.0;
    return u[(k * g->ny + j) * (long)g->nx + i];
}

/* Lambda(u) at one point, unit spacing.  Fixed order: centre term, then
 * r ascending, and within each r the six neighbours -x,+x,-y,+y,-z,+z summed
 * left to right before the multiply by c_r.  Points at least R away from
 * every face read their neighbours directly; the others through at(); both
 * paths evaluate the same expression in the same order. */
static inline double lap_point(const grid_t *g, const double *u, long i, long j, long k)
{
    const int R = g->R;
    if (i >= R && i < g->nx - R && j >= R && j < g->ny - R && k >= R && k < g->nz - R) {
        const long sx = 1, sy = g->nx, sz = (long)g->nx * g->ny;
        const double *c = u + (k * g->ny + j) * (long)g->nx + i;
        double acc = 3.0 * g->c[0] * c[0];
        for (int r = 1; r <= R; ++r) {
            double s = c[-r * sx];
            s += c[r * sx];
            s += c[-r * sy];
            s += c[r * sy];
            s += c[-r * sz];
            s += c[r * sz];
            acc += g->c[r] * s;
        }
        return acc;
    }
    double acc = 3.0 * g->c[0] * at(g, u, i, j, k);
    for (int r = 1; r <= R; ++r) {
        double s = at(g, u, i - r, j, k);
        s += at(g, u, i + r, j, k);
        s += at(g, u, i, j - r, k);
        s += at(g, u, i, j + r, k);
        s += at(g, u, i, j, k - r);
        s += at(g, u, i, j, k + r);
        acc += g->c[r] * s;
    }
    return acc;
}

static int grid_init(grid_t *g, int nx, int ny, int nz, int R)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    g->nx = nx; g->ny = ny; g->nz = nz; g->R = R;
    return oracle_fd_coeffs(R, g->c);
}

/* out = Lambda(u), unit grid spacing, ghost zeros. */
int oracle_laplacian(int nx, int ny, int nz, int R, const double *u, double *out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, R)) return -1;
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i)
                out[(k * ny + j) * (long)nx + i] = lap_point(&g, u, i, j, k);
    return 0;
}

typedef struct {
    int32_t nx, ny, nz, R;
    double dx, dt;
    const double *v;          /* velocity, nx*ny*nz, m/s */
    int32_t sx, sy, sz;       /* source grid index */
    double f, t0;             /* Ricker peak frequency and delay */
    double amp;               /* source amplitude multiplier (0 = no source) */
    int64_t n0;               /* absolute index of the first step taken */
} oracle_problem;

/*
 * Advance `steps` leapfrog steps (Algorithm 1's time loop, 3D-model step
 * only).  On entry u holds u^{n0}, u_prev holds u^{n0-1}; on exit u holds
 * u^{n0+steps} and u_prev u^{n0+steps-1}.  The sweep over points is done in
 * blocks of bi x bj x bk (0 = the whole extent, i.e. unblocked), blocks in
 * k, j, i order and points in each block in k, j, i order (Fig. 1b).
 * OpenMP threads split the k-blocks; that changes no arithmetic.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_run(const oracle_problem *p, int steps, int bi, int bj, int bk,
               double *u, double *u_prev, int nthreads)
{
    grid_t g;
    if (!p || !u || !u_prev || !p->v || steps < 0) return -1;
    if (grid_init(&g, p->nx, p->ny, p->nz, p->R)) return -1;
    const long nx = p->nx, ny = p->ny, nz = p->nz;
    const long n = nx * ny * nz;
    if (bi <= 0 || bi > nx) bi = (int)nx;
    if (bj <= 0 || bj > ny) bj = (int)ny;
    if (bk <= 0 || bk > nz) bk = (int)nz;
    double *kappa = (double *)malloc(sizeof(double) * n);
    double *spare = (double *)malloc(sizeof(double) * n);
    if (!kappa || !spare) { free(kappa); free(spare); return -1; }
    double *const u_out = u, *const up_out = u_prev;
    double *next = spare;
    const double dt2 = p->dt * p->dt, dx2 = p->dx * p->dx;
    /* each element's expression is independent of the thread count */
    #pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) kappa[q] = p->v[q] * p->v[q] * dt2 / dx2;
    const int has_src = p->amp != 0.0 && p->sx >= 0 && p->sx < nx && p->sy >= 0 &&
                        p->sy < ny && p->sz >= 0 && p->sz < nz;
    const long s = has_src ? ((long)p->sz * ny + p->sy) * nx + p->sx : 0;
    const long nbk = (nz + bk - 1) / bk;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    const int nt = 1;
#endif
    for (int step = 0; step < steps; ++step) {
        /* OpenMP splits the k-blocks when there are enough of them, else the
         * planes inside each block; either way each point is written once
         * with the same expression. */
        const int par_blocks = nbk >= 2 * nt;
        #pragma omp parallel for schedule(static) if (par_blocks) num_threads(nt)
        for (long kb = 0; kb < nbk; ++kb) {
            const long k0 = kb * bk, k1 = (k0 + bk < nz) ? k0 + bk : nz;
            for (long j0 = 0; j0 < ny; j0 += bj) {
                const long j1 = (j0 + bj < ny) ? j0 + bj : ny;
                for (long i0 = 0; i0 < nx; i0 += bi) {
                    const long i1 = (i0 + bi < nx) ? i0 + bi : nx;
                    #pragma omp parallel for schedule(static) if (!par_blocks) num_threads(nt)
                    for (long k = k0; k < k1; ++k)
                        for (long j = j0; j < j1; ++j)
                            for (long i = i0; i < i1; ++i) {
                                const long q = (k * ny + j) * nx + i;
                                next[q] = 2.0 * u[q] - u_prev[q] + kappa[q] * lap_point(&g, u, i, j, k);
                            }
                }
            }
        }
        if (has_src) {
            const double t = (double)(p->n0 + step) * p->dt;
            next[s] += p->amp * p->v[s] * p->v[s] * dt2 * oracle_ricker(p->f, p->t0, t);
        }
        /* rotate: u_prev <- u, u <- next (the old u_prev buffer is reused) */
        double *old_prev = u_prev;
        u_prev = u;
        u = next;
        next = old_prev;
    }
    /* Each step rotates (u, u_prev, next) -> (next, u, u_prev); move the
     * results back into the caller's two arrays. */
    if (u == spare) {              /* steps = 1 mod 3: u_prev is u_out */
        memcpy(up_out, u_out, sizeof(double) * n);
        memcpy(u_out, spare, sizeof(double) * n);
    } else if (u == up_out) {      /* steps = 2 mod 3: u_prev is spare */
        memcpy(u_out, up_out, sizeof(double) * n);
        memcpy(up_out, spare, sizeof(double) * n);
    }
    free(kappa);
    free(spare);
    return 0;
}

/*
 * The time loop with the pieces an RTM code adds around the 3D-model step
 * (the paper names RTM but prints none of them; readings in the design
 * notes):
 *   - an absorbing layer: the damped wave equation u_tt + 2 sigma u_t =
 *     v^2 Laplacian(u), centred in time, i.e. with eta = sigma dt
 *         u^{n+1} = (2 u^n - (1 - eta) u^{n-1} + kappa Lambda(u^n)) / (1 + eta),
 *     eta = eta_max ((W - d) / W)^2 within W points of a face (d = distance
 *     in points to the nearest face, 0 on the face), 0 elsewhere; with
 *     eta = 0 the expression is the plain update, bit for bit;
 *   - the point source (as oracle_run);
 *   - an injection on the plane z = inj_z (one row y = inj_y, or all rows
 *     when inj_y < 0): u^{n+1} += inj_scale * inj[m] at step m of this call,
 *     m counted from 0, with inj[inj_steps - 1 - m] instead when
 *     inj_reverse (time-reversed data, the adjoint source of RTM); steps
 *     beyond inj_steps inject nothing;
 *   - a record of u^{n+1} on the plane z = rec_z (row rec_y, or all rows)
 *     into rec[m] after every step m < rec_steps.
 * Layout of inj and rec: [step][rows][nx], rows = ny or 1.  Unblocked; the
 * same OpenMP plane split as oracle_run.
 */
typedef struct {
    int32_t width;          /* absorbing layer in points (0 = none) */
    double eta_max;
    int32_t inj_z, inj_y;   /* inj_z < 0: no injection */
    const double *inj;
    int32_t inj_steps, inj_reverse;
    double inj_scale;
    int32_t rec_z, rec_y;   /* rec_z < 0: no record */
    double *rec;
    int32_t rec_steps;
} oracle_ext;

/* eta at (i,j,k) for a layer of `w` points. */
double oracle_eta(int nx, int ny, int nz, int w, double eta_max, long i, long j, long k)
{
    if (w <= 0) return 0.0;
    long d = i;
    if (nx - 1 - i < d) d = nx - 1 - i;
    if (j < d) d = j;
    if (ny - 1 - j < d) d = ny - 1 - j;
    if (k < d) d = k;
    if (nz - 1 - k < d) d = nz - 1 - k;
    if (d >= w) return 0.0;
    const double a = (double)(w - d) / (double)w;
    return eta_max * a * a;
}

int oracle_run_ext(const oracle_problem *p, const oracle_ext *e, int steps, double *u, double *u_prev,
                   int nthreads)
{
    grid_t g;
    if (!p || !e || !u || !u_prev || !p->v || steps < 0) return -1;
    if (grid_init(&g, p->nx, p->ny, p->nz, p->R)) return -1;
    const long nx = p->nx, ny = p->ny, nz = p->nz;
    const long n = nx * ny * nz;
    if (e->inj_z >= nz || e->inj_y >= ny || e->rec_z >= nz || e->rec_y >= ny) return -1;
    if ((e->inj_z >= 0 && !e->inj) || (e->rec_z >= 0 && !e->rec)) return -1;
    double *kappa = (double *)malloc(sizeof(double) * n);
    double *eta = (double *)malloc(sizeof(double) * n);
    double *next = (double *)malloc(sizeof(double) * n);
    if (!kappa || !eta || !next) { free(kappa); free(eta); free(next); return -1; }
    const double dt2 = p->dt * p->dt, dx2 = p->dx * p->dx;
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                const long q = (k * ny + j) * nx + i;
                kappa[q] = p->v[q] * p->v[q] * dt2 / dx2;
                eta[q] = oracle_eta((int)nx, (int)ny, (int)nz, e->width, e->eta_max, i, j, k);
            }
    const int has_src = p->amp != 0.0 && p->sx >= 0 && p->sx < nx && p->sy >= 0 &&
                        p->sy < ny && p->sz >= 0 && p->sz < nz;
    const long s = has_src ? ((long)p->sz * ny + p->sy) * nx + p->sx : 0;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    const int nt = 1;
#endif
    const long inj_rows = e->inj_y < 0 ? ny : 1, rec_rows = e->rec_y < 0 ? ny : 1;
    for (int step = 0; step < steps; ++step) {
        #pragma omp parallel for schedule(static) num_threads(nt)
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < nx; ++i) {
                    const long q = (k * ny + j) * nx + i;
                    next[q] = (2.0 * u[q] - (1.0 - eta[q]) * u_prev[q] + kappa[q] * lap_point(&g, u, i, j, k)) /
                              (1.0 + eta[q]);
                }
        if (has_src) {
            const double t = (double)(p->n0 + step) * p->dt;
            next[s] += p->amp * p->v[s] * p->v[s] * dt2 * oracle_ricker(p->f, p->t0, t);
        }
        if (e->inj_z >= 0 && step < e->inj_steps) {
            const long m = e->inj_reverse ? e->inj_steps - 1 - step : step;
            const double *d = e->inj + m * inj_rows * nx;
            for (long r = 0; r < inj_rows; ++r) {
                const long j = e->inj_y < 0 ? r : e->inj_y;
                for (long i = 0; i < nx; ++i) next[((long)e->inj_z * ny + j) * nx + i] += e->inj_scale * d[r * nx + i];
            }
        }
        if (e->rec_z >= 0 && step < e->rec_steps) {
            double *d = e->rec + (long)step * rec_rows * nx;
            for (long r = 0; r < rec_rows; ++r) {
                const long j = e->rec_y < 0 ? r : e->rec_y;
                memcpy(d + r * nx, next + ((long)e->rec_z * ny + j) * nx, sizeof(double) * nx);
            }
        }
        /* u_prev <- u, u <- next, through copies (the caller's arrays stay put) */
        memcpy(u_prev, u, sizeof(double) * n);
        memcpy(u, next, sizeof(double) * n);
    }
    free(kappa);
    free(eta);
    free(next);
    return 0;
}

/*
 * Discrete energy of the leapfrog scheme between levels n and n+1,
 *   E^{n+1/2} = sum_p [ (u1[p]-u0[p])^2 / kappa[p] - u1[p] * Lambda(u0)[p] ],
 * kappa = v^2 dt^2/dx^2.  This is dx^2 times the scheme's energy
 * (1/dt^2) sum (u1-u0)^2/v^2 + sum u1 * (-Lambda/dx^2) u0.  With ghost zeros
 * Lambda is a symmetric matrix, so for a source-free run the quantity is
 * exactly conserved by the scheme (up to rounding).
 * Summation: one partial per k-plane (points in j, i order), then the planes
 * in k order, so the result does not depend on the thread count.
 */
double oracle_energy(int nx, int ny, int nz, int R, double dx, double dt,
                     const double *v, const double *u1, const double *u0)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz, R)) return NAN;
    double *part = (double *)calloc((size_t)nz, sizeof(double));
    if (!part) return NAN;
    const double dt2 = dt * dt, dx2 = dx * dx;
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k) {
        double acc = 0.0;
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                const long q = (k * ny + j) * (long)nx + i;
                const double kap = v[q] * v[q] * dt2 / dx2;
                const double d = u1[q] - u0[q];
                acc += d * d / kap - u1[q] * lap_point(&g, u0, i, j, k);
            }
        part[k] = acc;
    }
    double e = 0.0;
    for (long k = 0; k < nz; ++k) e += part[k];
    free(part);
    return e;
}

/* sum_p (a[p]-b[p])^2 and sum_p b[p]^2, per-plane partials then k order. */
int oracle_sq_diff(long nplanes, long plane, const double *a, const double *b,
                   double *diff2, double *ref2)
{
    double *pd = (double *)calloc((size_t)nplanes, sizeof(double));
    double *pr = (double *)calloc((size_t)nplanes, sizeof(double));
    if (!pd || !pr) { free(pd); free(pr); return -1; }
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < nplanes; ++k) {
        double sd = 0.0, sr = 0.0;
        for (long q = k * plane; q < (k + 1) * plane; ++q) {
            const double d = a[q] - b[q];
            sd += d * d;
            sr += b[q] * b[q];
        }
        pd[k] = sd;
        pr[k] = sr;
    }
    double sd = 0.0, sr = 0.0;
    for (long k = 0; k < nplanes; ++k) { sd += pd[k]; sr += pr[k]; }
    *diff2 = sd;
    *ref2 = sr;
    free(pd);
    free(pr);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
