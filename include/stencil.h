/*
 * libstencil -- GB300 (sm_103a) acoustic finite-difference stencil sweep.
 *
 * The operation (Sec. 2 of "Improving Memory Hierarchy Utilisation for
 * Stencil Computations on Multicore Machines", Fig. 1a, and the time loop of
 * Algorithm 1 "RTM()"): the "3D model" step of reverse-time migration, an
 * explicit finite-difference solution of the acoustic wave equation, 2nd
 * order in time and of order 2R in space (R = 5 is the paper's 10th order,
 * "five points in each direction for each dimension"; R = 4 is 8th order).
 * One time step n -> n+1 updates every grid point p:
 *
 *   u^{n+1}[p] = 2 u^n[p] - u^{n-1}[p] + kappa[p] * Lambda(u^n)[p]
 *   kappa[p]   = v[p]^2 dt^2 / dx^2
 *   Lambda(u)[p] = 3 c_0 u[p] + sum_{r=1..R} c_r (u[p -+ r e_x] + u[p -+ r e_y] + u[p -+ r e_z])
 *   u^{n+1}[s] += src_amp * v[s]^2 dt^2 * w(n dt)      (point source at s)
 *
 * with c_r the exact central second-difference weights of order 2R,
 * neighbours outside the grid read as 0 (homogeneous Dirichlet through ghost
 * zeros), u^0 = u^{-1} = 0 by default, and w the Ricker wavelet
 * w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0.
 *
 * Conventions for every entry point:
 *   - returns STENCIL_OK (0) or a negative STENCIL_E* code; no C++ exception
 *     crosses this boundary; stencil_last_error() gives a message for the
 *     calling thread's last failure;
 *   - arrays are 3D, x fastest, then y, then z: element (i,j,k) of a dense
 *     array is at (k*ny + j)*nx + i; "dense" means exactly nx*ny*nz elements;
 *   - the caller owns every array it passes; a plan copies what it keeps;
 *   - a pointer flagged "on device" is a CUDA device pointer on the device
 *     that was current when the plan was made; otherwise it is host memory;
 *   - a plan is used by one host thread at a time; different plans (each
 *     on its own stream) may be driven from different threads at once, and
 *     a call that waits waits only for its own plan's stream; a shot server
 *     is thread-safe.
 */
#ifndef STENCIL_H
#define STENCIL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STENCIL_API __attribute__((visibility("default")))
#else
#define STENCIL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define STENCIL_OK               0
#define STENCIL_EINVAL          -1  /* bad argument: dims <= 0, radius not 4/5, null pointer, source outside grid, v <= 0 ... */
#define STENCIL_ECFL            -2  /* dt above the stability bound for the largest velocity */
#define STENCIL_ENOMEM          -3  /* device allocation failed */
#define STENCIL_EBUDGET         -4  /* request larger than the whole memory budget */
#define STENCIL_ETIMEOUT        -5  /* a bounded device-side wait gave up */
#define STENCIL_ECUDA           -6  /* a CUDA call failed (message kept) */
#define STENCIL_ENOTREADY       -7  /* result not available yet */
#define STENCIL_EUNKNOWN_TICKET -8  /* no such shot ticket */
#define STENCIL_ENODEV          -9  /* no usable CUDA device */
#define STENCIL_EUNSUPPORTED   -10  /* configuration not built into this library */
#define STENCIL_ECANCELLED     -11  /* the shot was cancelled (server shut down before admitting it) */

/* ---- enums ----------------------------------------------------------- */
typedef enum {
    STENCIL_FP32 = 0,   /* u, u_prev stored in FP32 */
    STENCIL_FP16 = 1,   /* u and d = u - u_prev stored in FP16, each with per-z-plane FP32 scales */
    STENCIL_BF16 = 2    /* u and d = u - u_prev stored in BF16, each with per-z-plane FP32 scales */
} stencil_storage;

typedef enum {
    STENCIL_KERNEL_AUTO  = 0,  /* library default: the naive kernel for FP32 grids of at most 2^20
                                  points (latency-bound), else the tiled kernel, default tile */
    STENCIL_KERNEL_NAIVE = 1,  /* one thread per point, neighbours straight from global memory */
    STENCIL_KERNEL_TILED = 2,  /* 2.5D blocking: TMA-staged xy tile + halo, z-marching register queue */
    STENCIL_KERNEL_TWO_STEP = 3 /* two time steps per sweep (temporal blocking, the "3.5D" blocking
                                  of the paper's related work, Sec. 4): the first step on the tile
                                  plus a ring of R points, the second on the tile; 10 B of traffic
                                  per point update instead of 16.  FP32 storage only, no absorbing
                                  layer, recording, injection, tuning or caller-owned buffers
                                  (STENCIL_EUNSUPPORTED); tile fixed at 64 x 16 (R = 4) or 64 x 14
                                  (R = 5), tx and ty are ignored; an odd step count ends with one
                                  step of the tiled kernel.  The plan holds four FP32 wavefields. */
} stencil_kernel;

/* Tile parameters of the tiled kernel, the GPU analogue of the paper's
 * blocksize (i, j, k) (Sec. 3, Fig. 1b): tx x ty points of an xy plane per
 * thread block, marching over zchunk planes in z.  tx in {32, 64, 128},
 * ty in {4, 8, 16, 32} (stencil_tile_info says which are built);
 * zchunk >= 1, 0 = the whole nz, < 0 = chosen by the library from a model
 * of how the blocks fill the GPU. */
typedef struct {
    int32_t kernel;     /* stencil_kernel */
    int32_t tx, ty;
    int32_t zchunk;
} stencil_tile;

/* How stencil_plan picks the tile (Sec. 3.2-3.3 re-run on GPU tile parameters). */
typedef enum {
    STENCIL_TUNE_NONE       = 0,  /* use desc.tile as given (kernel AUTO = default tile) */
    STENCIL_TUNE_OWN        = 1,  /* library autotuner: time every feasible tile once, take the fastest */
    STENCIL_TUNE_MWMB       = 2,  /* three-stage selection, stage 2 = max (Eq. 2) */
    STENCIL_TUNE_OB         = 3,  /* original block: each stream its own candidates, global min */
    STENCIL_TUNE_MMMB       = 4,  /* three-stage selection, stage 2 = min (Eq. 1) */
    STENCIL_TUNE_MAMB       = 5,  /* three-stage selection, stage 2 = closest to mean (Eq. 3) */
    STENCIL_TUNE_EXHAUSTIVE = 6   /* every feasible tile, timed with all streams running it */
} stencil_tune_mode;

/* Selection-phase parameters (Sec. 3.2): nI iterations per candidate, C
 * concurrent streams (the "cores" that share L2 and HBM), N groups (the
 * "nodes"), P parts per parameter axis for the candidate list (Sec. 3.7). */
typedef struct {
    int32_t parts;        /* P, default 5 */
    int32_t iterations;   /* nI, default 8 */
    int32_t streams;      /* C, default 4 */
    int32_t groups;       /* N, default 2 */
} stencil_tune_params;

/* Problem description (the paper's statement of the problem: grid, order,
 * spacing, time step, velocity model, source).  Initialise with
 * stencil_desc_init() and then set fields. */
typedef struct {
    int32_t nx, ny, nz;          /* grid points per axis, >= 1 */
    int32_t radius;              /* R = 4 (8th order) or 5 (10th order) */
    double  dx;                  /* grid spacing, m (> 0) */
    double  dt;                  /* time step, s (> 0, checked against the CFL bound) */
    const float *velocity;       /* dense nx*ny*nz, m/s, every value > 0 and finite */
    int32_t velocity_on_device;  /* 1 if velocity is a device pointer */
    int32_t src_x, src_y, src_z; /* source grid index, inside the grid */
    double  src_freq_hz;         /* Ricker peak frequency f (> 0) */
    double  src_t0;              /* Ricker delay t0, s; < 0 means 1/f */
    double  src_amp;             /* source amplitude multiplier; 0 = no source */
    int32_t storage;             /* stencil_storage */
    int32_t tune_mode;           /* stencil_tune_mode */
    stencil_tile tile;           /* used when tune_mode == STENCIL_TUNE_NONE */
    stencil_tune_params tune;    /* used by the selection modes */
    void   *cuda_stream;         /* cudaStream_t to run on; NULL = the plan creates its own
                                    non-blocking stream (the legacy default stream, handle 0,
                                    cannot be requested: graphs cannot be captured on it) */
    int32_t graph_steps;         /* steps per captured CUDA graph; 0 = launch step by step */
    void   *user_buffers[3];     /* optional caller-owned device buffers, all three or none
                                    (NULL = the plan allocates): [0] and [1] the two wavefield
                                    levels, [2] kappa; each dense nx*ny*nz FP32 (x fastest),
                                    16-byte aligned, and nx a multiple of 4 (the rows are TMA
                                    strides), else STENCIL_EINVAL; FP32 storage only, else
                                    STENCIL_EUNSUPPORTED.  The plan zeroes [0] and [1] (u^0 =
                                    u^{-1} = 0) and writes kappa into [2]; u^n is then in
                                    user_buffers[stats.current_buffer].  They stay the caller's
                                    and must outlive the plan; the shot server does not take them. */
    int32_t absorb_width;        /* absorbing layer: points from each face, 0..255 (0 = none, the
                                    plain ghost-zero boundary; larger: STENCIL_EINVAL); FP32
                                    storage only (16-bit storage is
                                    refused with STENCIL_EUNSUPPORTED).  The tiled kernel applies
                                    it inside the sweep (single plans, batches, the shot server);
                                    the naive kernel as a save of u^{n-1} on the layer before
                                    each sweep and a damping pass after it */
    double  absorb_eta;          /* eta = sigma dt at the face, >= 0: the layer solves the damped
                                    equation u_tt + 2 sigma u_t = v^2 Laplacian(u), centred in time,
                                    u^{n+1} = (2u^n - (1-eta) u^{n-1} + kappa Lambda(u^n)) / (1+eta),
                                    eta = absorb_eta ((W-d)/W)^2 at distance d < W from the nearest
                                    face (the paper names RTM but not its boundary treatment) */
} stencil_desc;

/* Plan state, results of tuning and the device layout. */
typedef struct {
    int64_t steps_done;          /* n of the current level u^n */
    stencil_tile tile;           /* tile in use */
    double  vmax;                /* largest velocity */
    double  cfl;                 /* vmax * dt / dx */
    double  cfl_limit;           /* stability bound on vmax * dt / dx */
    int64_t pitch;               /* row pitch of the device fields, elements */
    int64_t field_bytes;         /* bytes of one device field */
    int64_t device_bytes;        /* bytes the plan holds on the device */
    /* tile selection (NaN when no selection ran) */
    double  min_time_ms;         /* MinTime: the chosen tile's selection-phase time (nI steps) */
    double  actual_time_ms;      /* ActualTime: verification in the selection's setting (nI steps):
                                    all C streams run the chosen tile together, max over streams
                                    (full grid for OWN / EXHAUSTIVE) */
    double  full_time_ms;        /* the chosen tile on the whole grid, nI steps */
    double  quality;             /* (ActualTime - MinTime) / MinTime */
    double  selection_ms;        /* wall time spent selecting */
    int32_t n_candidates;        /* candidates timed */
    int32_t tune_mode;
    int32_t current_buffer;      /* which of the plan's two field buffers holds u^n (0 or 1) */
    int32_t user_buffers;        /* 1 if the plan runs on caller-owned buffers */
} stencil_stats;

typedef struct stencil_plan_s *stencil_plan_t;

/* ---- plan lifecycle --------------------------------------------------- */

/* Fill *d with defaults: radius 5, dx 10, src_freq 15 Hz, t0 = 1/f,
 * src_amp 1, FP32 storage, no tuning, default tile, no graphs.  Dims,
 * dt, velocity and source must still be set. */
STENCIL_API void stencil_desc_init(stencil_desc *d);

/* Build a plan on the current CUDA device: validate *d, allocate the two
 * wavefield buffers and kappa on the device, compute kappa = v^2 dt^2/dx^2
 * (FP32, within 1 ulp of the FP64 product rounded once) and vmax there,
 * check vmax*dt/dx against the CFL bound (STENCIL_ECFL),
 * zero u^0 and u^{-1}, and pick the tile (tune_mode).  Synchronous.  The
 * velocity array is only read during this call. */
STENCIL_API int stencil_plan(const stencil_desc *d, stencil_plan_t *out);

/* Release every device resource of the plan (synchronises its stream). */
STENCIL_API int stencil_destroy(stencil_plan_t p);

/* ---- stepping --------------------------------------------------------- */

/* Enqueue nsteps time steps (Algorithm 1's loop, the 3D-model step, with the
 * source) on the plan's stream; returns without waiting.  nsteps >= 0. */
STENCIL_API int stencil_step(stencil_plan_t p, int32_t nsteps);

/* stencil_step(nsteps), then copy u^n (dense, nx*ny*nz floats) to out_u
 * (host or device per out_on_device; NULL = no copy), then wait for the
 * stream and report any device-side error. */
STENCIL_API int stencil_run(stencil_plan_t p, int32_t nsteps, float *out_u, int32_t out_on_device);

/* Wait for the plan's stream; report device-side errors (STENCIL_ETIMEOUT). */
STENCIL_API int stencil_sync(stencil_plan_t p);

/* ---- state ------------------------------------------------------------ */

/* Copy u^n (which = 0) or u^{n-1} (which = 1) out as a dense FP32 array
 * (16-bit storage: u^{n-1} = u^n - d^n from the two stored fields).
 * Synchronous. */
STENCIL_API int stencil_get_field(stencil_plan_t p, int32_t which, float *out, int32_t out_on_device);

/* Set the state: u^n = u, u^{n-1} = u_prev (dense FP32; NULL = zeros), and
 * the step counter n = step (16-bit storage keeps u^n and d^n = u^n -
 * u^{n-1}, each rounded once with its plane's scale).  Synchronous when it
 * copies from host memory (the arrays may be reused on return).  With
 * device arrays or NULLs it only enqueues the work on the plan's stream:
 * device arrays must stay unchanged until the stream has passed the copy,
 * and device-side errors are reported by the next synchronising call. */
STENCIL_API int stencil_set_fields(stencil_plan_t p, const float *u, const float *u_prev,
                       int32_t on_device, int64_t step);

/* Replace the velocity model of an existing plan (dense nx*ny*nz, host or
 * device): recompute kappa and vmax on the device and re-check the CFL bound
 * with the plan's dt (STENCIL_ECFL leaves the plan unusable until a valid
 * model is set).  The wavefields and step counter are left as they are.
 * Enqueued on the plan's stream; waits for it before returning. */
STENCIL_API int stencil_set_velocity(stencil_plan_t p, const float *velocity, int32_t on_device);

STENCIL_API int stencil_get_stats(stencil_plan_t p, stencil_stats *s);

/* ---- recording inside the time loop ----------------------------------
 * Algorithm 1's loop body records the seismic traces ("sismic") and the
 * energy beside the 3D model step; here the sweep itself writes them after
 * every step n -> n+1 (single-plan stencil_step / stencil_run, either
 * kernel; batched and served shots record nothing).
 *   traces: u^{n+1} on the receiver plane z = receiver_z (receiver_y = -1:
 *           all ny x nx points; else the nx points of row receiver_y), as
 *           stored (exactly what stencil_get_field returns), copied by a
 *           small kernel after each step;
 *   energy: E^{n+1/2} = sum_p (u^{n+1}-u^n)^2 / kappa - u^{n+1} Lambda(u^n)
 *           (conserved by the scheme without a source), summed inside the
 *           sweep: FP32 per warp over a few planes, FP64 over warps and
 *           blocks in a fixed order; not with an absorbing layer or an
 *           injection (STENCIL_EUNSUPPORTED).
 * Record m holds the step from u^{n0+m} to u^{n0+m+1}, n0 = steps_done when
 * recording started; steps beyond `capacity` records are not recorded. */
typedef struct {
    int32_t receiver_z;   /* receiver plane, -1 = no traces */
    int32_t receiver_y;   /* -1 = the whole plane, else one row */
    int32_t energy;       /* 1 = record E^{n+1/2} */
    int32_t capacity;     /* records kept (>= 1) */
} stencil_record_cfg;

/* receiver_z = receiver_y = -1, energy 0, capacity 0. */
STENCIL_API void stencil_record_cfg_init(stencil_record_cfg *c);
/* Start (or restart) recording at the current step: allocates capacity x
 * (ny or 1) x nx floats of traces and capacity + blocks doubles on the
 * device.  STENCIL_EINVAL for a receiver outside the grid, capacity < 1 or
 * nothing to record. */
STENCIL_API int stencil_record_start(stencil_plan_t p, const stencil_record_cfg *c);
/* Copy the records made so far (*nrecorded = min(capacity, steps since the
 * start)): traces into `traces` ([record][ny or 1][nx] floats; device memory
 * if traces_on_device), energies into host `energy` ([record] doubles);
 * either may be NULL.  Waits for the plan's stream. */
STENCIL_API int stencil_record_read(stencil_plan_t p, float *traces, int32_t traces_on_device, double *energy,
                                    int32_t *nrecorded);
/* Stop recording and free its buffers (no-op when not recording). */
STENCIL_API int stencil_record_stop(stencil_plan_t p);

/* ---- RTM pieces: plane injection and the imaging condition ------------
 * Reverse-time migration (the application the paper's kernel serves, Sec. 2)
 * propagates the recorded traces backwards in time from the receiver plane
 * and correlates that wavefield with the source wavefield.  Injection: after
 * every step n -> n+1, u^{n+1} += scale * data[m] on the plane z (row y, or
 * all rows when y < 0), m = n - n0 (n0 = steps_done at the start), or
 * data[steps - 1 - m] when reverse (time-reversed traces); steps outside
 * [0, steps) inject nothing.  data: device memory, [steps][ny or 1][nx]
 * FP32, owned by the caller, read during the plan's steps until
 * stencil_inject_stop.  FP32 storage only (STENCIL_EUNSUPPORTED otherwise:
 * the 16-bit scale bound does not cover injected values).  Order within a
 * step: sweep, absorbing layer, point source, injection, record. */
typedef struct {
    int32_t z, y;
    const float *data;
    int32_t steps;
    int32_t reverse;
    float   scale;
} stencil_inject_cfg;

STENCIL_API int stencil_inject_start(stencil_plan_t p, const stencil_inject_cfg *c);
STENCIL_API int stencil_inject_stop(stencil_plan_t p);

/* Zero-lag cross-correlation imaging condition: image[p] += scale *
 * snapshot[p] * u^n[p] for every grid point, u^n the plan's current level.
 * snapshot and image: device memory, dense nx*ny*nz FP32.  Enqueued on the
 * plan's stream (returns at once).  16 B per point of HBM traffic. */
STENCIL_API int stencil_image_accumulate(stencil_plan_t p, const float *snapshot, float *image, float scale);

/* ---- failure-path testing ---------------------------------------------
 * Every shared-memory wait of the tiled sweep is bounded; a wait that runs
 * out sets the plan's error word, its thread block leaves after the copies
 * it issued have landed (also bounded), and the next synchronising call
 * returns STENCIL_ETIMEOUT and clears the word, so the plan stays usable.
 * This hook exercises that path without any GPU fault: with enable = 1 the
 * first copy of every block is expected to bring 16 more bytes than it
 * does, so that block's first wait runs out after wait_ns nanoseconds (0 =
 * the default 2 s).  enable = 0 restores normal sweeps (wait_ns stays the
 * wait limit).  Tiled and two-step kernels only (STENCIL_EUNSUPPORTED
 * otherwise).  The paper has no counterpart; for tests of the error path. */
STENCIL_API int stencil_debug_wait_fault(stencil_plan_t p, int32_t enable, uint32_t wait_ns);

/* ---- checkpoint / restore ---------------------------------------------
 * The time loop's state (Sec. 2, Algorithm 1): the two levels u^n and
 * u^{n-1} (16-bit storage: u^n and d^n = u^n - u^{n-1}) in the plan's
 * storage encoding, the step n (the source reads w(n dt)) and, for 16-bit
 * storage, the per-plane scales and maxima of u^n and d^n.  A plan restored
 * from a checkpoint continues bit for bit as the plan that wrote it would
 * have.  Format: a 128-byte header (magic "STNCKPT1", version 2, dims,
 * radius, storage, element size, step, dx, dt, source position / frequency /
 * delay / scale, payload bytes), then u^n and u^{n-1} (or d^n) dense (x
 * fastest), then for 16-bit storage the scales of u^n and d^n (nz floats
 * each) and their maxima (nz uint32 each).  The velocity
 * model is not included: restore into a plan made from the same descriptor
 * (dims, radius, storage, dx, dt and source are checked, STENCIL_EINVAL on a
 * mismatch; a different velocity model at the source point is caught, one
 * elsewhere is not).  Tile and graph settings may differ. */

/* Bytes stencil_checkpoint writes for this plan. */
STENCIL_API int stencil_checkpoint_size(stencil_plan_t p, uint64_t *bytes);
/* Write the state after everything enqueued so far into dst (bytes >=
 * stencil_checkpoint_size, else STENCIL_EINVAL; on_device: dst is device
 * memory).  Waits for the plan's stream; synchronous. */
STENCIL_API int stencil_checkpoint(stencil_plan_t p, void *dst, uint64_t bytes, int32_t on_device);
/* Replace the plan's state by the checkpoint in src (on_device: device
 * memory); steps_done becomes the checkpoint's step.  Synchronous: src may
 * be freed on return. */
STENCIL_API int stencil_restore(stencil_plan_t p, const void *src, uint64_t bytes, int32_t on_device);

/* ---- batches: many shots, one launch per time step --------------------- */

/* Shots are the paper's unit of data parallelism (one grid per process,
 * Sec. 3.1, 3.5); a batch runs many shots of different grid sizes together:
 * every time step is one launch over all the shots' tiles, and steps are
 * replayed from a captured CUDA graph of graph_steps steps (0 = no graph).
 * All descriptors must share radius and storage; descs[0] gives the stream
 * (NULL = the batch creates one) and the tile shape (tx, ty; the z-chunk is
 * chosen for the whole batch).  Each shot keeps its own wavefields, kappa,
 * source and step counter, and computes exactly what stencil_run computes
 * for it alone. */
typedef struct stencil_batch_s *stencil_batch_t;

STENCIL_API int stencil_batch_create(const stencil_desc *descs, int32_t n, int32_t graph_steps,
                                     stencil_batch_t *out);
/* Enqueue nsteps time steps of every shot; returns without waiting. */
STENCIL_API int stencil_batch_run(stencil_batch_t b, int32_t nsteps);
/* Wait for the batch's stream; report device-side errors. */
STENCIL_API int stencil_batch_sync(stencil_batch_t b);
STENCIL_API int stencil_batch_size(stencil_batch_t b, int32_t *n);
/* The plan of shot i, for stencil_get_field / set_fields / energy / rel_l2 /
 * get_stats (the batch owns it: never pass it to stencil_destroy). */
STENCIL_API int stencil_batch_plan(stencil_batch_t b, int32_t shot, stencil_plan_t *plan);
/* The z-chunk the batch runs with. */
STENCIL_API int stencil_batch_zchunk(stencil_batch_t b, int32_t *zchunk);
STENCIL_API int stencil_batch_destroy(stencil_batch_t b);

/* ---- shot server: continuous batching ----------------------------------- */

/* A request loop for seismic shots arriving at any time.  One engine thread
 * admits queued shots in arrival order whenever a slot is free and the
 * shot's projected device bytes fit under the memory budget and keeps every
 * admitted shot's wavefields resident.  Resident shots are split by size
 * into `lanes`: lane k takes shots of [2^(19+2k), 2^(21+2k)) points per
 * step (lane 0 everything below 2^21, the last lane everything above).  Each
 * lane advances its shots together, chunk_steps time steps per chunk, one
 * launch per step over all their tiles (the batch engine), on a stream of
 * its own whose priority falls with the shot size; a lane starts its next
 * chunk as soon as its last one ends, so small shots are not held to the
 * step rate of large ones.  A shot that reaches its step count retires: u^N
 * is copied to its host buffer and its memory is freed.  Each shot's result
 * is exactly what stencil_run computes for it alone.  All entry points are
 * thread-safe. */
typedef struct shot_server_s *shot_server_t;

typedef struct {
    double  hbm_budget_frac;    /* share of the device memory free at shot_server_create that the server
                                   may hold (default 0.8) */
    int64_t hbm_budget_bytes;   /* > 0: a byte budget instead of the fraction */
    int32_t max_slots;          /* resident shots at most (default 64) */
    int32_t chunk_steps;        /* time steps per lane chunk (default 20) */
    int32_t radius;             /* every shot's radius (default 5) */
    int32_t storage;            /* every shot's storage (default FP32) */
    void   *cuda_stream;        /* NULL = the server creates its lanes' streams; else one lane on it */
    stencil_tile tile;          /* tile shape (AUTO = 64 x 16) */
    int32_t lanes;              /* size classes stepped independently, 1 .. 6 (default 3) */
    int32_t pad;
} shot_server_cfg;

typedef enum { SHOT_QUEUED = 0, SHOT_RUNNING = 1, SHOT_DONE = 2, SHOT_FAILED = 3 } shot_state;

typedef struct {
    double  t_submit, t_admit, t_done;  /* seconds since the server was created; < 0 = not yet */
    int64_t steps_done;
    int32_t status;                     /* STENCIL_OK, or why the shot failed */
    int32_t pad;
} shot_timing;

typedef struct {
    int64_t submitted, admitted, done, failed, queued, running;
    int64_t bytes_in_use, budget_bytes;
    int64_t iterations;                 /* lane chunks run (all lanes) */
    int64_t point_updates;              /* nx*ny*nz*steps summed over finished shots */
    double  busy_s;                     /* wall time with at least one lane's chunk on the GPU */
    double  admit_s;                    /* engine time spent admitting shots (plan set-up) */
    double  build_s;                    /* engine time spent re-describing the resident set */
    double  retire_s;                   /* retire-thread time (read-back and free) */
} shot_server_stats;

STENCIL_API void shot_server_cfg_init(shot_server_cfg *cfg);
STENCIL_API int shot_server_create(const shot_server_cfg *cfg, shot_server_t *out);
/* Queue a shot of nsteps time steps; u^N will be written to out_host (dense
 * nx*ny*nz floats, or NULL), which must stay valid until the shot is DONE or
 * FAILED.  A page-locked out_host (cudaHostAlloc, cudaHostRegister) is
 * written by one device-to-host copy, any other through the server's pinned
 * bounce buffers.  A pageable host velocity is copied at once; a page-locked
 * host velocity or a device velocity is read in place at admission and must
 * stay valid until the shot is RUNNING (or DONE / FAILED).  STENCIL_EBUDGET if the shot alone
 * exceeds the budget (it is recorded as FAILED). */
STENCIL_API int shot_submit(shot_server_t s, const stencil_desc *d, int32_t nsteps, float *out_host,
                            uint64_t *ticket);
/* A served reverse-time migration: the application the paper's kernel is
 * the "3D model" step of (Sec. 2, Algorithm 1), with the readings of the
 * single-plan migration (stencil_record_*, stencil_inject_*,
 * stencil_image_accumulate).  The shot runs nsteps forward steps with its
 * point source (and absorbing layer, if any), recording u on the receiver
 * plane (or row) after every step and keeping u at the times t = k, 2k, ...,
 * nsteps in device memory; then nsteps backward steps on the same model
 * without the point source, the recorded traces injected on the receiver
 * plane in reverse time order, adding image_scale * S(t) * r (the zero-lag
 * cross-correlation of the snapshot of time t with the backward field that
 * belongs to time t) at every snapshot time.  Both phases run in the shot's
 * lane beside the other resident shots (the per-step record, injection,
 * snapshot and imaging work in one small grouped kernel after each grouped
 * sweep).  The image equals the single-plan migration's with the server's
 * tile, bit for bit. */
typedef struct {
    int32_t receiver_z;     /* receiver plane, 0 <= z < nz */
    int32_t receiver_y;     /* -1: every row of the plane; else that row */
    int32_t snap_every;     /* k >= 1; nsteps must be a multiple of k */
    float   image_scale;    /* default 1 */
} shot_rtm_cfg;

STENCIL_API void shot_rtm_cfg_init(shot_rtm_cfg *c);
/* Queue a migration of nsteps forward + nsteps backward steps.  image_host:
 * dense nx*ny*nz floats (required); traces_host: nsteps * rows * nx floats
 * (rows = ny, or 1 for one receiver row) or NULL; both must stay valid until
 * the shot is DONE or FAILED.  FP32 servers only (STENCIL_EUNSUPPORTED).  The
 * shot's device bytes include nsteps / k snapshots, the traces and the image;
 * STENCIL_EBUDGET if they alone exceed the budget.  shot_poll counts both
 * phases' steps (2 nsteps in all). */
STENCIL_API int shot_submit_rtm(shot_server_t s, const stencil_desc *d, int32_t nsteps, const shot_rtm_cfg *cfg,
                                float *image_host, float *traces_host, uint64_t *ticket);
/* State (shot_state) and timing of a shot; does not block. */
STENCIL_API int shot_poll(shot_server_t s, uint64_t ticket, int32_t *state, shot_timing *t);
/* Block until the shot is DONE or FAILED, or timeout_s passes (STENCIL_ENOTREADY). */
STENCIL_API int shot_wait(shot_server_t s, uint64_t ticket, double timeout_s, int32_t *state);
STENCIL_API int shot_server_get_stats(shot_server_t s, shot_server_stats *out);
/* Finish the resident shots, cancel the queued ones (FAILED,
 * STENCIL_ECANCELLED), stop the engine and free everything. */
STENCIL_API int shot_server_destroy(shot_server_t s);

/* ---- FP64 validation reductions (on the device, deterministic) -------- */

/* Discrete energy between the two current levels,
 *   E = sum_p (u^n - u^{n-1})^2 / kappa - u^n * Lambda(u^{n-1}),
 * evaluated in FP64; conserved by the scheme without a source. */
STENCIL_API int stencil_energy(stencil_plan_t p, double *out);

/* ||u^n - ref|| / ||ref|| in FP64; ref is a dense FP64 device array. */
STENCIL_API int stencil_rel_l2(stencil_plan_t p, const double *ref_device, double *out);

/* ---- blocksize-selection building blocks (host only, no device work) ---- */

/* Candidate values of one block axis of extent S split into P parts
 * (Sec. 3.7): b = <1, S/(P-1)+1, 2S/(P-1)+1, ..., S>, integer division, the
 * last value clamped to S, duplicates dropped.  Writes *n values to out
 * (capacity cap; STENCIL_EINVAL if too small, *n still set). */
STENCIL_API int stencil_candidates_1d(int32_t S, int32_t P, int32_t *out, int32_t cap, int32_t *n);

/* Three-stage contention-aware selection (Sec. 3.3): times[(g*C + c)*K + k]
 * is the time of group g's k-th candidate measured on stream c (all streams
 * of a group run the same candidates in the same order; +inf marks a
 * missing entry).  Stage 1: each stream's fastest candidate; stage 2: one
 * stream per group by target 0 = min (MMMB, Eq. 1), 1 = max (MWMB, Eq. 2),
 * 2 = closest to the group mean (MAMB, Eq. 3); stage 3: the group whose
 * stage-2 time is smallest.  Ties go to the lowest index. */
STENCIL_API int stencil_select(const double *times, int32_t groups, int32_t streams, int32_t cands,
                               int32_t target, int32_t *group, int32_t *stream, int32_t *cand,
                               double *time);

/* Original Block (Sec. 3.3): times[c*K + k] is stream c's k-th own
 * candidate; the global minimum wins. */
STENCIL_API int stencil_select_ob(const double *times, int32_t streams, int32_t cands, int32_t *stream,
                                  int32_t *cand, double *time);

/* ---- FP64 sums of squares without device allocation -------------------- */

/* The paper has no counterpart to this entry point; it is a library service
 * for callers that cannot call cudaMalloc: for example a process whose
 * device memory is all held by a caching allocator (PyTorch's keeps freed
 * memory for itself), or a latency-critical loop that must not stall on
 * cudaMalloc / cudaFree (cudaFree synchronises the device).
 *
 * Computes out[0] = sum (a - b)^2 and out[1] = sum b^2 over the nx*ny*nz
 * points in FP64 (||a - b|| / ||b|| = sqrt(out[0] / out[1])):
 *   a       FP32 device array, ny*nz rows of nx values, row pitch a_pitch
 *           elements (a_pitch >= nx; a dense array has a_pitch = nx);
 *   b       dense FP64 device array of nx*ny*nz values;
 *   out     2 doubles of device memory, written by the call;
 *   stream  cudaStream_t to enqueue on (NULL = the legacy default stream);
 *           the call returns without waiting.
 * Allocates nothing: the per-block partial sums live in a 256 KiB array in
 * the library's static device memory, which every GPU that loads the
 * library holds until the process exits.  Limit: nx*ny*nz <= 2^28
 * (268435456) elements, else STENCIL_EINVAL before any device work.  All
 * calls share that array and it keeps the last call's contents (each call
 * overwrites the slots it reads, so nothing needs clearing); calls that
 * overlap on the GPU, e.g. on two streams, race on it.  The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture. */
STENCIL_API int stencil_sqdiff_noalloc(const float *a, int64_t a_pitch, const double *b, int32_t nx,
                                       int32_t ny, int32_t nz, double *out, void *stream);

/* ---- helpers ---------------------------------------------------------- */

/* Whether the tiled kernel is built for (radius, storage, tx, ty); if so
 * *smem_bytes and *threads receive its dynamic shared memory and block size.
 * Returns 1 (available) or 0. */
STENCIL_API int stencil_tile_info(int32_t radius, int32_t storage, int32_t tx, int32_t ty, int32_t *smem_bytes,
                                  int32_t *threads);

/* Stability bound on v*dt/dx of the 3D leapfrog scheme of radius R:
 * 2 / sqrt(3 W), W = |c_0| + 2 sum |c_r|.  Returns < 0 for an unsupported R. */
STENCIL_API double stencil_cfl_limit(int32_t radius);

/* Message for the calling thread's last failed call ("" if none). */
STENCIL_API const char *stencil_last_error(void);

/* Library version string. */
STENCIL_API const char *stencil_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STENCIL_H */
