/*
 * A plain C11 client of libstencil: proves the boundary is a C ABI (no C++,
 * no CUDA headers, no torch) and that every call behaves from C.
 *
 *   abi_client host            host-side calls only (no GPU needed)
 *   abi_client layout          size and field offsets of every struct of the header
 *   abi_client run OUT.bin     one 40 x 36 x 30 shot, R = 5, 12 steps, written to OUT.bin
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "stencil.h"

#define NX 40
#define NY 36
#define NZ 30

static int fails = 0;

static void expect(int cond, const char *what)
{
    if (!cond) {
        fprintf(stderr, "FAIL: %s (%s)\n", what, stencil_last_error());
        ++fails;
    }
}

/* 4 layers along z, 1800 .. 3300 m/s */
static void layered(float *v)
{
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) v[((size_t)k * NY + j) * NX + i] = 1800.0f + 500.0f * (float)((4 * k) / NZ);
}

static void host_checks(void)
{
    expect(strstr(stencil_version(), "sm_103a") != NULL, "version");
    expect(stencil_cfl_limit(5) > 0.0 && stencil_cfl_limit(4) > stencil_cfl_limit(5), "cfl limits");
    expect(stencil_cfl_limit(3) < 0.0, "cfl limit of an unsupported radius");

    int32_t cand[8], n = 0;
    expect(stencil_candidates_1d(200, 5, cand, 8, &n) == STENCIL_OK && n == 5, "candidates");
    expect(cand[0] == 1 && cand[1] == 51 && cand[4] == 200, "candidate values (Sec. 3.7 example)");

    /* MWMB (Sec. 3.3) on one group of two streams and two candidates:
     * stream 0's best is candidate 1 (1.0), stream 1's is candidate 0 (2.0);
     * the slowest of the bests is stream 1's */
    const double times[4] = {3.0, 1.0, 2.0, 5.0};   /* [group][stream][cand] */
    int32_t g = -1, c = -1, k = -1;
    double t = 0;
    expect(stencil_select(times, 1, 2, 2, 1, &g, &c, &k, &t) == STENCIL_OK, "select call");
    expect(g == 0 && c == 1 && k == 0 && t == 2.0, "MWMB pick");

    stencil_desc d;
    stencil_desc_init(&d);
    expect(d.radius == 5 && d.storage == STENCIL_FP32 && d.user_buffers[0] == NULL, "desc defaults");
    stencil_plan_t p = NULL;
    expect(stencil_plan(NULL, &p) == STENCIL_EINVAL, "null descriptor");
    d.nx = NX; d.ny = NY; d.nz = NZ; d.dt = 1e-3;
    expect(stencil_plan(&d, &p) == STENCIL_EINVAL, "missing velocity");
    static float v[NX * NY * NZ];
    layered(v);
    d.velocity = v;
    d.radius = 3;
    expect(stencil_plan(&d, &p) == STENCIL_EINVAL, "radius 3");
    d.radius = 5;
    d.src_x = NX;
    expect(stencil_plan(&d, &p) == STENCIL_EINVAL, "source outside the grid");
    expect(stencil_step(NULL, 1) == STENCIL_EINVAL, "null plan");
    stencil_record_cfg rc;
    stencil_record_cfg_init(&rc);
    expect(rc.receiver_z == -1 && rc.capacity == 0, "record defaults");
    shot_server_cfg sc;
    shot_server_cfg_init(&sc);
    expect(sc.max_slots > 0 && sc.hbm_budget_frac > 0.0, "server defaults");
}

static int run(const char *path)
{
    static float v[NX * NY * NZ], out[NX * NY * NZ];
    layered(v);
    stencil_desc d;
    stencil_desc_init(&d);
    d.nx = NX; d.ny = NY; d.nz = NZ;
    d.radius = 5;
    d.dx = 10.0;
    d.dt = 0.5 * stencil_cfl_limit(5) * 10.0 / 3300.0;
    d.velocity = v;
    d.src_x = NX / 2; d.src_y = NY / 2; d.src_z = NZ / 2;
    d.tile.kernel = STENCIL_KERNEL_TILED;
    d.tile.tx = 64; d.tile.ty = 16; d.tile.zchunk = -1;
    d.graph_steps = 4;
    stencil_plan_t p = NULL;
    int rc = stencil_plan(&d, &p);
    if (rc) {
        fprintf(stderr, "stencil_plan: %d %s\n", rc, stencil_last_error());
        return 1;
    }
    rc = stencil_run(p, 12, out, 0);
    stencil_stats s;
    if (!rc) rc = stencil_get_stats(p, &s);
    if (!rc && s.steps_done != 12) rc = -100;
    stencil_destroy(p);
    if (rc) {
        fprintf(stderr, "run: %d %s\n", rc, stencil_last_error());
        return 1;
    }
    FILE *f = fopen(path, "wb");
    if (!f || fwrite(out, sizeof out, 1, f) != 1) return 1;
    fclose(f);
    printf("dt %.17g\n", d.dt);
    return 0;
}

/* as the C compiler lays the header's structs out, for the Python
 * binding's ctypes mirrors to be compared against */
#define SZ(T) printf(#T " %zu\n", sizeof(T))
#define OF(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
static void layout(void)
{
    SZ(stencil_tile);
    OF(stencil_tile, kernel);
    OF(stencil_tile, tx);
    OF(stencil_tile, ty);
    OF(stencil_tile, zchunk);
    SZ(stencil_tune_params);
    OF(stencil_tune_params, parts);
    OF(stencil_tune_params, iterations);
    OF(stencil_tune_params, streams);
    OF(stencil_tune_params, groups);
    SZ(stencil_desc);
    OF(stencil_desc, nx);
    OF(stencil_desc, ny);
    OF(stencil_desc, nz);
    OF(stencil_desc, radius);
    OF(stencil_desc, dx);
    OF(stencil_desc, dt);
    OF(stencil_desc, velocity);
    OF(stencil_desc, velocity_on_device);
    OF(stencil_desc, src_x);
    OF(stencil_desc, src_y);
    OF(stencil_desc, src_z);
    OF(stencil_desc, src_freq_hz);
    OF(stencil_desc, src_t0);
    OF(stencil_desc, src_amp);
    OF(stencil_desc, storage);
    OF(stencil_desc, tune_mode);
    OF(stencil_desc, tile);
    OF(stencil_desc, tune);
    OF(stencil_desc, cuda_stream);
    OF(stencil_desc, graph_steps);
    OF(stencil_desc, user_buffers);
    OF(stencil_desc, absorb_width);
    OF(stencil_desc, absorb_eta);
    SZ(stencil_stats);
    OF(stencil_stats, steps_done);
    OF(stencil_stats, tile);
    OF(stencil_stats, vmax);
    OF(stencil_stats, cfl);
    OF(stencil_stats, cfl_limit);
    OF(stencil_stats, pitch);
    OF(stencil_stats, field_bytes);
    OF(stencil_stats, device_bytes);
    OF(stencil_stats, min_time_ms);
    OF(stencil_stats, actual_time_ms);
    OF(stencil_stats, full_time_ms);
    OF(stencil_stats, quality);
    OF(stencil_stats, selection_ms);
    OF(stencil_stats, n_candidates);
    OF(stencil_stats, tune_mode);
    OF(stencil_stats, current_buffer);
    OF(stencil_stats, user_buffers);
    SZ(stencil_record_cfg);
    OF(stencil_record_cfg, receiver_z);
    OF(stencil_record_cfg, receiver_y);
    OF(stencil_record_cfg, energy);
    OF(stencil_record_cfg, capacity);
    SZ(stencil_inject_cfg);
    OF(stencil_inject_cfg, z);
    OF(stencil_inject_cfg, y);
    OF(stencil_inject_cfg, data);
    OF(stencil_inject_cfg, steps);
    OF(stencil_inject_cfg, reverse);
    OF(stencil_inject_cfg, scale);
    SZ(shot_server_cfg);
    OF(shot_server_cfg, hbm_budget_frac);
    OF(shot_server_cfg, hbm_budget_bytes);
    OF(shot_server_cfg, max_slots);
    OF(shot_server_cfg, chunk_steps);
    OF(shot_server_cfg, radius);
    OF(shot_server_cfg, storage);
    OF(shot_server_cfg, cuda_stream);
    OF(shot_server_cfg, tile);
    OF(shot_server_cfg, lanes);
    OF(shot_server_cfg, pad);
    SZ(shot_rtm_cfg);
    OF(shot_rtm_cfg, receiver_z);
    OF(shot_rtm_cfg, receiver_y);
    OF(shot_rtm_cfg, snap_every);
    OF(shot_rtm_cfg, image_scale);
    SZ(shot_timing);
    OF(shot_timing, t_submit);
    OF(shot_timing, t_admit);
    OF(shot_timing, t_done);
    OF(shot_timing, steps_done);
    OF(shot_timing, status);
    OF(shot_timing, pad);
    SZ(shot_server_stats);
    OF(shot_server_stats, submitted);
    OF(shot_server_stats, admitted);
    OF(shot_server_stats, done);
    OF(shot_server_stats, failed);
    OF(shot_server_stats, queued);
    OF(shot_server_stats, running);
    OF(shot_server_stats, bytes_in_use);
    OF(shot_server_stats, budget_bytes);
    OF(shot_server_stats, iterations);
    OF(shot_server_stats, point_updates);
    OF(shot_server_stats, busy_s);
    OF(shot_server_stats, admit_s);
    OF(shot_server_stats, build_s);
    OF(shot_server_stats, retire_s);
}

int main(int argc, char **argv)
{
    if (argc >= 2 && strcmp(argv[1], "layout") == 0) {
        layout();
        return 0;
    }
    if (argc >= 2 && strcmp(argv[1], "host") == 0) {
        host_checks();
        if (fails) return 1;
        printf("host ok\n");
        return 0;
    }
    if (argc >= 3 && strcmp(argv[1], "run") == 0) return run(argv[2]);
    fprintf(stderr, "usage: abi_client host | layout | run OUT.bin\n");
    return 2;
}
