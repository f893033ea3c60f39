#!/usr/bin/env python
"""Benchmark of the blocked 3D acoustic stencil sweep on GB300.

Workload: one seismic shot on a 512^3 FP32 grid, layered velocity model of 8
horizontal layers with velocities drawn uniform in [1500, 4500) m/s
(seed 1310), dx = 10 m, dt = 0.5 x the CFL bound for the largest velocity,
15 Hz Ricker source at the grid centre, ghost-zero boundaries, 10th-order
space / 2nd-order time stencil (R = 5; --radius 4 for 8th order), 200 time
steps.  One benchmark "step" = one whole shot (reset the wavefields, 200
sweeps); the velocity model, kappa and the tile are set up once, outside the
timed region.  Every array (3 x 512 MiB) is larger than L2, so no L2 flush is
needed between iterations.

Metric: grid-point updates per second (nx*ny*nz*timesteps / time), reported
in GPt-updates/s, with the dominant kernel's achieved HBM bandwidth at the
algorithmic 16 B per point update (read u, u_prev, kappa; write u_next in
place) against the measured HBM copy bandwidth.

Prints exactly one JSON line (rank 0).  --impl reference times the FP64 CPU
oracle on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPt-updates/s"
BYTES_PER_POINT = 16            # algorithmic minimum, FP32: u, u_prev, kappa read; u_next written
# the storage's own minimum: 16-bit storage reads u^n, d^n (2 B each) and
# kappa (4 B) and writes u^{n+1}, d^{n+1} (2 B each)
OWN_BYTES = {"fp32": 16, "fp16": 12, "bf16": 12}
STORAGE_ID = {"fp32": 0, "fp16": 1, "bf16": 2}
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5, help="timed shots")
    ap.add_argument("--warmup", type=int, default=3, help="untimed shots")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="cube side")
    ap.add_argument("--timesteps", type=int, default=200)
    ap.add_argument("--radius", type=int, default=5, choices=[4, 5])
    ap.add_argument("--graph", type=int, default=20, help="time steps per captured CUDA graph")
    ap.add_argument("--tile", type=str, default="",
                    help="tx,ty,zchunk of the tiled kernel (with --two-step only zchunk is used)")
    ap.add_argument("--naive", action="store_true", help="time the one-thread-per-point kernel")
    ap.add_argument("--two-step", action="store_true",
                    help="time the two-steps-per-sweep kernel (temporal blocking; 10 B per point update)")
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16"], default="fp32",
                    help="wavefield storage (fp16/bf16: per-plane scaled, FP32 arithmetic)")
    ap.add_argument("--record", choices=["none", "energy", "traces", "both"], default="none",
                    help="single: also record the per-step energy and/or a receiver plane at z = 10")
    ap.add_argument("--absorb", type=int, default=0,
                    help="single / batch: absorbing layer of this many points on every face (eta_max 0.2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-timesteps", type=int, default=10)
    ap.add_argument("--host-method", action="store_true",
                    help="single: also time the paper's method on the host cores (FP32 blocked sweep, "
                         "MWMB-selected block, P=3, nI=1) on the same grid")
    ap.add_argument("--workload", choices=["single", "batch", "serve", "rtm"], default="single",
                    help="single: one 512^3 shot; batch: 64 uneven shots in one grouped launch per step "
                         "vs a per-shot loop; serve: Poisson arrivals through the shot server")
    ap.add_argument("--shots", type=int, default=64, help="batch: number of shots")
    ap.add_argument("--window", type=float, default=10.0, help="serve: arrival window (s)")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--lanes", type=int, default=0, help="serve: size lanes of the shot server (0 = its default)")
    ap.add_argument("--served", type=int, default=0,
                    help="rtm: also run this many copies of the migration through the shot server together")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def code_digest(texts) -> str:
    """16 hex digits of SHA-256 over C/C++ sources with comments and
    whitespace runs removed: a change of code changes it, a note does not."""
    h = hashlib.sha256()
    for text in texts:
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def kernel_source_hash() -> str:
    """Digest of the dominant kernel's code (sweep_tiled.cuh, common.cuh), the
    key of the recorded traffic in profiles/traffic.txt."""
    texts = []
    for name in ("sweep_tiled.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1310_8232_gb300", "csrc", name), encoding="utf-8") as fh:
            texts.append(fh.read())
    return code_digest(texts)


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None, None
    want = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel_tag and parts[1] == want:
                return float(parts[2]), parts[3]
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(suffix=".csv", prefix="clocks_")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return None
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
            os.remove(self.path)
        except OSError:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(args, extra=None):
    cfg = {"workload": f"single shot {args.n}^3 FP32, 8-layer random velocity model (seed 1310), "
                       f"R={args.radius} ({2 * args.radius}th-order space / 2nd-order time), "
                       f"{args.timesteps} time steps, dx=10 m, dt=0.5 CFL, 15 Hz Ricker at centre",
           "nx": args.n, "ny": args.n, "nz": args.n, "radius": args.radius,
           "timesteps": args.timesteps, "parallelism": "replicas (one independent shot per GPU)",
           "l2": "no flush needed: every array (u, u_prev, kappa) is larger than L2"}
    if extra:
        cfg.update(extra)
    return cfg


def cpu_baseline(args, v, dt):
    """The FP64 oracle, as it stands, on this host's cores: the first
    --cpu-timesteps steps of the same shot."""
    import numpy as np

    import oracle
    from paper_1310_8232_gb300 import workloads
    steps = max(1, min(args.cpu_timesteps, args.timesteps))      # a sample of the shot's own steps
    t0 = time.perf_counter()
    oracle.run(v.astype(np.float64), workloads.DX, dt, args.radius, steps)
    el = time.perf_counter() - t0
    pts = float(args.n) ** 3 * steps
    return {"value": pts / el / 1e9, "unit": METRIC, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"first {steps} of {args.timesteps} time steps of the {args.n}^3 shot, "
                      f"FP64 unblocked oracle, {el:.1f} s"}


def host_method_baseline(args, v, dt):
    """The paper's method on this host's cores: MWMB (P = 3, nI = 1) picks the
    block of an FP32 blocked sweep across the cores, which then runs the
    first --cpu-timesteps steps of the same shot on the whole grid."""
    import numpy as np

    from oracle import host_method as hm
    from paper_1310_8232_gb300 import workloads
    n, R, steps = args.n, args.radius, max(1, min(args.cpu_timesteps, args.timesteps))
    kap = hm.kappa(v, workloads.DX, dt)
    t0 = time.perf_counter()
    sel = hm.select_mwmb(kap, R, P=3, nI=1)
    sel_s = time.perf_counter() - t0
    u = np.zeros((n, n, n), np.float32)
    up = np.zeros_like(u)
    src = (n // 2, n // 2, n // 2)
    scale = float(v[src[2], src[1], src[0]]) ** 2 * dt * dt
    el = hm.run(kap, R, steps, u, up, src=src, src_scale=scale, dt=dt, block=sel["block"])
    return {"value": float(n) ** 3 * steps / el / 1e9, "unit": METRIC, "cores": sel["cores"],
            "kind": "paper method on the host: FP32 blocked sweep, block chosen by MWMB across the cores",
            "block": list(sel["block"]), "candidates": sel["candidates"], "selection_s": sel_s,
            "min_time_s": sel["min_time"], "actual_time_s": sel["actual_time"], "quality": sel["quality"],
            "sample": f"first {steps} of {args.timesteps} time steps of the {n}^3 shot after the selection"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1310_8232_gb300 import workloads
    v = workloads.layered_velocity(args.n, args.n, args.n, seed=1310).astype(np.float64)
    dt = workloads.time_step(oracle.cfl_limit(args.radius), workloads.DX, float(v.max()))
    per = max(1, min(args.cpu_timesteps, args.timesteps))
    for _ in range(args.warmup):
        oracle.run(v, workloads.DX, dt, args.radius, per)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(v, workloads.DX, dt, args.radius, per)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    pts = float(args.n) ** 3 * per * args.steps
    val = pts / total / 1e9
    sample = (f"each step: first {per} of {args.timesteps} time steps of the {args.n}^3 shot "
              f"(FP64 unblocked oracle)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, {"sample_timesteps_per_step": per}),
        "cpu_baseline": {"value": val, "unit": METRIC, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batch(args, torch, st, workloads, ranks):
    """64 shots with uneven grids (each dim in {96, 128, ..., 320}, seed 4064),
    8-layer random models, 100 steps each: one grouped launch per step
    (graph-captured) against a loop of per-shot plans.  On N GPUs every rank
    takes a contiguous share of the 64 shots (fixed total: strong scaling)."""
    R, T = args.radius, args.timesteps if args.timesteps != 200 else 100
    all_dims = workloads.batch_dims(args.shots)
    if args.shots < ranks.env.world:
        raise SystemExit("batch: need at least one shot per rank")
    lo, hi = ranks.shard(args.shots)
    dims = all_dims[lo:hi]
    seeds = workloads.batch_layer_seeds(args.shots)[lo:hi]
    stream = torch.cuda.current_stream()
    descs, vels = [], []
    for (nx, ny, nz), sd in zip(dims, seeds):
        v = torch.from_numpy(workloads.layered_velocity(nx, ny, nz, seed=sd)).cuda()
        dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
        vels.append(v)
        descs.append(st.make_desc(v, dt, radius=R, dx=workloads.DX, graph_steps=20, stream=stream.cuda_stream,
                                  absorb=(args.absorb, 0.2 if args.absorb else 0.0)))
    pts = float(sum(nx * ny * nz for nx, ny, nz in all_dims)) * T
    batch = st.stencil_batch_create(descs, graph_steps=20)
    plans = [st.stencil_plan(d) for d in descs]

    def reset():
        for i in range(len(plans)):
            st.stencil_set_fields(st.stencil_batch_plan(batch, i), None, None, 0)
            st.stencil_set_fields(plans[i], None, None, 0)

    def run_grouped():
        st.stencil_batch_run(batch, T)

    def run_loop():
        for p in plans:
            st.stencil_step(p, T)

    times = {"grouped": [], "loop": []}
    for _ in range(args.warmup):
        reset()
        run_grouped()
        run_loop()
    torch.cuda.synchronize()
    with ClockSampler(ranks.env.local) as clk:
        for _ in range(args.steps):
            for name, fn in (("grouped", run_grouped), ("loop", run_loop)):
                reset()
                ranks.barrier()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                ranks.barrier()
                times[name].append(ranks.max(a.elapsed_time(b)))
    zc = st.stencil_batch_zchunk(batch)
    st.stencil_batch_sync(batch)
    st.stencil_batch_destroy(batch)
    for p in plans:
        st.stencil_destroy(p)
    g_ms = sum(times["grouped"]) / len(times["grouped"])
    l_ms = sum(times["loop"]) / len(times["loop"])
    if not ranks.is_root:
        return
    line = {
        "metric": METRIC, "value": pts / (g_ms / 1e3) / 1e9, "unit": METRIC, "n_gpus": ranks.env.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": g_ms, "higher_is_better": True,
        "scaling": "strong" if ranks.env.world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batch of {len(all_dims)} shots, dims uniform in {{96..320 step 32}} (seed 4064), "
                               f"8-layer random models, R={R}, {T} steps each; one grouped launch per step, "
                               f"20-step CUDA graphs", "shots": len(all_dims), "timesteps": T,
                   "parallelism": f"replicas: contiguous shot shares over {ranks.env.world} GPU(s)",
                   "point_updates": pts, "zchunk": zc, "absorb": args.absorb},
        "per_shot_loop": {"value": pts / (l_ms / 1e3) / 1e9, "ms_per_step": l_ms,
                          "what": "the same shots, one plan each, stencil_step(100) in a loop (20-step graphs)"},
        "speedup_vs_loop": l_ms / g_ms,
        "roofline": {"bound": "hbm", "achieved": BYTES_PER_POINT * pts / (g_ms / 1e3) / 1e9,
                     "unit": "GB/s", "bytes_per_point": BYTES_PER_POINT},
        "clocks": clk.summary(),
    }
    peaks = measured_peaks()
    if peaks and "hbm_gbs" in peaks:
        line["roofline"]["peak"] = float(peaks["hbm_gbs"])
        line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
    print(json.dumps(line), flush=True)


def run_serve(args, torch, st, workloads, ranks):
    """Open-loop Poisson arrivals (seed 5020, mean --rate per second) over
    --window seconds: cube side log-uniform on [64, 400], steps uniform on
    [50, 500], FP32, 8-layer random models, admitted under an 80 % HBM
    budget; reports throughput and p50 / p99 latency (done - submit).  On N
    GPUs the arrivals are dealt round-robin, one shot server per GPU."""
    import numpy as np
    R = args.radius
    all_arrivals = workloads.poisson_arrivals(args.rate, args.window)
    arrivals = all_arrivals[ranks.env.rank::ranks.env.world]
    cfg = st.shot_server_cfg_init()
    cfg.radius = R
    cfg.chunk_steps = 20
    if args.lanes:
        cfg.lanes = args.lanes
    lanes = cfg.lanes
    server = st.shot_server_create(cfg)
    # every request's velocity model and output buffer are made before the
    # window opens (device models stay valid until admission), so the
    # generator below only sleeps and submits
    reqs = []
    for a in arrivals:
        n = a["side"]
        vl_host = workloads.layer_velocities(8, seed=a["seed"])
        vl = torch.from_numpy(vl_host).cuda()
        z = torch.arange(n, device="cuda")
        v = vl[(8 * z) // n].view(n, 1, 1).expand(n, n, n).contiguous()
        dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(vl_host.max()))
        out = np.empty((n, n, n), dtype=np.float32)
        reqs.append((a, v, st.make_desc(v, dt, radius=R, dx=workloads.DX), out))
    ranks.barrier()
    jobs = []
    submit_s = 0.0
    t_start = time.perf_counter()
    with ClockSampler(ranks.env.local) as clk:
        for a, v, d, out in reqs:
            delay = a["t"] - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            ts = time.perf_counter()
            t = st.shot_submit(server, d, a["steps"], out)
            submit_s += time.perf_counter() - ts
            jobs.append((t, a["side"], a["steps"], v, out))
        for t, *_ in jobs:
            st.shot_wait(server, t, 600.0)
    stats = st.shot_server_get_stats(server)
    mine = []
    for t, n, steps, v, out in jobs:
        state, tm = st.shot_poll(server, t)
        if state != st.SHOT_DONE:
            continue
        mine.append((tm.t_submit, tm.t_admit, tm.t_done, float(n) ** 3 * steps, n))
    st.shot_server_destroy(server)
    pooled = ranks.gather({"shots": mine, "stats": (stats.done, stats.failed, stats.iterations, stats.busy_s,
                                                    stats.admit_s, stats.build_s, stats.retire_s),
                           "submit_s": submit_s})
    if not ranks.is_root:
        return
    # the ranks start together (barrier); the job spans the longest rank's
    # first-submit to last-done interval
    lat, queue_s, service, pts, span = [], [], [], 0.0, 0.0
    by_size = {"side<128": [], "128<=side<203": [], "side>=203": []}
    for part in pooled:
        for ts, ta, td, p, n in part["shots"]:
            by_size["side<128" if n ** 3 < 2 ** 21 else "128<=side<203" if n ** 3 < 2 ** 23 else "side>=203"].append(td - ts)
            lat.append(td - ts)
            queue_s.append(ta - ts)
            service.append(td - ta)
            pts += p
        if part["shots"]:
            span = max(span, max(s[2] for s in part["shots"]) - min(s[0] for s in part["shots"]))
    span = span or None
    submit_s = sum(part["submit_s"] for part in pooled)
    agg = [sum(part["stats"][i] for part in pooled) for i in range(7)]
    lat_s = sorted(lat)

    def pct(xs, q):
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None

    line = {
        "metric": "shot latency p50/p99 (s) and throughput", "value": pts / span / 1e9 if span else None,
        "unit": METRIC, "n_gpus": ranks.env.world, "steps": len(lat), "warmup": 0,
        "ms_per_step": 1e3 * statistics.mean(lat) if lat else None, "higher_is_better": True,
        "scaling": "strong" if ranks.env.world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"Poisson arrivals, mean {args.rate}/s over {args.window} s (seed 5020), "
                               f"cube side log-uniform 64-400, steps uniform 50-500, R={R}, "
                               "8-layer random models, 80% HBM budget, 20 steps per lane chunk, "
                               f"{lanes} size lane(s)",
                   "shots": len(all_arrivals),
                   "parallelism": f"replicas: arrivals dealt round-robin to {ranks.env.world} shot server(s)"},
        "latency_s": {"p50": pct(lat_s, 0.50), "p99": pct(lat_s, 0.99), "mean": statistics.mean(lat) if lat else None},
        "latency_by_size_s": {k: {"shots": len(v), "p50": pct(sorted(v), 0.50), "p99": pct(sorted(v), 0.99)}
                              for k, v in by_size.items()},
        "queue_s": {"mean": statistics.mean(queue_s) if queue_s else None,
                    "p99": pct(sorted(queue_s), 0.99)},
        "service_s": {"mean": statistics.mean(service) if service else None},
        "offered_gpts_per_s": sum(float(a["side"]) ** 3 * a["steps"] for a in all_arrivals) / args.window / 1e9,
        "server": {"done": agg[0], "failed": agg[1], "iterations": agg[2], "busy_s": agg[3],
                   "admit_s": agg[4], "build_s": agg[5], "retire_s": agg[6], "submit_s": submit_s},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_rtm(args, torch, st, workloads, ranks):
    """One-shot reverse-time migration: the 8-layer model (seed 1310) on an
    n^3 grid (--n, default 256 here), --timesteps forward steps (default 600
    here) with a 20-point absorbing layer, receivers on the plane z = 10,
    snapshots every 10 steps kept in HBM, then as many backward steps with
    the reversed traces injected and the imaging condition at every
    snapshot.  Value = sweep point-updates (2 T n^3) per second of the whole
    migration (both sweeps, recording, snapshot copies, injection, imaging)."""
    from paper_1310_8232_gb300 import rtm
    n = args.n if args.n != 512 else 256
    T = args.timesteps if args.timesteps != 200 else 600
    R, k = args.radius, 10
    v = torch.from_numpy(workloads.layered_velocity(n, n, n, seed=1310)).cuda()
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    src = (n // 2, n // 2, 12)

    def once():
        return rtm.migrate(torch, v, dt, T, src, 10, k, radius=R, dx=workloads.DX, absorb=(20, 0.2),
                           graph_steps=10)

    served = None
    if args.served:
        # the same migrations through a shot server (shot_submit_rtm), all
        # submitted at once, so they run together in one lane
        import numpy as np
        hv = v.cpu().numpy()
        cfg = st.shot_server_cfg_init()
        cfg.radius = R
        server = st.shot_server_create(cfg)
        imgs = [np.empty((n, n, n), np.float32) for _ in range(args.served)]

        def once_served():
            ts = [st.shot_submit_rtm(server, st.make_desc(v, dt, radius=R, dx=workloads.DX, src=src,
                                                          absorb=(20, 0.2)), T, 10, k, img) for img in imgs]
            for t in ts:
                if st.shot_wait(server, t, 600.0) != st.SHOT_DONE:
                    raise SystemExit("served migration failed")
        once_served()
        t0 = time.perf_counter()
        once_served()
        served_s = time.perf_counter() - t0
        st.shot_server_destroy(server)
        served = {"migrations": args.served, "value": args.served * 2.0 * T * float(n) ** 3 / served_s / 1e9,
                  "unit": METRIC, "seconds": served_s,
                  "api": "shot_submit_rtm: forward and backward phases in the server's lane, per-step "
                         "record / snapshot / injection / imaging in a grouped kernel, image copied to host"}
        del hv

    for _ in range(max(1, args.warmup)):
        once()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(ranks.env.local) as clk:
        for _ in range(args.steps):
            ranks.barrier()
            t0 = time.perf_counter()
            image, _ = once()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    ms = 1e3 * ranks.max(sum(times) / len(times))
    pts = 2.0 * T * float(n) ** 3
    if not ranks.is_root:
        return
    print(json.dumps({
        "metric": METRIC, "value": ranks.env.world * pts / (ms / 1e3) / 1e9, "unit": METRIC,
        "n_gpus": ranks.env.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"one-shot RTM, {n}^3 8-layer model (seed 1310), R={R}, {T} forward + {T} backward "
                               "steps, 20-point absorbing layer, receiver plane z=10, snapshots every 10 steps "
                               "in HBM, zero-lag cross-correlation image", "n": n, "timesteps": T,
                   "snapshots": T // k, "parallelism": "replicas (one shot per GPU)"},
        "timing": "host wall clock around the whole migration with device synchronisation",
        "clocks": clk.summary(),
        **({"served": served} if served else {}),
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "single":
        import torch

        from paper_1310_8232_gb300.replicas import Ranks, rank_env
        env = rank_env()
        torch.cuda.set_device(env.local)
        ranks = Ranks(env)
        torch.cuda.set_stream(torch.cuda.Stream())
        import __graft_entry__
        __graft_entry__.build_library()
        from paper_1310_8232_gb300 import binding as st
        from paper_1310_8232_gb300 import workloads
        fn = {"batch": run_batch, "serve": run_serve, "rtm": run_rtm}[args.workload]
        fn(args, torch, st, workloads, ranks)
        ranks.close()
        return
    import numpy as np
    import torch

    from paper_1310_8232_gb300.replicas import Ranks, rank_env

    env = rank_env()
    world, rank, local = env.world, env.rank, env.local
    torch.cuda.set_device(local)
    ranks = Ranks(env)             # replicas: a barrier and a max over ranks, no data exchange
    barrier = ranks.barrier

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1310_8232_gb300 import binding as st
    from paper_1310_8232_gb300 import workloads

    n, R, T = args.n, args.radius, args.timesteps
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    # a dedicated stream, current for torch too: the plan's kernels, torch's
    # copies and the timing events are all ordered on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dv = torch.from_numpy(v).cuda()
    if args.naive:
        tile = (st.STENCIL_KERNEL_NAIVE, 0, 0, 0)
    elif args.two_step:
        zc = int(args.tile.split(",")[2]) if args.tile else -1
        tile = (st.STENCIL_KERNEL_TWO_STEP, 0, 0, zc)
    elif args.tile:
        tx, ty, zc = (int(x) for x in args.tile.split(","))
        tile = (st.STENCIL_KERNEL_TILED, tx, ty, zc)
    else:
        tile = None
    desc = st.make_desc(dv, dt, radius=R, dx=workloads.DX, tile=tile, graph_steps=args.graph,
                        stream=stream.cuda_stream, storage=STORAGE_ID[args.storage],
                        absorb=(args.absorb, 0.2 if args.absorb else 0.0))
    t_plan = time.perf_counter()
    plan = st.stencil_plan(desc)
    plan_ms = 1e3 * (time.perf_counter() - t_plan)
    if args.record != "none":
        st.stencil_record_start(plan, receiver_z=10 if args.record in ("traces", "both") else -1,
                                energy=args.record in ("energy", "both"), capacity=T)
    stats = st.stencil_get_stats(plan)
    t = stats.tile
    etype = {"fp32": "float", "fp16": "__half", "bf16": "__nv_bfloat16"}[args.storage]
    two = t.kernel == st.STENCIL_KERNEL_TWO_STEP
    kernel_tag = ("sweep_naive_kernel" if t.kernel == st.STENCIL_KERNEL_NAIVE
                  else f"sweep_two_step_kernel<{R},{t.tx},{t.ty}>" if two
                  else f"sweep_tiled_kernel<{R},{t.tx},{t.ty}>" if args.storage == "fp32"
                  else f"sweep_tiled_kernel<{R},{t.tx},{t.ty},{etype}>")
    rec_variant = args.record in ("energy", "both")
    if t.kernel == st.STENCIL_KERNEL_TILED and (rec_variant or args.absorb > 0):
        # the energy and absorbing instantiations are kernels of their own
        kernel_tag = f"sweep_tiled_kernel<{R},{t.tx},{t.ty},{etype},{int(rec_variant)},{int(args.absorb > 0)}>"
    # point updates per launch of the timed kernel, and its own algorithmic
    # bytes per update: the two-step kernel reads u^n, u^{n-1}, kappa and
    # writes u^{n+1}, u^{n+2} (20 B per two updates)
    upd_per_launch = 2 if two else 1
    own_bytes = 10 if two else OWN_BYTES[args.storage]

    def shot():
        st.stencil_set_fields(plan, None, None, 0)
        st.stencil_step(plan, T)

    for _ in range(args.warmup):
        shot()
    barrier()
    # our kernels per shot: one sweep per time step (two-step kernel: one per
    # two steps, and a one-step sweep for an odd remainder), plus one
    # step-counter kernel per captured graph and per eager chunk of <= 64 steps
    def sweeps(k):
        return (k // 2 + k % 2) if two else k
    if args.graph:
        rem = T % args.graph
        launches_per_shot = (T // args.graph) * (sweeps(args.graph) + 1) + sweeps(rem) + (rem + 63) // 64
        sweeps_per_shot = (T // args.graph) * sweeps(args.graph) + sweeps(rem)
    else:
        launches_per_shot = sweeps(T) + (T + 63) // 64
        sweeps_per_shot = sweeps(T)
    # and the work around the sweeps: each shot's reset (stencil_set_fields
    # with no arrays: one kernel for FP32; the 16-bit pack of both fields, two
    # kernels each, and the step counter), a receiver record kernel per step,
    # and, where the layer is not folded into the sweep (naive kernel), its
    # save and damping passes (three kernels each) and the source kernel
    launches_per_shot += 1 if args.storage == "fp32" else 5
    if args.record in ("traces", "both"):
        launches_per_shot += T
    if args.absorb > 0 and t.kernel == st.STENCIL_KERNEL_NAIVE:
        launches_per_shot += 7 * T
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for k in range(args.steps):
            st.stencil_set_fields(plan, None, None, 0)
            ev[k][0].record(stream)
            st.stencil_step(plan, T)
            ev[k][1].record(stream)
        end.record(stream)
        barrier()
    st.stencil_sync(plan)
    elapsed_ms = start.elapsed_time(end)
    sweep_ms = sum(a.elapsed_time(b) for a, b in ev)
    elapsed_ms = ranks.max(elapsed_ms)
    pts_per_shot = float(n) ** 3 * T
    value = world * pts_per_shot * args.steps / (elapsed_ms / 1e3) / 1e9
    kernel_ms = sweep_ms / (args.steps * sweeps_per_shot)
    # per launch: the timed kernel's own algorithmic bytes (16 B per update
    # for the one-step FP32 sweep, its storage's bytes otherwise)
    achieved = own_bytes * upd_per_launch * float(n) ** 3 / (kernel_ms / 1e3) / 1e9
    # the metric's denominator: updates at the plain FP32 sweep's 16 B each
    achieved16 = BYTES_PER_POINT * upd_per_launch * float(n) ** 3 / (kernel_ms / 1e3) / 1e9
    peaks = measured_peaks()
    if peaks and "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    else:
        peak, peak_src = FALLBACK_HBM_GBS, "fallback 6.8 TB/s"
    traffic, traffic_src = profiled_traffic(kernel_tag + f"@{n}")

    e2e = None
    if not args.no_e2e:
        # Through the public API with host buffers: H2D of the velocity model
        # (kappa recomputed on the device), one shot, D2H of the final field.
        hv = torch.from_numpy(v).pin_memory()
        hout = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
        for _ in range(1):
            st.stencil_set_velocity(plan, hv)
            st.stencil_set_fields(plan, None, None, 0)
            st.stencil_run(plan, T, hout)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st.stencil_set_velocity(plan, hv)
            st.stencil_set_fields(plan, None, None, 0)
            st.stencil_run(plan, T, hout)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s = ranks.max(e2e_s)
        e2e = {"value": world * pts_per_shot * args.steps / e2e_s / 1e9, "unit": METRIC,
               "h2d_bytes_per_step": int(hv.numel() * 4), "d2h_bytes_per_step": int(hout.numel() * 4),
               "api": "stencil_set_velocity(host pinned) + stencil_set_fields + stencil_run(out=host pinned)"}
        if args.record == "none":
            # The same shots through two plans on their own streams, each
            # driven by its own host thread, as a caller with many shots would
            # run them: one plan's copies overlap the other's sweeps.  Each
            # plan runs --steps shots (2 x --steps in all).
            import threading
            stream2 = torch.cuda.Stream()
            plan2 = st.stencil_plan(st.make_desc(dv, dt, radius=R, dx=workloads.DX, tile=tile,
                                                 graph_steps=args.graph, stream=stream2.cuda_stream,
                                                 storage=STORAGE_ID[args.storage],
                                                 absorb=(args.absorb, 0.2 if args.absorb else 0.0)))
            hout2 = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
            errors = []

            def shots(pl, k, out):
                try:
                    for _ in range(k):
                        st.stencil_set_velocity(pl, hv)
                        st.stencil_set_fields(pl, None, None, 0)
                        st.stencil_run(pl, T, out)
                except Exception as ex:          # reported after the join
                    errors.append(ex)

            shots(plan2, 1, hout2)
            barrier()
            t0 = time.perf_counter()
            workers = [threading.Thread(target=shots, args=(plan, args.steps, hout)),
                       threading.Thread(target=shots, args=(plan2, args.steps, hout2))]
            for w in workers:
                w.start()
            for w in workers:
                w.join()
            barrier()
            two_s = ranks.max(time.perf_counter() - t0)
            st.stencil_destroy(plan2)
            if errors:
                raise errors[0]
            e2e["two_plans"] = {
                "value": world * pts_per_shot * 2 * args.steps / two_s / 1e9, "unit": METRIC,
                "api": "two plans on their own streams, one host thread each, each shot as above "
                       "(the copies of one plan overlap the sweeps of the other)"}
    st.stencil_destroy(plan)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, v, dt)
    host = None
    if rank == 0 and world == 1 and args.host_method:
        host = host_method_baseline(args, v, dt)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "fp32" else f"f32 arithmetic, {args.storage} storage",
            "data": "synthetic",
            "config": workload_config(args, {"storage": args.storage, "record": args.record, "absorb": args.absorb,
                "tile": {"kernel": kernel_tag, "tx": t.tx, "ty": t.ty, "zchunk": t.zchunk},
                "graph_steps": args.graph, "plan_ms": plan_ms}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": kernel_tag,
                         "bytes_per_point": own_bytes, "updates_per_launch": upd_per_launch,
                         "launch_ms": kernel_ms,
                         "frac_at_16B_per_update": achieved16 / peak,
                         "peak_source": peak_src, "traffic_source": traffic_src,
                         "timing": "CUDA events around each shot's sweeps on the launching stream; "
                                   "per-launch time = sum / launches (includes the step-counter kernel)"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            **({"host_method": host} if host else {}),
            "gpu_launches": args.steps * launches_per_shot,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
