"""Tile selection report: the paper's blocksize-selection methodology
(Sec. 3.2-3.7) re-run on GPU tile parameters, against the library's own
tuner, an exhaustive search, the default tile, a poor tile and the naive
kernel.

For every row: the tile used, the selection cost, MinTime / ActualTime /
quality (Sec. 3.6) where a selection ran, and the throughput of a full shot
(--steps time steps) with that tile.  Prints one JSON line per row.

    python -m paper_1310_8232_gb300.tile_report [--n 512] [--radius 5] [--steps 200]

With --study nc it re-runs the paper's study of the number of candidates
(Sec. 3.7, Table 6): MWMB with P = 2, 3, 5, 10 parts per axis, reporting
nC, the selection cost Total_MWMB(nC), the shot time with the chosen tile
(Total) and the amortisation rule: a larger candidate set pays off only
after (Total_MWMB(nC') - Total_MWMB(nC)) / (Total(nC) - Total(nC')) shots.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--radius", type=int, default=5, choices=[4, 5])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--parts", type=int, default=5, help="P, parts per tile axis (Sec. 3.7)")
    ap.add_argument("--iterations", type=int, default=8, help="nI, sweeps timed per candidate")
    ap.add_argument("--streams", type=int, default=4, help="C, concurrent streams ('cores')")
    ap.add_argument("--groups", type=int, default=2, help="N, candidate groups ('nodes')")
    ap.add_argument("--repeat", type=int, default=3, help="timed shots per row")
    ap.add_argument("--study", choices=["modes", "nc"], default="modes",
                    help="modes: every selection mode at --parts; nc: MWMB at several P (Sec. 3.7)")
    ap.add_argument("--parts-list", type=str, default="2,3,5,10", help="--study nc: the values of P")
    args = ap.parse_args(argv)

    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1310_8232_gb300 import binding as st
    from paper_1310_8232_gb300 import workloads

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n, R = args.n, args.radius
    v = torch.from_numpy(workloads.layered_velocity(n, n, n, seed=1310)).cuda()
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    rows = [
        ("naive kernel (no blocking)", dict(tile=(st.STENCIL_KERNEL_NAIVE, 0, 0, 0))),
        ("poor tile 128x4, one z-chunk", dict(tile=(st.STENCIL_KERNEL_TILED, 128, 4, 0))),
        ("default tile", dict()),
        ("own tuner", dict(tune_mode=st.STENCIL_TUNE_OWN)),
        ("MWMB", dict(tune_mode=st.STENCIL_TUNE_MWMB)),
        ("OB", dict(tune_mode=st.STENCIL_TUNE_OB)),
        ("MMMB", dict(tune_mode=st.STENCIL_TUNE_MMMB)),
        ("MAMB", dict(tune_mode=st.STENCIL_TUNE_MAMB)),
        ("exhaustive", dict(tune_mode=st.STENCIL_TUNE_EXHAUSTIVE)),
    ]
    if args.study == "nc":
        rows = [("default tile", dict(), args.parts)] + [
            (f"MWMB P={P}", dict(tune_mode=st.STENCIL_TUNE_MWMB), P)
            for P in (int(x) for x in args.parts_list.split(","))]
    else:
        rows = [(name, kw, args.parts) for name, kw in rows]
    pts = float(n) ** 3 * args.steps
    results = []
    for name, kw, parts in rows:
        d = st.make_desc(v, dt, radius=R, dx=workloads.DX, graph_steps=20, stream=stream.cuda_stream, **kw)
        d.tune.parts, d.tune.iterations = parts, args.iterations
        d.tune.streams, d.tune.groups = args.streams, args.groups
        plan = st.stencil_plan(d)
        try:
            s = st.stencil_get_stats(plan)
            st.stencil_set_fields(plan, None, None, 0)
            st.stencil_step(plan, args.steps)           # warm-up shot
            times = []
            for _ in range(args.repeat):
                st.stencil_set_fields(plan, None, None, 0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st.stencil_step(plan, args.steps)
                b.record(stream)
                st.stencil_sync(plan)
                times.append(a.elapsed_time(b))
        finally:
            st.stencil_destroy(plan)
        ms = min(times)

        def num(x):
            return None if x is None or not math.isfinite(x) else x

        row = {
            "row": name, "tile": {"kernel": s.tile.kernel, "tx": s.tile.tx, "ty": s.tile.ty,
                                  "zchunk": s.tile.zchunk},
            "shot_ms": ms, "gpts_per_s": pts / (ms / 1e3) / 1e9,
            "selection_ms": num(s.selection_ms), "candidates": s.n_candidates,
            "min_time_ms": num(s.min_time_ms), "actual_time_ms": num(s.actual_time_ms),
            "quality": num(s.quality), "full_time_ms": num(s.full_time_ms),
            "config": {"n": n, "radius": R, "steps": args.steps, "P": parts, "nI": args.iterations,
                       "C": args.streams, "N": args.groups},
        }
        results.append(row)
        print(json.dumps(row), flush=True)
    if args.study == "nc":
        # the paper's amortisation rule between consecutive candidate sets,
        # and against taking the default tile with no selection at all
        base = results[0]
        prev = None
        for r in results[1:]:
            out = {"row": r["row"] + " amortisation", "candidates": r["candidates"]}
            for label, other in (("vs_default", base), ("vs_previous_P", prev)):
                if other is None:
                    continue
                extra_ms = (r["selection_ms"] or 0.0) - (other["selection_ms"] or 0.0)
                gain_ms = other["shot_ms"] - r["shot_ms"]
                out[label] = {"extra_selection_ms": extra_ms, "gain_per_shot_ms": gain_ms,
                              "shots_to_break_even": extra_ms / gain_ms if gain_ms > 0 else None}
            prev = r
            print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
