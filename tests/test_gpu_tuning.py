"""Tile selection on the GPU (Sec. 3.2-3.3 methodology on tile parameters):
every mode picks a feasible tile, reports MinTime / ActualTime / quality, and
the tuned plan still matches the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1310_8232_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_8232_gb300 import binding as st
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    return torch, st


MODES = ["OWN", "MWMB", "OB", "MMMB", "MAMB", "EXHAUSTIVE"]


@pytest.mark.parametrize("mode", MODES)
def test_tuned_plan_picks_feasible_tile_and_matches_oracle(env, mode):
    torch, st = env
    nx, ny, nz, R = 96, 80, 72, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=1310)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, tune_mode=getattr(st, f"STENCIL_TUNE_{mode}"),
                     stream=torch.cuda.current_stream().cuda_stream)
    d.tune.iterations = 4
    d.tune.streams = 3
    d.tune.groups = 2
    plan = st.stencil_plan(d)
    try:
        s = st.stencil_get_stats(plan)
        assert s.tile.kernel == st.STENCIL_KERNEL_TILED
        assert s.tile.tx in (32, 64, 128) and s.tile.ty in (4, 8, 16, 32)
        assert 1 <= s.tile.zchunk <= nz
        assert s.n_candidates > 0
        for f in (s.min_time_ms, s.actual_time_ms, s.full_time_ms, s.selection_ms):
            assert math.isfinite(f) and f > 0
        assert s.quality == pytest.approx((s.actual_time_ms - s.min_time_ms) / s.min_time_ms)
        out = np.empty_like(v)
        st.stencil_run(plan, 30, out)       # the fields were cleared after tuning
    finally:
        st.stencil_destroy(plan)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 30)
    assert oracle.rel_l2(out, ref) <= 1e-5


def test_exhaustive_is_no_slower_than_default_on_full_grid(env):
    """The exhaustive search's pick, timed on the full grid, is within noise
    of (or better than) the default tile."""
    torch, st = env
    n, R = 160, 5
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, tune_mode=st.STENCIL_TUNE_EXHAUSTIVE,
                     stream=torch.cuda.current_stream().cuda_stream)
    d.tune.iterations = 6
    plan = st.stencil_plan(d)
    try:
        s = st.stencil_get_stats(plan)
        assert s.n_candidates >= 20
        assert s.full_time_ms <= 1.5 * s.min_time_ms
    finally:
        st.stencil_destroy(plan)


def z_axis(nz: int) -> list[int]:
    """The admissible z-chunk values of the candidate space: 8, 12, 16, 24,
    32, 48, ... (powers of two and 1.5 times them) below nz, then nz."""
    out, v = [], 8
    while v < nz:
        out.append(v)
        if v + v // 2 < nz:
            out.append(v + v // 2)
        v *= 2
    return out + [nz]


def expected_nc(st, R: int, nz: int, P: int) -> int:
    """nC of Sec. 3.7 on the tile space: the P-part rule on each axis list
    (positions into tx = 32, 64, 128; ty = 4, 8, 16, 32; the z-chunk list),
    keeping the (tx, ty) pairs the library builds."""
    from oracle import selection
    pick = lambda vals: [vals[i - 1] for i in selection.candidates_1d(len(vals), P)]
    pairs = [(tx, ty) for tx in pick([32, 64, 128]) for ty in pick([4, 8, 16, 32])
             if st.stencil_tile_info(R, tx, ty) is not None]
    return len(pairs) * len(pick(z_axis(nz)))


def test_candidate_count_study(env, capsys):
    """The paper's study of the number of candidates (Sec. 3.7, Table 6) on a
    small grid: nC follows the P-part rule, the selection cost Total_MWMB
    grows with nC, and the amortisation count is (extra selection time) /
    (time saved per shot) on the printed times."""
    import json
    from paper_1310_8232_gb300 import tile_report
    torch, st = env
    n, R = 96, 5
    rc = tile_report.main(["--study", "nc", "--n", str(n), "--radius", str(R), "--steps", "10",
                           "--parts-list", "2,3", "--iterations", "2", "--repeat", "1", "--streams", "2"])
    assert rc == 0
    rows = [json.loads(line) for line in capsys.readouterr().out.splitlines() if line.startswith("{")]
    by = {r["row"]: r for r in rows}
    base, p2, p3 = by["default tile"], by["MWMB P=2"], by["MWMB P=3"]
    assert p2["candidates"] == expected_nc(st, R, n, 2)
    assert p3["candidates"] == expected_nc(st, R, n, 3)
    assert p3["candidates"] > p2["candidates"]
    assert p3["selection_ms"] > p2["selection_ms"] > 0
    for r in (p2, p3):
        assert r["tile"]["kernel"] == st.STENCIL_KERNEL_TILED and r["shot_ms"] > 0
    am = by["MWMB P=3 amortisation"]
    for label, other in (("vs_default", base), ("vs_previous_P", p2)):
        extra = p3["selection_ms"] - (other["selection_ms"] or 0.0)
        gain = other["shot_ms"] - p3["shot_ms"]
        got = am[label]
        assert got["extra_selection_ms"] == pytest.approx(extra)
        assert got["gain_per_shot_ms"] == pytest.approx(gain)
        if gain > 0:
            assert got["shots_to_break_even"] == pytest.approx(extra / gain)
        else:
            assert got["shots_to_break_even"] is None


def test_mwmb_pick_close_to_exhaustive(env):
    """MWMB's tile (streams on full-depth row slabs) timed on the full grid is
    within 10 % of the exhaustive search's best full-grid time (Sec. 3.5
    compares the methodology's pick with the best block found by search)."""
    torch, st = env
    n, R = 384, 5
    v = torch.from_numpy(workloads.layered_velocity(n, n, n, seed=1310)).cuda()
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    stream = torch.cuda.current_stream()
    tiles = {}
    for mode in ("MWMB", "EXHAUSTIVE"):
        d = st.make_desc(v, dt, radius=R, tune_mode=getattr(st, f"STENCIL_TUNE_{mode}"), stream=stream.cuda_stream)
        d.tune.iterations = 8
        plan = st.stencil_plan(d)
        try:
            t = st.stencil_get_stats(plan).tile
            tiles[mode] = (t.kernel, t.tx, t.ty, t.zchunk)
        finally:
            st.stencil_destroy(plan)
    # each pick timed again on the full grid: best of three 20-step runs
    full = {}
    for mode, tile in tiles.items():
        plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=tile, graph_steps=20, stream=stream.cuda_stream))
        try:
            st.stencil_step(plan, 20)
            best = float("inf")
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st.stencil_step(plan, 20)
                b.record(stream)
                st.stencil_sync(plan)
                best = min(best, a.elapsed_time(b))
            full[mode] = best
        finally:
            st.stencil_destroy(plan)
    print(f"\nMWMB {tiles['MWMB']} {full['MWMB']:.3f} ms, exhaustive {tiles['EXHAUSTIVE']} "
          f"{full['EXHAUSTIVE']:.3f} ms per 20 steps")
    assert full["MWMB"] <= 1.10 * full["EXHAUSTIVE"], (tiles, full)
