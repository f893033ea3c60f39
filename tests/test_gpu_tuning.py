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
