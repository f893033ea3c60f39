"""The two-step sweep (temporal blocking, STENCIL_KERNEL_TWO_STEP) against the
FP64 oracle, element by element, through the C-ABI.

Two time steps per launch: the first on the tile plus a ring of R points, the
second on the tile.  Same FP32 bar as the one-step kernel: relative L2 <=
1e-5 and every element within 1e-5 * max|ref|."""
import time

import numpy as np
import pytest

import oracle
from paper_1310_8232_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def stream(torch):
    return torch.cuda.current_stream().cuda_stream


def check(got, ref, tol=TOL):
    err = oracle.rel_l2(got, ref)
    assert err <= tol, f"relative L2 {err:.3e}"
    scale = np.max(np.abs(ref))
    assert scale > 0
    worst = np.max(np.abs(got.astype(np.float64) - ref))
    assert worst <= tol * scale, f"max abs error {worst:.3e} vs scale {scale:.3e}"
    return err


def two_step(st, zchunk=-1):
    return (st.STENCIL_KERNEL_TWO_STEP, 0, 0, zchunk)


def tile_y(R):
    return 14 if R == 5 else 16


def run(env, v, dt, R, steps, src, zchunk=-1, graph=0, u0=None, um1=None, n0=0):
    torch, st = env
    d = st.make_desc(v, dt, radius=R, src=src, tile=two_step(st, zchunk), graph_steps=graph, stream=stream(torch))
    plan = st.stencil_plan(d)
    try:
        if u0 is not None:
            st.stencil_set_fields(plan, u0, um1, step=n0)
        out = np.empty_like(v)
        st.stencil_run(plan, steps, out)
        prev = np.empty_like(v)
        st.stencil_get_field(plan, 1, prev)
        stats = st.stencil_get_stats(plan)
    finally:
        st.stencil_destroy(plan)
    return out, prev, stats


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("steps", [30, 31])
@pytest.mark.parametrize("zchunk", [-1, 7])
def test_ragged_grid_matches_oracle(env, R, steps, zchunk):
    """67 x 45 x 33 (no dimension a multiple of the tile), source on a tile
    corner; an odd count ends with one step of the one-step kernel."""
    torch, st = env
    nx, ny, nz = 67, 45, 33
    v = workloads.layered_velocity(nx, ny, nz, seed=71)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    src = (64, tile_y(R), 14)                       # first column and row of the next tile
    got, prev, s = run(env, v, dt, R, steps, src, zchunk=zchunk)
    assert s.tile.kernel == st.STENCIL_KERNEL_TWO_STEP and s.tile.tx == 64 and s.tile.ty == tile_y(R)
    ref, ref_prev = oracle.run(v, workloads.DX, dt, R, steps, src=src)
    check(got, ref)
    check(prev, ref_prev)


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("src", [(63, 20, 16), (0, 0, 0), (66, 44, 32), (31, 13, 7)])
def test_source_on_tile_and_grid_edges(env, R, src):
    torch, st = env
    nx, ny, nz = 67, 45, 33
    v = workloads.layered_velocity(nx, ny, nz, seed=72)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    got, _, _ = run(env, v, dt, R, 24, src, zchunk=8)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 24, src=src)
    check(got, ref)


@pytest.mark.parametrize("shape", [(1, 1, 40), (5, 5, 5), (9, 11, 1), (64, 14, 3), (130, 33, 2)])
def test_degenerate_grids(env, shape):
    torch, st = env
    nx, ny, nz = shape
    R = 5
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, 2000.0)
    u0 = workloads.random_field(nx, ny, nz, seed=3)
    um1 = workloads.random_field(nx, ny, nz, seed=4)
    src = (nx // 2, ny // 2, nz // 2)
    got, _, _ = run(env, v, dt, R, 9, src, u0=u0, um1=um1, n0=5)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 9, src=src, u0=u0, um1=um1, n0=5)
    check(got, ref)


def test_graph_replay_is_bit_identical_to_eager(env):
    torch, st = env
    n, R = 70, 5
    v = workloads.layered_velocity(n, n, n, seed=73)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    src = (n // 2, n // 2, n // 2)
    a, ap, _ = run(env, v, dt, R, 26, src, graph=0)
    b, bp, _ = run(env, v, dt, R, 26, src, graph=6)
    assert np.array_equal(a, b) and np.array_equal(ap, bp)


def test_split_runs_and_odd_counts(env):
    """7 + 1 + 9 + 13 steps (the levels change order in their pair after an
    odd count and back after the next two-step launch) against one oracle
    run; the fields read back between calls are the oracle's levels."""
    torch, st = env
    n, R = 72, 4
    v = workloads.layered_velocity(n, n, n, seed=74)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    src = (n // 3, n // 2, n // 2)
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, tile=two_step(st), graph_steps=4,
                                        stream=stream(torch)))
    done = 0
    u = up = None
    try:
        for k in (7, 1, 9, 13):
            st.stencil_step(plan, k)
            got, prev = np.empty_like(v), np.empty_like(v)
            st.stencil_get_field(plan, 0, got)
            st.stencil_get_field(plan, 1, prev)
            u, up = oracle.run(v, workloads.DX, dt, R, k, src=src, u0=u, um1=up, n0=done)
            done += k
            check(got, u)
            check(prev, up)
        assert st.stencil_get_stats(plan).steps_done == 30
    finally:
        st.stencil_destroy(plan)


@pytest.mark.parametrize("R", [5, 4])
@pytest.mark.parametrize("k", [2, 3])
def test_full_size_512_cube_sampled_points(env, R, k):
    """512^3 layered model in the benchmark's launch configuration
    (graph-captured steps, the library's z-chunk): k steps from random
    states, ~200 sampled points against the oracle evaluated point by point
    on the sub-cube that can reach each point."""
    torch, st = env
    from test_gpu_parity import local_oracle, sample_points
    n = 512
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.random_field(n, n, n, seed=33)
    um1 = workloads.random_field(n, n, n, seed=34)
    src = (n // 2, n // 2, n // 2)
    d = st.make_desc(torch.from_numpy(v).cuda(), dt, radius=R, tile=two_step(st), graph_steps=2,
                     stream=stream(torch))
    plan = st.stencil_plan(d)
    try:
        st.stencil_set_fields(plan, torch.from_numpy(u0).cuda(), torch.from_numpy(um1).cuda(), step=60)
        out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        st.stencil_run(plan, k, out)
        got = out.cpu().numpy()
    finally:
        st.stencil_destroy(plan)
    errs = []
    pts = sample_points(n, n, n, 200, seed=8) + [(64 * 3, tile_y(R) * 5, 100), (64 * 3 - 1, tile_y(R) * 5 - 1, 99)]
    for p in pts:
        ref = local_oracle(v, u0, um1, p, R, k, dt, n0=60, src=src)
        g = got[p[2], p[1], p[0]]
        errs.append(abs(g - ref) / max(1.0, abs(ref)))
    assert max(errs) < 1e-5, max(errs)


def test_wait_that_runs_out_reports_timeout_and_plan_recovers(env):
    torch, st = env
    n, R = 64, 5
    v = workloads.layered_velocity(n, n, n, seed=75)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=two_step(st), graph_steps=4, stream=stream(torch)))
    try:
        st.stencil_debug_wait_fault(plan, True, 20_000_000)        # 20 ms wait limit
        t0 = time.perf_counter()
        st.stencil_step(plan, 2)
        with pytest.raises(st.StencilError) as ei:
            st.stencil_sync(plan)
        assert ei.value.code == st.STENCIL_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        st.stencil_sync(plan)
        st.stencil_debug_wait_fault(plan, False, 0)
        st.stencil_set_fields(plan, None, None, 0)
        out = np.empty_like(v)
        st.stencil_run(plan, 12, out)
    finally:
        st.stencil_destroy(plan)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 12)
    check(out, ref)


def test_refused_combinations(env):
    torch, st = env
    n, R = 40, 5
    v = workloads.constant_velocity(n, n, n, 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, 2000.0)
    s = stream(torch)
    for kw in (dict(storage=1), dict(absorb=(4, 0.2)), dict(tune_mode=st.STENCIL_TUNE_MWMB)):
        with pytest.raises(st.StencilError) as ei:
            st.stencil_plan(st.make_desc(v, dt, radius=R, tile=two_step(st), stream=s, **kw))
        assert ei.value.code == st.STENCIL_EUNSUPPORTED
    bufs = [torch.zeros((n, n, n), dtype=torch.float32, device="cuda") for _ in range(3)]
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v, dt, radius=R, tile=two_step(st), stream=s, buffers=bufs))
    assert ei.value.code == st.STENCIL_EUNSUPPORTED
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=two_step(st), stream=s))
    try:
        with pytest.raises(st.StencilError) as ei:
            st.stencil_record_start(plan, receiver_z=3, capacity=4)
        assert ei.value.code == st.STENCIL_EUNSUPPORTED
        inj = torch.zeros((4, 1, n), dtype=torch.float32, device="cuda")
        with pytest.raises(st.StencilError) as ei:
            st.stencil_inject_start(plan, 0, inj, y=1)
        assert ei.value.code == st.STENCIL_EUNSUPPORTED
    finally:
        st.stencil_destroy(plan)


def test_checkpoint_restore_continues_bit_for_bit(env):
    """A two-step plan checkpointed after an odd count (its levels sit in
    their pair the other way round) and restored into a fresh two-step plan:
    both continue with the same launches and agree bit for bit."""
    torch, st = env
    n, R = 60, 5
    v = workloads.layered_velocity(n, n, n, seed=76)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    src = (n // 2, n // 3, n // 2)
    mk = lambda: st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, tile=two_step(st), stream=stream(torch)))
    a, b = mk(), mk()
    try:
        st.stencil_step(a, 7)
        ck = st.stencil_checkpoint(a)
        st.stencil_restore(b, ck)
        outs = []
        for plan in (a, b):
            st.stencil_step(plan, 9)
            u, up = np.empty_like(v), np.empty_like(v)
            st.stencil_get_field(plan, 0, u)
            st.stencil_get_field(plan, 1, up)
            outs.append((u, up))
        assert st.stencil_get_stats(b).steps_done == 16
    finally:
        st.stencil_destroy(a)
        st.stencil_destroy(b)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ref, _ = oracle.run(v, workloads.DX, dt, R, 16, src=src)
    check(outs[0][0], ref)
