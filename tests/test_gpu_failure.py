"""The failure path and the bounds of every write, without a GPU fault.

- A shared-memory wait made to run out (the first copy of every block is
  expected to bring more bytes than it does) returns STENCIL_ETIMEOUT after
  the wait limit, and the plan is usable again afterwards.
- Guard bands: the plan runs on caller-owned buffers cut from larger
  tensors whose margins hold a sentinel; after sweeps with every kernel and
  every per-step operation, the margins are unchanged bit for bit.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1310_8232_gb300 import workloads

pytestmark = pytest.mark.gpu

DX = workloads.DX


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


def test_wait_that_runs_out_reports_timeout_and_plan_recovers(env):
    torch, st = env
    n, R = 64, 5
    v = workloads.layered_velocity(n, n, n, seed=61)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, float(v.max()))
    tile = (st.STENCIL_KERNEL_TILED, 64, 16, -1)
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=tile, graph_steps=4, stream=stream(torch)))
    try:
        st.stencil_debug_wait_fault(plan, True, 20_000_000)        # 20 ms wait limit
        t0 = time.perf_counter()
        st.stencil_step(plan, 1)
        with pytest.raises(st.StencilError) as ei:
            st.stencil_sync(plan)
        assert ei.value.code == st.STENCIL_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        st.stencil_sync(plan)                                      # the error word was cleared
        st.stencil_debug_wait_fault(plan, False, 0)
        st.stencil_set_fields(plan, None, None, 0)
        out = np.empty_like(v)
        st.stencil_run(plan, 12, out)
    finally:
        st.stencil_destroy(plan)
    ref, _ = oracle.run(v, DX, dt, R, 12)
    assert oracle.rel_l2(out, ref) <= 1e-5


GUARD = 1024                       # floats of margin on each side (16-byte aligned cut)
SENTINEL = np.float32(-7.25e33)


def guarded(torch, shape):
    n = int(np.prod(shape))
    big = torch.full((n + 2 * GUARD,), float(SENTINEL), dtype=torch.float32, device="cuda")
    return big, big[GUARD:GUARD + n].view(*shape)


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("tile", [(1, 0, 0, 0), (2, 64, 16, -1), (2, 32, 8, 7), (2, 128, 4, 3)],
                         ids=["naive", "64x16", "32x8z7", "128x4z3"])
def test_every_write_stays_inside_its_buffer(env, R, tile):
    torch, st = env
    nx, ny, nz = 68, 45, 33
    if tile[0] == 2 and st.stencil_tile_info(R, tile[1], tile[2]) is None:
        pytest.skip("tile not built")
    v = workloads.layered_velocity(nx, ny, nz, seed=62)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, float(v.max()))
    bigs, views = zip(*(guarded(torch, (nz, ny, nx)) for _ in range(3)))
    traces = torch.zeros((12, ny, nx), dtype=torch.float32, device="cuda")
    inj = torch.randn((12, 1, nx), dtype=torch.float32, device="cuda") * 1e-3
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=tile, buffers=list(views), absorb=(5, 0.2),
                                        graph_steps=4, src=(nx // 2, ny // 2, nz // 2), stream=stream(torch)))
    try:
        st.stencil_record_start(plan, receiver_z=nz - 1, capacity=12)
        st.stencil_inject_start(plan, 0, inj, y=ny - 1)
        st.stencil_step(plan, 12)
        st.stencil_record_read(plan, traces)
        st.stencil_sync(plan)
    finally:
        st.stencil_destroy(plan)
    for big in bigs:
        margin = torch.cat([big[:GUARD], big[-GUARD:]]).cpu().numpy()
        assert np.array_equal(margin.view(np.uint32), np.full(2 * GUARD, SENTINEL).view(np.uint32))
    assert torch.isfinite(views[0]).all() and torch.count_nonzero(views[0]) > 0
