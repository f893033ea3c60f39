"""Receiver traces and per-step energy recorded by the sweep itself (the
"sismic" and energy steps of Algorithm 1's loop body)."""
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


SHAPE = (40, 36, 30)     # nx, ny, nz: ragged for every tile


def tiles(st):
    return [(st.STENCIL_KERNEL_NAIVE, 0, 0, 0), (st.STENCIL_KERNEL_TILED, 64, 16, -1),
            (st.STENCIL_KERNEL_TILED, 32, 8, 7)]


def make(env, R=5, tile=None, storage=0, graph=0, amp=1.0, shape=SHAPE, seed=4):
    torch, st = env
    nx, ny, nz = shape
    v = workloads.layered_velocity(nx, ny, nz, seed=seed)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, src=(nx // 2, ny // 3, nz // 2), amp=amp, tile=tile, storage=storage,
                     graph_steps=graph, stream=torch.cuda.current_stream().cuda_stream)
    return st.stencil_plan(d), v, dt


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_traces_are_the_fields_after_each_step(env, R, k):
    torch, st = env
    tile = tiles(st)[k]
    plan, v, dt = make(env, R=R, tile=tile)
    row, _, _ = make(env, R=R, tile=tile)
    nx, ny, nz = SHAPE
    zr, yr, steps = 17, 5, 9
    try:
        st.stencil_step(plan, 3)                   # recording starts at n0 = 3
        st.stencil_step(row, 3)
        st.stencil_record_start(plan, receiver_z=zr, capacity=steps)
        st.stencil_record_start(row, receiver_z=zr, receiver_y=yr, capacity=steps)
        fields = []
        for _ in range(steps):
            st.stencil_step(plan, 1)
            st.stencil_step(row, 1)
            u = np.empty_like(v)
            st.stencil_get_field(plan, 0, u)
            fields.append(u)
        tr = np.full((steps, ny, nx), np.nan, dtype=np.float32)
        assert st.stencil_record_read(plan, tr) == steps
        tl = np.full((steps, 1, nx), np.nan, dtype=np.float32)
        assert st.stencil_record_read(row, tl) == steps
    finally:
        st.stencil_destroy(plan)
        st.stencil_destroy(row)
    for m, u in enumerate(fields):
        assert np.array_equal(tr[m], u[zr]), m
        assert np.array_equal(tl[m, 0], u[zr, yr]), m


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_energy_matches_oracle_on_the_same_fields_and_is_conserved(env, R, k):
    torch, st = env
    tile = tiles(st)[k]
    plan, v, dt = make(env, R=R, tile=tile, amp=0.0)
    nx, ny, nz = SHAPE
    u0 = workloads.gaussian_bump(nx, ny, nz, width=3.0)
    steps = 24
    try:
        st.stencil_set_fields(plan, u0, u0, 0)
        st.stencil_record_start(plan, energy=True, capacity=steps)
        prev = u0.copy()
        want = []
        for _ in range(steps):
            st.stencil_step(plan, 1)
            u = np.empty_like(v)
            st.stencil_get_field(plan, 0, u)
            want.append(oracle.energy(v, workloads.DX, dt, R, u, prev))
            prev = u
        got = np.full(steps, np.nan)
        assert st.stencil_record_read(plan, energy=got) == steps
    finally:
        st.stencil_destroy(plan)
    want = np.array(want)
    assert np.all(np.abs(got - want) <= 2e-6 * np.abs(want)), np.max(np.abs(got - want) / np.abs(want))
    # source-free: the scheme conserves it (FP32 fields)
    assert np.max(np.abs(got - got[0])) <= 1e-4 * abs(got[0])


def test_recording_with_graphs_equals_eager_and_stops_at_capacity(env):
    torch, st = env
    outs = []
    for graph in (0, 6):
        plan, v, dt = make(env, R=5, graph=graph)
        try:
            st.stencil_record_start(plan, receiver_z=3, energy=True, capacity=10)
            st.stencil_step(plan, 17)
            tr = np.empty((10, SHAPE[1], SHAPE[0]), dtype=np.float32)
            en = np.empty(10)
            assert st.stencil_record_read(plan, tr, en) == 10
            outs.append((tr, en))
            st.stencil_record_stop(plan)
            st.stencil_step(plan, 2)                       # stepping goes on without recording
            assert st.stencil_get_stats(plan).steps_done == 19
        finally:
            st.stencil_destroy(plan)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.all(np.isfinite(outs[0][1]))


@pytest.mark.parametrize("storage", [1, 2])
def test_traces_with_16bit_storage_are_the_stored_values(env, storage):
    torch, st = env
    plan, v, dt = make(env, R=4, storage=storage)
    try:
        st.stencil_record_start(plan, receiver_z=15, capacity=12)
        st.stencil_step(plan, 12)
        tr = np.empty((12, SHAPE[1], SHAPE[0]), dtype=np.float32)
        st.stencil_record_read(plan, tr)
        u = np.empty_like(v)
        st.stencil_get_field(plan, 0, u)
    finally:
        st.stencil_destroy(plan)
    assert np.max(np.abs(u[15])) > 0
    assert np.array_equal(tr[-1], u[15])


def test_record_start_rejects_bad_requests(env):
    torch, st = env
    plan, v, dt = make(env)
    try:
        for kw in (dict(receiver_z=SHAPE[2], capacity=4), dict(receiver_z=2, receiver_y=SHAPE[1], capacity=4),
                   dict(receiver_z=2, capacity=0), dict(capacity=4)):
            with pytest.raises(st.StencilError) as ei:
                st.stencil_record_start(plan, **kw)
            assert ei.value.code == st.STENCIL_EINVAL
        with pytest.raises(st.StencilError):
            st.stencil_record_read(plan)                   # nothing started
    finally:
        st.stencil_destroy(plan)
