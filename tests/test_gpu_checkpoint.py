"""Checkpoint / restore of the time loop's state: a plan restored from a
checkpoint continues bit for bit as the plan that wrote it."""
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


def make(env, shape=(67, 45, 33), R=5, storage=0, graph=0, seed=3):
    torch, st = env
    nx, ny, nz = shape
    v = workloads.layered_velocity(nx, ny, nz, seed=seed)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, src=(nx // 3, ny // 2, nz // 2), storage=storage, graph_steps=graph,
                     tile=(2, 64, 16, -1),
                     stream=torch.cuda.current_stream().cuda_stream)
    return st.stencil_plan(d), v


def fields(st, plan, like):
    a, b = np.empty_like(like), np.empty_like(like)
    st.stencil_get_field(plan, 0, a)
    st.stencil_get_field(plan, 1, b)
    return a, b


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("R", [4, 5])
def test_restore_continues_bit_for_bit(env, storage, R):
    torch, st = env
    a, v = make(env, R=R, storage=storage, graph=0)
    b, _ = make(env, R=R, storage=storage, graph=6)
    try:
        st.stencil_step(a, 17)
        ck = st.stencil_checkpoint(a)
        esize = 4 if storage == 0 else 2
        extra = 0 if storage == 0 else v.shape[0] * 16
        assert ck.nbytes == st.stencil_checkpoint_size(a) == 128 + 2 * v.size * esize + extra
        assert bytes(ck[:8]) == b"STNCKPT1"
        st.stencil_step(a, 13)
        want = fields(st, a, v)
        st.stencil_restore(b, ck)
        assert st.stencil_get_stats(b).steps_done == 17
        st.stencil_step(b, 13)
        got = fields(st, b, v)
        assert st.stencil_get_stats(b).steps_done == 30
        assert np.array_equal(want[0], got[0]) and np.array_equal(want[1], got[1])
        # back to step 17 on the plan that wrote it, now through device memory
        dev = torch.from_numpy(ck).cuda()
        st.stencil_restore(a, dev)
        st.stencil_step(a, 13)
        again = fields(st, a, v)
        assert np.array_equal(want[0], again[0]) and np.array_equal(want[1], again[1])
        out = torch.empty(ck.nbytes, dtype=torch.uint8, device="cuda")
        st.stencil_checkpoint(a, out)
        assert np.array_equal(out.cpu().numpy()[128:], st.stencil_checkpoint(b)[128:])
    finally:
        st.stencil_destroy(a)
        st.stencil_destroy(b)


def test_restore_rejects_other_plans_and_short_buffers(env):
    torch, st = env
    a, v = make(env)
    other, _ = make(env, shape=(66, 45, 33))
    half, _ = make(env, storage=1)
    try:
        st.stencil_step(a, 5)
        ck = st.stencil_checkpoint(a)
        for plan in (other, half):
            with pytest.raises(st.StencilError) as ei:
                st.stencil_restore(plan, ck)
            assert ei.value.code == st.STENCIL_EINVAL
        with pytest.raises(st.StencilError):
            st.stencil_restore(a, ck[:-1].copy())
        bad = ck.copy()
        bad[0] ^= 1
        with pytest.raises(st.StencilError):
            st.stencil_restore(a, bad)
        with pytest.raises(st.StencilError):
            st.stencil_checkpoint(a, np.empty(ck.nbytes - 1, dtype=np.uint8))
        # a refused restore leaves the plan as it was
        assert st.stencil_get_stats(a).steps_done == 5
        u = np.empty_like(v)
        st.stencil_get_field(a, 0, u)
        assert np.array_equal(u.view(np.uint8).ravel()[: 4 * 67], ck[128: 128 + 4 * 67])
    finally:
        for p in (a, other, half):
            st.stencil_destroy(p)


def test_user_buffers_run_in_place(env):
    """Caller-owned (torch) buffers: the plan sweeps them in place and gives
    the same result as a plan on its own allocations."""
    torch, st = env
    nx, ny, nz, R = 68, 45, 33, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=11)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    s = torch.cuda.current_stream().cuda_stream
    bufs = [torch.full((nz, ny, nx), 7.0, device="cuda") for _ in range(3)]
    tile = (2, 64, 16, -1)
    own = st.stencil_plan(st.make_desc(v, dt, radius=R, stream=s, tile=tile))
    mine = st.stencil_plan(st.make_desc(v, dt, radius=R, stream=s, buffers=bufs, graph_steps=4, tile=tile))
    try:
        stats = st.stencil_get_stats(mine)
        assert stats.user_buffers == 1 and stats.pitch == nx
        assert torch.count_nonzero(bufs[0]) == 0 and torch.count_nonzero(bufs[1]) == 0
        kappa = (v.astype(np.float64) ** 2 * dt * dt / workloads.DX ** 2)
        assert np.allclose(bufs[2].cpu().numpy(), kappa, rtol=1e-6, atol=0)
        for steps in (11, 12):
            want = np.empty_like(v)
            st.stencil_run(own, steps, want)
            st.stencil_step(mine, steps)
            st.stencil_sync(mine)
            cur = st.stencil_get_stats(mine).current_buffer
            assert np.array_equal(bufs[cur].cpu().numpy(), want)
            prev = np.empty_like(v)
            st.stencil_get_field(own, 1, prev)
            assert np.array_equal(bufs[cur ^ 1].cpu().numpy(), prev)
    finally:
        st.stencil_destroy(own)
        st.stencil_destroy(mine)
    assert bufs[0].is_cuda            # still the caller's after the plan is gone


def test_user_buffers_rejected_when_unusable(env):
    torch, st = env
    s = torch.cuda.current_stream().cuda_stream
    v = workloads.constant_velocity(67, 20, 20, 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(5), workloads.DX, 2000.0)
    odd = [torch.zeros((20, 20, 67), device="cuda") for _ in range(3)]
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v, dt, stream=s, buffers=odd))            # nx not a multiple of 4
    assert ei.value.code == st.STENCIL_EINVAL
    v4 = workloads.constant_velocity(68, 20, 20, 2000.0)
    ok = [torch.zeros((20, 20, 68), device="cuda") for _ in range(3)]
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v4, dt, stream=s, buffers=ok, storage=1))
    assert ei.value.code == st.STENCIL_EUNSUPPORTED
    d = st.make_desc(v4, dt, stream=s, buffers=ok)
    d.user_buffers[2] = None
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == st.STENCIL_EINVAL
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v4, dt, stream=s, buffers=[ok[0], ok[0], ok[2]]))
    assert ei.value.code == st.STENCIL_EINVAL
