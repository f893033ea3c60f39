"""The plan's coefficient setup: kappa = v^2 dt^2 / dx^2 in FP32 over the
pitched copy of v (Section 2's wave equation written with the update
coefficient), the largest velocity and the count of invalid velocities,
on the two row layouts plans give the setup kernel: rows of whole 16-byte
vectors (user buffers, pitch = nx, nx % 4 == 0) and vectors followed by a
scalar tail (owned 128-byte rows, nx % 4 != 0).  Field parity on ragged and
tiny grids (nx = 1, 4, 5, 9, 33, 67) covers the tail's kappa too.
"""
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


def random_velocity(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)


def ulp_distance(a, b):
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("nx", [64, 68, 72])
def test_kappa_is_the_nearest_float(env, nx):
    """Against the FP64 product rounded once: at most 1 ulp anywhere and
    equal at all but a handful of near-midpoint points (nx = 68, 72: rows
    of 17 and 18 vectors, part of a warp's lanes idle)."""
    torch, st = env
    ny, nz, R = 19, 11, 5
    v = random_velocity(nx, ny, nz, seed=nx)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    s = torch.cuda.current_stream().cuda_stream
    bufs = [torch.zeros((nz, ny, nx), device="cuda") for _ in range(3)]
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, stream=s, buffers=bufs))
    try:
        st.stencil_sync(plan)
        got = bufs[2].cpu().numpy()
        want = (v.astype(np.float64) ** 2 * (dt * dt / workloads.DX ** 2)).astype(np.float32)
        d = ulp_distance(got, want)
        assert d.max() <= 1
        assert np.count_nonzero(d) <= 4
        assert st.stencil_get_stats(plan).vmax == float(v.max())
    finally:
        st.stencil_destroy(plan)


@pytest.mark.parametrize("nx, xs, user", [(70, (5, 69), False), (67, (66,), False), (72, (0, 71), True)])
def test_invalid_velocities_are_counted_in_every_part_of_a_row(env, nx, xs, user):
    """Bad values where the 16-byte loads reach and in the row's scalar tail
    (owned rows, nx = 70: vectors up to x = 67; nx = 67: up to x = 63): each
    is counted once (the error message carries the count)."""
    torch, st = env
    ny, nz = 9, 7
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    for i, x in enumerate(xs):
        v[2 + i, 3 + i, x] = (-1.0, float("nan"))[i]
    s = torch.cuda.current_stream().cuda_stream
    kw = {"buffers": [torch.zeros((nz, ny, nx), device="cuda") for _ in range(3)]} if user else {}
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v, 1e-3, radius=4, stream=s, **kw))
    assert ei.value.code == st.STENCIL_EINVAL
    assert f"{len(xs)} velocities" in str(ei.value)
