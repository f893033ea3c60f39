"""The RTM pieces on the GPU against the FP64 oracle: absorbing layer,
plane injection, the imaging condition and a whole one-shot migration."""
import numpy as np
import pytest

import oracle
from oracle import rtm as oracle_rtm
from paper_1310_8232_gb300 import workloads

pytestmark = pytest.mark.gpu

DX = workloads.DX
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


def tiles(st):
    return [(st.STENCIL_KERNEL_NAIVE, 0, 0, 0), (st.STENCIL_KERNEL_TILED, 64, 16, -1),
            (st.STENCIL_KERNEL_TILED, 32, 8, 7)]


def check(got, ref, tol=TOL):
    err = oracle.rel_l2(got, ref)
    assert err <= tol, f"relative L2 {err:.3e}"
    return err


SHAPE = (45, 38, 33)


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_absorbing_layer_matches_oracle(env, R, k):
    torch, st = env
    nx, ny, nz = SHAPE
    v = workloads.layered_velocity(nx, ny, nz, seed=31)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, float(v.max()))
    absorb = (7, 0.25)
    src = (nx // 2, ny // 2, 9)
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, tile=tiles(st)[k], absorb=absorb,
                                        stream=stream(torch)))
    try:
        out = np.empty_like(v)
        st.stencil_run(plan, 90, out)
    finally:
        st.stencil_destroy(plan)
    ref, _, _ = oracle.run_ext(v, DX, dt, R, 90, src=src, absorb=absorb)
    check(out, ref)
    plain, _ = oracle.run(v, DX, dt, R, 90, src=src)
    assert oracle.rel_l2(ref, plain) > 1e-2            # the layer does change the field


@pytest.mark.parametrize("k", [0, 1, 2])
def test_injection_matches_oracle_forward_and_reversed(env, k):
    torch, st = env
    nx, ny, nz = SHAPE
    R = 5
    v = workloads.layered_velocity(nx, ny, nz, seed=32)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, float(v.max()))
    rng = np.random.default_rng(33)
    for y, reverse in ((-1, False), (11, True)):
        data = (rng.standard_normal((20, ny if y < 0 else 1, nx)) * 1e-3).astype(np.float32)
        plan = st.stencil_plan(st.make_desc(v, dt, radius=R, amp=0.0, tile=tiles(st)[k], absorb=(5, 0.2),
                                            stream=stream(torch)))
        try:
            st.stencil_step(plan, 2)                     # injection starts at n0 = 2
            dd = torch.from_numpy(data).cuda()
            st.stencil_inject_start(plan, 6, dd, y=y, reverse=reverse, scale=0.5)
            out = np.empty_like(v)
            st.stencil_run(plan, 25, out)                # the last 5 steps inject nothing
            st.stencil_inject_stop(plan)
        finally:
            st.stencil_destroy(plan)
        ref, _, _ = oracle.run_ext(v, DX, dt, R, 25, amp=0.0, absorb=(5, 0.2),
                                   inject=(6, y, data.astype(np.float64), reverse, 0.5))
        check(out, ref)


def test_recording_leaves_the_fields_bit_for_bit(env):
    """The record pass after each step only reads: the fields are bit for
    bit those of a plan that records nothing."""
    torch, st = env
    nx, ny, nz = SHAPE
    v = workloads.layered_velocity(nx, ny, nz, seed=34)
    dt = workloads.time_step(oracle.cfl_limit(5), DX, float(v.max()))
    outs = []
    for rec in (False, True):
        plan = st.stencil_plan(st.make_desc(v, dt, radius=5, tile=tiles(st)[1], stream=stream(torch)))
        try:
            if rec:
                st.stencil_record_start(plan, receiver_z=4, capacity=8)
            out = np.empty_like(v)
            st.stencil_run(plan, 31, out)
        finally:
            st.stencil_destroy(plan)
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])


def test_image_accumulate(env):
    torch, st = env
    nx, ny, nz = 37, 21, 19                             # pitched plan rows, dense snapshot and image
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    plan = st.stencil_plan(st.make_desc(v, 1e-3, radius=4, tile=tiles(st)[1], stream=stream(torch)))
    try:
        u = workloads.random_field(nx, ny, nz, seed=40)
        st.stencil_set_fields(plan, u, None, 0)
        s = workloads.random_field(nx, ny, nz, seed=41)
        img0 = workloads.random_field(nx, ny, nz, seed=42)
        img = torch.from_numpy(img0).cuda()
        st.stencil_image_accumulate(plan, torch.from_numpy(s).cuda(), img, 0.25)
        st.stencil_sync(plan)
        got = img.cpu().numpy()
    finally:
        st.stencil_destroy(plan)
    want = img0.astype(np.float64) + 0.25 * s.astype(np.float64) * u.astype(np.float64)
    assert np.max(np.abs(got - want)) <= 2e-7 * np.max(np.abs(want))


@pytest.mark.parametrize("k", [0, 1])
def test_one_shot_migration_matches_oracle(env, k):
    torch, st = env
    from paper_1310_8232_gb300 import rtm
    n, R = 48, 4
    v = np.full((n, n, n), 2000.0, dtype=np.float32)
    v[n // 2:] = 3000.0
    dt = workloads.time_step(oracle.cfl_limit(R), DX, 3000.0)
    T, snap, zr, src, absorb = 240, 6, 4, (n // 2, n // 2, 6), (8, 0.2)
    image, traces = rtm.migrate(torch, torch.from_numpy(v).cuda(), dt, T, src, zr, snap, radius=R, dx=DX,
                                absorb=absorb, f=25.0, tile=tiles(st)[k], graph_steps=6)
    ref_img, ref_tr, _ = oracle_rtm.migrate(v, DX, dt, R, T, src, zr, snap, absorb=absorb, f=25.0)
    # the FP32 bar for both: measured 1.4e-6 (traces) and 4.6e-7 (image)
    e_tr = check(traces.cpu().numpy(), ref_tr, TOL)
    e_img = check(image.cpu().numpy(), ref_img, TOL)
    print(f"\nmigration vs FP64 oracle: traces {e_tr:.3e}, image {e_img:.3e}")


def test_unsupported_combinations_are_refused(env):
    torch, st = env
    nx, ny, nz = 24, 20, 18
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(4), DX, 2000.0)
    s = stream(torch)
    with pytest.raises(st.StencilError) as ei:            # the layer needs FP32 storage
        st.stencil_plan(st.make_desc(v, dt, radius=4, storage=1, absorb=(4, 0.2), stream=s))
    assert ei.value.code == st.STENCIL_EUNSUPPORTED
    plan = st.stencil_plan(st.make_desc(v, dt, radius=4, absorb=(4, 0.2), stream=s))
    try:                                                   # energy only without layer / injection
        with pytest.raises(st.StencilError) as ei:
            st.stencil_record_start(plan, energy=True, capacity=4)
        assert ei.value.code == st.STENCIL_EUNSUPPORTED
    finally:
        st.stencil_destroy(plan)
    d = st.make_desc(v, dt, radius=4, absorb=(4, 0.2), storage=1, stream=s)
    with pytest.raises(st.StencilError) as ei:             # nor in a 16-bit batch
        st.stencil_batch_create([d])
    assert ei.value.code == st.STENCIL_EUNSUPPORTED
