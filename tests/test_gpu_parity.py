"""GPU sweep vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (FP32 arithmetic and storage against FP64):
  * relative L2 <= 1e-5 of the whole field (the stated FP32 bar);
  * every element within 1e-5 * max|ref| (absolute), which bounds the
    pointwise error where the field is small.
"""
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
    # one non-default stream, current for torch and used by every plan, so
    # that torch's copies and the plans' kernels are ordered
    torch.cuda.set_stream(torch.cuda.Stream())
    return torch, st


def run_gpu(env, v, dt, R, steps, tile="default", src=None, amp=1.0, u0=None, um1=None, n0=0,
            graph_steps=0, on_device=True):
    """tile: "default" = the tiled kernel with the library's default tile
    shape, None = the library's automatic choice (naive on small grids)."""
    torch, st = env
    if isinstance(tile, str):
        tile = DEFAULT_TILED
    vel = torch.from_numpy(v).cuda() if on_device else v
    d = st.make_desc(vel, dt, radius=R, dx=workloads.DX, src=src, amp=amp, tile=tile,
                     graph_steps=graph_steps, stream=cur_stream(torch))
    plan = st.stencil_plan(d)
    try:
        if u0 is not None or um1 is not None or n0:
            st.stencil_set_fields(plan, u0, um1, step=n0)
        out = np.empty_like(v)
        st.stencil_run(plan, steps, out)
        prev = np.empty_like(v)
        st.stencil_get_field(plan, 1, prev)
        stats = st.stencil_get_stats(plan)
    finally:
        st.stencil_destroy(plan)
    return out, prev, stats


def check(got, ref, tol=TOL):
    err = oracle.rel_l2(got, ref)
    assert err <= tol, f"relative L2 {err:.3e}"
    scale = np.max(np.abs(ref))
    assert scale > 0
    worst = np.max(np.abs(got.astype(np.float64) - ref))
    assert worst <= tol * scale, f"max abs error {worst:.3e} vs scale {scale:.3e}"
    return err


def cur_stream(torch):
    return torch.cuda.current_stream().cuda_stream


NAIVE = (1, 0, 0, 0)


def tiled(tx, ty, zc):
    return (2, tx, ty, zc)


DEFAULT_TILED = tiled(64, 16, -1)


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("tile", [NAIVE, None, "default"])
@pytest.mark.parametrize("steps", [10, 100])
def test_single_shot_64_cube(env, R, tile, steps):
    """64^3, constant 2000 m/s, dt = 0.5 CFL, Ricker at the centre."""
    n = 64
    v = workloads.constant_velocity(n, n, n, 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, 2000.0)
    got, prev, _ = run_gpu(env, v, dt, R, steps, tile=tile)
    ref, ref_prev = oracle.run(v, workloads.DX, dt, R, steps)
    check(got, ref)
    check(prev, ref_prev)


TILES = [tiled(tx, ty, zc) for tx, ty, zc in
         [(32, 4, 7), (32, 8, 0), (32, 16, 5), (32, 32, 9), (64, 4, 3), (64, 8, 11), (64, 16, 0),
          (64, 32, 13), (128, 4, 6), (128, 8, 1), (128, 16, 17)]]


@pytest.mark.parametrize("tile", TILES, ids=lambda t: f"{t[1]}x{t[2]}z{t[3]}")
@pytest.mark.parametrize("R", [4, 5])
def test_ragged_grid_every_tile(env, R, tile):
    """Grid sizes that are no multiple of any tile, zchunks that do not divide nz."""
    torch, st = env
    if st.stencil_tile_info(R, tile[1], tile[2]) is None:
        pytest.skip(f"tile {tile[1]}x{tile[2]} not built")
    nx, ny, nz = 67, 45, 33
    v = workloads.layered_velocity(nx, ny, nz, seed=21)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.random_field(nx, ny, nz, seed=3)
    um1 = workloads.random_field(nx, ny, nz, seed=4)
    steps = 12
    got, prev, _ = run_gpu(env, v, dt, R, steps, tile=tile, u0=u0, um1=um1, src=(5, 40, 30))
    ref, ref_prev = oracle.run(v, workloads.DX, dt, R, steps, src=(5, 40, 30), u0=u0, um1=um1)
    check(got, ref)
    check(prev, ref_prev)


@pytest.mark.parametrize("shape", [(1, 1, 40), (5, 5, 5), (9, 11, 1), (33, 1, 17), (4, 70, 3),
                                   (131, 2, 2), (11, 11, 11)])
@pytest.mark.parametrize("tile", [NAIVE, None, "default", tiled(128, 4, 2)])
def test_degenerate_and_tiny_grids(env, shape, tile):
    nx, ny, nz = shape
    R = 5
    v = workloads.layered_velocity(nx, ny, nz, n_layers=2, seed=5)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.random_field(nx, ny, nz, seed=8)
    got, _, _ = run_gpu(env, v, dt, R, 9, tile=tile, u0=u0, um1=u0, src=(0, 0, 0))
    ref, _ = oracle.run(v, workloads.DX, dt, R, 9, src=(0, 0, 0), u0=u0, um1=u0)
    check(got, ref)


@pytest.mark.parametrize("src", [(0, 0, 0), (66, 44, 32), (64, 3, 31)])
def test_source_at_faces_and_corners(env, src):
    nx, ny, nz, R = 67, 45, 33, 4
    v = workloads.layered_velocity(nx, ny, nz, seed=2)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    got, _, _ = run_gpu(env, v, dt, R, 60, src=src)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 60, src=src)
    check(got, ref)


def test_graph_replay_is_bit_identical_to_eager(env):
    n, R = 48, 5
    v = workloads.layered_velocity(n, n, n, seed=9)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    a, ap, _ = run_gpu(env, v, dt, R, 37, graph_steps=0)
    b, bp, _ = run_gpu(env, v, dt, R, 37, graph_steps=8)
    assert np.array_equal(a, b) and np.array_equal(ap, bp)


def test_runs_are_deterministic(env):
    n, R = 40, 4
    v = workloads.layered_velocity(n, n, n, seed=10)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    a, _, _ = run_gpu(env, v, dt, R, 25)
    b, _, _ = run_gpu(env, v, dt, R, 25)
    assert np.array_equal(a, b)


def test_host_velocity_equals_device_velocity(env):
    n, R = 32, 5
    v = workloads.layered_velocity(n, n, n, seed=12)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    a, _, _ = run_gpu(env, v, dt, R, 20, on_device=True)
    b, _, _ = run_gpu(env, v, dt, R, 20, on_device=False)
    assert np.array_equal(a, b)


def test_step_counter_resume_matches_oracle(env):
    """Start at step n0 = 7 (the source term uses t = n dt)."""
    n, R = 36, 5
    v = workloads.layered_velocity(n, n, n, seed=13)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.gaussian_bump(n, n, n)
    got, _, _ = run_gpu(env, v, dt, R, 30, u0=u0, um1=u0, n0=7)
    ref, _ = oracle.run(v, workloads.DX, dt, R, 30, u0=u0, um1=u0, n0=7)
    check(got, ref)


def test_split_runs_equal_one_run(env):
    torch, st = env
    n, R = 40, 4
    v = workloads.layered_velocity(n, n, n, seed=14)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, tile=DEFAULT_TILED, stream=cur_stream(torch))
    plan = st.stencil_plan(d)
    try:
        st.stencil_step(plan, 13)
        st.stencil_step(plan, 1)
        out = np.empty_like(v)
        st.stencil_run(plan, 16, out)
        assert st.stencil_get_stats(plan).steps_done == 30
    finally:
        st.stencil_destroy(plan)
    one, _, _ = run_gpu(env, v, dt, R, 30, on_device=False)
    assert np.array_equal(out, one)


@pytest.mark.parametrize("R", [4, 5])
def test_device_energy_matches_oracle_on_same_fields(env, R):
    torch, st = env
    n = 30
    v = workloads.layered_velocity(n, n, n, seed=15)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u1 = workloads.random_field(n, n, n, seed=1)
    u0 = workloads.random_field(n, n, n, seed=2)
    d = st.make_desc(v, dt, radius=R)
    plan = st.stencil_plan(d)
    try:
        st.stencil_set_fields(plan, u1, u0)
        e_gpu = st.stencil_energy(plan)
    finally:
        st.stencil_destroy(plan)
    e_ref = oracle.energy(v, workloads.DX, dt, R, u1, u0)
    # kappa is stored in FP32 on the device (one rounding of v^2 dt^2/dx^2)
    assert e_gpu == pytest.approx(e_ref, rel=1e-6)


def test_energy_conserved_on_device_without_source(env):
    torch, st = env
    n, R = 48, 5
    v = workloads.layered_velocity(n, n, n, n_layers=4, seed=16)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.gaussian_bump(n, n, n, width=4.0)
    d = st.make_desc(v, dt, radius=R, amp=0.0)
    plan = st.stencil_plan(d)
    try:
        st.stencil_set_fields(plan, u0, u0)
        e0 = st.stencil_energy(plan)
        energies = []
        for _ in range(5):
            st.stencil_step(plan, 100)
            energies.append(st.stencil_energy(plan))
    finally:
        st.stencil_destroy(plan)
    drift = max(abs(e - e0) for e in energies) / e0
    assert drift < 1e-4, drift


def test_device_rel_l2_matches_host(env):
    torch, st = env
    n, R = 33, 4
    v = workloads.layered_velocity(n, n, n, seed=17)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    d = st.make_desc(v, dt, radius=R, stream=cur_stream(torch))
    plan = st.stencil_plan(d)
    try:
        out = np.empty_like(v)
        st.stencil_run(plan, 40, out)
        ref, _ = oracle.run(v, workloads.DX, dt, R, 40)
        dev = st.stencil_rel_l2(plan, torch.from_numpy(ref).cuda())
    finally:
        st.stencil_destroy(plan)
    assert dev == pytest.approx(oracle.rel_l2(out, ref), rel=1e-9)


def test_time_reversal_on_device(env):
    torch, st = env
    n, R, N = 40, 5, 80
    v = workloads.layered_velocity(n, n, n, seed=18)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.gaussian_bump(n, n, n)
    d = st.make_desc(v, dt, radius=R, amp=0.0)
    plan = st.stencil_plan(d)
    try:
        st.stencil_set_fields(plan, u0, u0)
        st.stencil_step(plan, N)
        u = np.empty_like(v)
        up = np.empty_like(v)
        st.stencil_get_field(plan, 0, u)
        st.stencil_get_field(plan, 1, up)
        st.stencil_set_fields(plan, up, u)
        st.stencil_step(plan, N)
        back = np.empty_like(v)
        st.stencil_get_field(plan, 1, back)
    finally:
        st.stencil_destroy(plan)
    np.testing.assert_allclose(back, u0, rtol=0, atol=1e-4)


def test_plan_rejects_unstable_dt(env):
    torch, st = env
    v = workloads.constant_velocity(16, 16, 16, 3000.0)
    dt = 1.01 * oracle.cfl_limit(5) * workloads.DX / 3000.0
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v, dt, radius=5))
    assert ei.value.code == st.STENCIL_ECFL


@pytest.mark.parametrize("bad", [0.0, -5.0, float("nan"), float("inf")])
def test_plan_rejects_invalid_velocity(env, bad):
    torch, st = env
    v = workloads.constant_velocity(16, 16, 16, 2000.0)
    v[3, 4, 5] = bad
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(st.make_desc(v, 1e-3, radius=4))
    assert ei.value.code == st.STENCIL_EINVAL


def sample_points(nx, ny, nz, count, seed):
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz // 2), (0, ny - 1, 1),
           (nx // 2, ny // 2, nz // 2), (nx // 2, ny // 2, 0), (3, ny - 4, nz - 2)]
    for _ in range(count):
        pts.append((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    return pts


def local_oracle(v, u0, um1, p, R, k, dt, n0=0, src=None):
    """Oracle value at point p after k steps, from the sub-cube of half-width
    k*R around p (values outside it cannot reach p in k steps)."""
    nz, ny, nx = v.shape
    W = k * R
    x, y, z = p
    xs, ys, zs = slice(max(0, x - W), min(nx, x + W + 1)), slice(max(0, y - W), min(ny, y + W + 1)), \
        slice(max(0, z - W), min(nz, z + W + 1))
    # the sub-cube keeps the true boundary where it touches a face; its cut
    # faces are at distance W, which the dependency cone never reaches
    sub = (zs, ys, xs)
    ls = None
    if src is not None:
        ls = (src[0] - xs.start, src[1] - ys.start, src[2] - zs.start)
        inside = all(0 <= ls[i] < (xs, ys, zs)[i].stop - (xs, ys, zs)[i].start for i in range(3))
        if not inside:
            ls = None
    amp = 1.0 if ls is not None else 0.0
    out, _ = oracle.run(v[sub], workloads.DX, dt, R, k, src=ls or (0, 0, 0), amp=amp,
                        u0=u0[sub], um1=um1[sub], n0=n0)
    return out[z - zs.start, y - ys.start, x - xs.start]


@pytest.mark.parametrize("R", [5, 4])
def test_full_size_512_cube_sampled_points(env, R):
    """512^3 layered model in the benchmark's launch configuration (default
    tile, graph-captured steps): 2 steps from random states, ~200 sampled
    points checked against the oracle evaluated point by point."""
    torch, st = env
    n, k = 512, 2
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.random_field(n, n, n, seed=31)
    um1 = workloads.random_field(n, n, n, seed=32)
    src = (n // 2, n // 2, n // 2)
    d = st.make_desc(torch.from_numpy(v).cuda(), dt, radius=R, graph_steps=2, stream=cur_stream(torch))
    plan = st.stencil_plan(d)
    try:
        st.stencil_set_fields(plan, torch.from_numpy(u0).cuda(), torch.from_numpy(um1).cuda(), step=60)
        out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        st.stencil_run(plan, k, out)
        got = out.cpu().numpy()
    finally:
        st.stencil_destroy(plan)
    errs = []
    for p in sample_points(n, n, n, 200, seed=7):
        ref = local_oracle(v, u0, um1, p, R, k, dt, n0=60, src=src)
        g = got[p[2], p[1], p[0]]
        errs.append(abs(g - ref) / max(1.0, abs(ref)))
    assert max(errs) < 1e-5, max(errs)


def test_automatic_kernel_choice_by_grid_size(env):
    """FP32 grids of at most 2^20 points take the one-pass naive kernel
    (latency-bound), larger ones and 16-bit storage the tiled kernel."""
    torch, st = env
    for shape, storage, kernel in (((64, 64, 64), 0, NAIVE[0]), ((128, 64, 128), 0, NAIVE[0]),
                                   ((102, 102, 102), 0, 2), ((64, 64, 64), 1, 2)):
        v = workloads.constant_velocity(*shape, 2000.0)
        dt = workloads.time_step(oracle.cfl_limit(4), workloads.DX, 2000.0)
        plan = st.stencil_plan(st.make_desc(v, dt, radius=4, storage=storage, stream=cur_stream(torch)))
        try:
            assert st.stencil_get_stats(plan).tile.kernel == kernel, (shape, storage)
        finally:
            st.stencil_destroy(plan)


def test_set_velocity_replaces_the_model_with_graphs_captured(env):
    """A new model through stencil_set_velocity gives what a fresh plan on
    that model gives, whether or not its source-point velocity changed (the
    captured graphs are kept only when nothing they carry changed)."""
    torch, st = env
    nx, ny, nz, R = 48, 40, 36, 5
    src = (20, 20, 18)
    a = workloads.layered_velocity(nx, ny, nz, seed=51)
    b = a.copy()
    b[:, :, : nx // 2] *= 0.9                      # same velocity at the source, different elsewhere
    c = workloads.layered_velocity(nx, ny, nz, seed=52)   # different at the source too
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(max(a.max(), c.max())))

    def fresh(v):
        got, _, _ = run_gpu(env, v, dt, R, 24, src=src, graph_steps=6, on_device=False)
        return got

    d = st.make_desc(a, dt, radius=R, src=src, tile=DEFAULT_TILED, graph_steps=6, stream=cur_stream(torch))
    plan = st.stencil_plan(d)
    try:
        st.stencil_step(plan, 12)                   # graphs captured on model a
        for v in (b, c, a):
            st.stencil_set_velocity(plan, v)
            st.stencil_set_fields(plan, None, None, 0)
            out = np.empty_like(v)
            st.stencil_run(plan, 24, out)
            assert np.array_equal(out, fresh(v))
    finally:
        st.stencil_destroy(plan)


@pytest.mark.parametrize("tile", [NAIVE, DEFAULT_TILED, (3, 0, 0, -1)])
def test_reset_to_zero_fields_at_a_step_equals_a_fresh_start(env, tile):
    """stencil_set_fields with no arrays (one launch clears both levels and
    sets the step counter, with no host wait): after 7 steps, a reset to
    step 3 followed by 5 steps gives the fields of a fresh plan set to step 3
    and run 5 steps, bit for bit (the source term follows the counter)."""
    torch, st = env
    nx, ny, nz, R = 52, 37, 29, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=77)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    out = []
    for warm in (7, 0):
        plan = st.stencil_plan(st.make_desc(v, dt, radius=R, tile=tile, graph_steps=2, stream=cur_stream(torch)))
        try:
            st.stencil_step(plan, warm)
            st.stencil_set_fields(plan, None, None, 3)
            assert st.stencil_get_stats(plan).steps_done == 3
            u = np.empty_like(v)
            st.stencil_run(plan, 5, u)
            um1 = np.empty_like(v)
            st.stencil_get_field(plan, 1, um1)
            out.append((u, um1))
        finally:
            st.stencil_destroy(plan)
    assert np.count_nonzero(out[0][0]) > 0
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
