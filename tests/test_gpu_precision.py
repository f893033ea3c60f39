"""Reduced-precision storage (FP16 / BF16 u^n and d^n = u^n - u^{n-1}, one
power-of-two scale per z plane and time level, FP32 arithmetic) against the
FP64 oracle.

Bars: FP32 storage relative L2 <= 1e-5 after 100 steps; reduced-precision
storage <= 5e-3.  FP16 meets 5e-3 at steps 50, 100 and 200 of the 512^3
layered shot.  BF16's 8-bit significand cannot: each step rounds u once, and
those roundings add up like a random walk whatever the encoding of the step's
change; BF16 is held to that derived bound (``rw_bound``)."""
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


def stream(torch):
    return torch.cuda.current_stream().cuda_stream


def rw_bound(steps: int, mant_bits: int) -> float:
    """Relative L2 error the difference form can reach after ``steps`` steps.

    One round-to-nearest to ``mant_bits`` explicit significand bits has a
    relative L2 error sigma = 2^-p / sqrt(12 E[m^2]) over significands m
    log-uniform on [1, 2) (E[m^2] = 3 / (2 ln 2)).  Each step rounds u^{n+1}
    and d^{n+1} once; a rounding of u is a displacement error that the
    (energy-conserving) scheme carries without amplification, a rounding of d
    a velocity error of the size of d's own rounding.  n steps of independent
    roundings of the two add up to at most sqrt(2 n) sigma."""
    sigma = 2.0 ** -mant_bits / math.sqrt(12.0 * 1.5 / math.log(2.0))
    return math.sqrt(2.0 * steps) * sigma


FP16_BITS, BF16_BITS = 10, 7


@pytest.mark.parametrize("storage,eps", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_set_get_roundtrip(env, storage, eps):
    """u^n comes back after one rounding; u^{n-1} = u^n - d^n after two (u^n
    and d^n = 0.5 u^n, each within half an ulp): 3 eps relative."""
    torch, st = env
    nx, ny, nz = 70, 33, 21
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    u = workloads.random_field(nx, ny, nz, seed=5)
    u[3] *= 1e-6                          # planes of very different magnitude
    u[7] *= 1e5
    plan = st.stencil_plan(st.make_desc(v, 1e-3, radius=5, storage=storage, stream=stream(torch)))
    try:
        st.stencil_set_fields(plan, u, u * 0.5, step=3)
        got = np.empty_like(u)
        st.stencil_get_field(plan, 0, got)
        prev = np.empty_like(u)
        st.stencil_get_field(plan, 1, prev)
    finally:
        st.stencil_destroy(plan)
    rel = np.abs(got - u) / np.abs(u)
    assert np.max(rel) <= eps * (1 + 1e-6)
    assert np.max(np.abs(prev - u * 0.5) / np.abs(u * 0.5)) <= 3 * eps * (1 + 1e-6)


@pytest.mark.parametrize("storage", [1, 2])
def test_small_grid_matches_oracle_and_tiles(env, storage):
    """Ragged grid, several tiles and z-chunks: same answer within the
    storage's rounding, and the tiles agree with one another closely."""
    torch, st = env
    nx, ny, nz, R = 67, 45, 33, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=21)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    ref, _ = oracle.run(v, workloads.DX, dt, R, 30, src=(5, 40, 30))
    outs = []
    for tile in (None, (2, 64, 8, 7), (2, 32, 32, 16), (2, 128, 16, 5)):
        if tile and st.stencil_tile_info(R, tile[1], tile[2], storage) is None:
            continue
        plan = st.stencil_plan(st.make_desc(v, dt, radius=R, storage=storage, tile=tile, src=(5, 40, 30),
                                            stream=stream(torch)))
        try:
            out = np.empty_like(v)
            st.stencil_run(plan, 30, out)
        finally:
            st.stencil_destroy(plan)
        outs.append(out)
        assert np.all(np.isfinite(out))
        assert oracle.rel_l2(out, ref) <= (5e-3 if storage == 1 else rw_bound(30, BF16_BITS))
    assert len(outs) >= 3


@pytest.mark.parametrize("storage", [1, 2])
def test_graph_replay_equals_eager_16bit(env, storage):
    torch, st = env
    n, R = 40, 4
    v = workloads.layered_velocity(n, n, n, seed=9)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    res = []
    for g in (0, 6):
        plan = st.stencil_plan(st.make_desc(v, dt, radius=R, storage=storage, graph_steps=g, stream=stream(torch)))
        try:
            out = np.empty_like(v)
            st.stencil_run(plan, 25, out)
        finally:
            st.stencil_destroy(plan)
        res.append(out)
    assert np.array_equal(res[0], res[1])


def test_512_layered_shot_errors_at_50_100_200_steps(env):
    """The 512^3 layered model, R = 5, 200 steps, FP32 / FP16 / BF16 storage,
    relative L2 against the FP64 oracle at steps 50, 100 and 200."""
    torch, st = env
    n, R = 512, 5
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    marks = (50, 100, 200)
    refs = {}
    u = up = None
    done = 0
    for s in marks:
        u, up = oracle.run(v, workloads.DX, dt, R, s - done, u0=u, um1=up, n0=done)
        refs[s] = u
        done = s
    del u, up
    dv = torch.from_numpy(v).cuda()
    table = {}
    for name, storage in (("fp32", 0), ("fp16", 1), ("bf16", 2)):
        plan = st.stencil_plan(st.make_desc(dv, dt, radius=R, storage=storage, graph_steps=10,
                                            stream=stream(torch)))
        errs = {}
        try:
            done = 0
            for s in marks:
                st.stencil_step(plan, s - done)
                done = s
                errs[s] = st.stencil_rel_l2(plan, torch.from_numpy(refs[s]).cuda())
        finally:
            st.stencil_destroy(plan)
        table[name] = errs
    print("\nrelative L2 vs FP64 oracle, 512^3 layered, R=5:")
    for name, errs in table.items():
        print(f"  {name}: " + ", ".join(f"step {s}: {e:.3e}" for s, e in errs.items()))
    assert table["fp32"][100] <= 1e-5
    assert table["fp32"][50] <= 1e-5 and table["fp32"][200] <= 2e-5
    for s in marks:
        assert table["fp16"][s] <= min(5e-3, rw_bound(s, FP16_BITS)), (s, table["fp16"][s])
        assert table["bf16"][s] <= rw_bound(s, BF16_BITS), (s, table["bf16"][s])


def test_256_layered_shot_radius_4_errors(env):
    """The 8th-order stencil with 16-bit storage: 256^3 layered model, 100
    steps, relative L2 against the FP64 oracle."""
    torch, st = env
    n, R, T = 256, 4, 100
    v = workloads.layered_velocity(n, n, n, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
    ref, _ = oracle.run(v, workloads.DX, dt, R, T)
    dv = torch.from_numpy(v).cuda()
    dref = torch.from_numpy(ref).cuda()
    errs = {}
    for name, storage in (("fp32", 0), ("fp16", 1), ("bf16", 2)):
        plan = st.stencil_plan(st.make_desc(dv, dt, radius=R, storage=storage, graph_steps=10,
                                            stream=stream(torch)))
        try:
            st.stencil_step(plan, T)
            errs[name] = st.stencil_rel_l2(plan, dref)
        finally:
            st.stencil_destroy(plan)
    print(f"\nrelative L2 vs FP64 oracle, 256^3 layered, R=4, 100 steps: {errs}")
    assert errs["fp32"] <= 1e-5
    assert errs["fp16"] <= min(5e-3, rw_bound(T, FP16_BITS))
    assert errs["bf16"] <= rw_bound(T, BF16_BITS)


@pytest.mark.parametrize("storage", [1, 2])
def test_energy_with_16bit_storage(env, storage):
    """The fused energy sum with 16-bit storage against the oracle's energy of
    the stored (rounded) state: u^{n+1} and u^n = u^{n+1} - d^{n+1} as read
    back; equal within the storage's rounding."""
    torch, st = env
    nx, ny, nz, R = 48, 40, 36, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=81)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    u0 = workloads.gaussian_bump(nx, ny, nz, width=3.0)
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, amp=0.0, storage=storage, stream=stream(torch)))
    steps = 10
    try:
        st.stencil_set_fields(plan, u0, u0, 0)
        st.stencil_record_start(plan, energy=True, capacity=steps)
        want = []
        for _ in range(steps):
            st.stencil_step(plan, 1)
            u = np.empty_like(v)
            prev = np.empty_like(v)
            st.stencil_get_field(plan, 0, u)
            st.stencil_get_field(plan, 1, prev)
            want.append(oracle.energy(v, workloads.DX, dt, R, u, prev))
        got = np.empty(steps)
        assert st.stencil_record_read(plan, energy=got) == steps
    finally:
        st.stencil_destroy(plan)
    want = np.array(want)
    tol = 2.0 ** -9 if storage == 1 else 2.0 ** -6
    assert np.all(np.abs(got - want) <= tol * np.abs(want)), np.max(np.abs(got - want) / np.abs(want))
