"""The batch and serving workloads at their full sizes.

- 64 uneven shots (each dim in {96, ..., 320}, seed 4064), 100 steps, one
  grouped launch per step: 8 sampled shots against the FP64 oracle
  (relative L2 <= 1e-5) and against the same shot run alone (bit for bit).
- The serving workload's first 16 arrivals (cube side 64-400, 50-500 steps,
  seed 5020), submitted together to the shot server: each result bit for
  bit equal to the shot run alone.
"""
import numpy as np
import pytest

import oracle
from paper_1310_8232_gb300 import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def alone(st, torch, v, dt, R, steps, src=None):
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, graph_steps=20, tile=(2, 64, 16, -1),
                                        stream=torch.cuda.current_stream().cuda_stream))
    try:
        out = np.empty(v.shape, dtype=np.float32)
        st.stencil_run(plan, steps, out)
    finally:
        st.stencil_destroy(plan)
    return out


def test_batch_of_64_shots_sampled_against_oracle(env):
    torch, st = env
    R, T = 5, 100
    dims = workloads.batch_dims(64)
    seeds = workloads.batch_layer_seeds(64)
    vels, dts, descs = [], [], []
    s = torch.cuda.current_stream().cuda_stream
    for (nx, ny, nz), sd in zip(dims, seeds):
        v = workloads.layered_velocity(nx, ny, nz, seed=sd)
        dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
        vels.append(v)
        dts.append(dt)
        descs.append(st.make_desc(v, dt, radius=R, dx=workloads.DX, graph_steps=20, stream=s))
    batch = st.stencil_batch_create(descs, graph_steps=20)
    sample = sorted(np.random.default_rng(64).choice(64, size=8, replace=False).tolist())
    outs = {}
    try:
        st.stencil_batch_run(batch, T)
        st.stencil_batch_sync(batch)
        for i in sample:
            out = np.empty(vels[i].shape, dtype=np.float32)
            st.stencil_get_field(st.stencil_batch_plan(batch, i), 0, out)
            outs[i] = out
    finally:
        st.stencil_batch_destroy(batch)
    for i in sample:
        v, dt = vels[i], dts[i]
        assert np.array_equal(outs[i], alone(st, torch, v, dt, R, T)), i
        ref, _ = oracle.run(v, workloads.DX, dt, R, T)
        err = oracle.rel_l2(outs[i], ref)
        assert err <= 1e-5, (i, dims[i], err)


def test_server_first_16_arrivals_equal_alone_runs(env):
    torch, st = env
    R = 5
    arrivals = workloads.poisson_arrivals(20.0, 60.0)[:16]
    cfg = st.shot_server_cfg_init()
    cfg.radius = R
    cfg.chunk_steps = 20
    server = st.shot_server_create(cfg)
    jobs = []
    try:
        for a in arrivals:
            n = a["side"]
            v = workloads.layered_velocity(n, n, n, seed=a["seed"] % (2 ** 31))
            dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(v.max()))
            out = np.full(v.shape, np.nan, dtype=np.float32)
            t = st.shot_submit(server, st.make_desc(v, dt, radius=R, dx=workloads.DX), a["steps"], out)
            jobs.append((t, v, dt, a["steps"], out))
        for t, *_ in jobs:
            assert st.shot_wait(server, t, 600.0) == st.SHOT_DONE
    finally:
        st.shot_server_destroy(server)
    for t, v, dt, steps, out in jobs:
        assert np.array_equal(out, alone(st, torch, v, dt, R, steps)), (t, v.shape, steps)
