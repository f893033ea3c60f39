"""Independent plans driven from concurrent host threads, each on its own
stream (a caller overlapping one shot's host copies with another's sweeps):
every shot's result is the same to the bit as when the shots run one after
another, and an error in one plan stays with that plan."""
import threading

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
    return torch, st


def shot(st, plan, v, T, out):
    st.stencil_set_velocity(plan, v)
    st.stencil_set_fields(plan, None, None, 0)
    st.stencil_run(plan, T, out)


@pytest.mark.parametrize("tile", [None, (2, 64, 16, -1), (3, 0, 0, -1)])
def test_two_plans_on_two_threads_equal_their_sequential_runs(env, tile):
    torch, st = env
    nx, ny, nz, R, T = 96, 80, 72, 5, 30
    models = [workloads.layered_velocity(nx, ny, nz, seed=s) for s in (1, 2, 3, 4)]
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(max(m.max() for m in models)))
    hv = [torch.from_numpy(m).pin_memory() for m in models]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = [st.stencil_plan(st.make_desc(models[0], dt, radius=R, tile=tile, graph_steps=10,
                                          stream=s.cuda_stream)) for s in streams]
    try:
        want = []
        for m in hv:                                    # one after another on plan 0
            out = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
            shot(st, plans[0], m, T, out)
            want.append(out.numpy().copy())
        got = [torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory() for _ in hv]
        errors = []

        def worker(k):
            try:
                for i in (k, k + 2):                    # plan k takes models k and k + 2
                    shot(st, plans[k], hv[i], T, got[i])
            except Exception as ex:
                errors.append(ex)

        threads = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for i in range(4):
            assert np.count_nonzero(want[i]) > 0
            assert np.array_equal(got[i].numpy(), want[i]), i
    finally:
        for p in plans:
            st.stencil_destroy(p)


def test_an_error_stays_with_its_plan(env):
    """A wait made to run out in one plan (the debug hook) is reported by that
    plan only; the other plan, driven at the same time, completes normally."""
    torch, st = env
    n, R, T = 64, 5, 12
    v = workloads.layered_velocity(n, n, n, seed=61)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    tile = (2, 64, 16, -1)
    plans = [st.stencil_plan(st.make_desc(v, dt, radius=R, tile=tile, stream=s.cuda_stream)) for s in streams]
    try:
        st.stencil_debug_wait_fault(plans[0], True, 20_000_000)      # 20 ms limit in plan 0 only
        results = {}

        def run(k):
            try:
                out = np.empty_like(v)
                st.stencil_run(plans[k], T, out)
                results[k] = out
            except st.StencilError as ex:
                results[k] = ex

        threads = [threading.Thread(target=run, args=(k,)) for k in (0, 1)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert isinstance(results[0], st.StencilError) and results[0].code == st.STENCIL_ETIMEOUT
        ref, _ = oracle.run(v, workloads.DX, dt, R, T)
        assert oracle.rel_l2(results[1], ref) <= 1e-5
    finally:
        for p in plans:
            st.stencil_destroy(p)
