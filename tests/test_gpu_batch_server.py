"""Batched shots (one grouped launch per step) and the continuous-batching
shot server: every shot's result is bit-identical to the same shot run alone
through stencil_run, and matches the FP64 oracle."""
import time

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


SHAPES = [(67, 45, 33), (96, 64, 40), (40, 40, 40), (130, 20, 51), (33, 97, 12), (64, 64, 64)]


def shot(i, shape, R=5, storage=0):
    nx, ny, nz = shape
    v = workloads.layered_velocity(nx, ny, nz, n_layers=4, seed=100 + i)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    src = (nx // 3, ny // 2, nz // 2)
    return v, dt, src


def alone(env, v, dt, src, steps, R=5, storage=0, absorb=(0, 0.0)):
    torch, st = env
    # the tiled kernel, as batches and the server run it
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, storage=storage, tile=(2, 64, 16, -1),
                                        absorb=absorb, stream=stream(torch)))
    try:
        out = np.empty_like(v)
        st.stencil_run(plan, steps, out)
    finally:
        st.stencil_destroy(plan)
    return out


@pytest.mark.parametrize("graph", [0, 6])
def test_batch_shots_equal_alone_runs(env, graph):
    torch, st = env
    shots = [shot(i, s) for i, s in enumerate(SHAPES)]
    descs = [st.make_desc(v, dt, radius=5, src=src, stream=stream(torch)) for v, dt, src in shots]
    batch = st.stencil_batch_create(descs, graph_steps=graph)
    try:
        assert st.stencil_batch_size(batch) == len(shots)
        st.stencil_batch_run(batch, 17)
        st.stencil_batch_run(batch, 13)
        st.stencil_batch_sync(batch)
        outs = []
        for i, (v, dt, src) in enumerate(shots):
            out = np.empty_like(v)
            plan = st.stencil_batch_plan(batch, i)
            st.stencil_get_field(plan, 0, out)
            assert st.stencil_get_stats(plan).steps_done == 30
            outs.append(out)
    finally:
        st.stencil_batch_destroy(batch)
    for (v, dt, src), out in zip(shots, outs):
        assert np.array_equal(out, alone(env, v, dt, src, 30))
        ref, _ = oracle.run(v, workloads.DX, dt, 5, 30, src=src)
        assert oracle.rel_l2(out, ref) <= 1e-5


def test_batch_16bit_equals_alone(env):
    torch, st = env
    shots = [shot(i, s) for i, s in enumerate(SHAPES[:3])]
    descs = [st.make_desc(v, dt, radius=4, src=src, storage=1, stream=stream(torch)) for v, dt, src in shots]
    batch = st.stencil_batch_create(descs, graph_steps=4)
    try:
        st.stencil_batch_run(batch, 22)
        outs = []
        for i, (v, dt, src) in enumerate(shots):
            out = np.empty_like(v)
            st.stencil_get_field(st.stencil_batch_plan(batch, i), 0, out)
            outs.append(out)
    finally:
        st.stencil_batch_destroy(batch)
    for (v, dt, src), out in zip(shots, outs):
        assert np.array_equal(out, alone(env, v, dt, src, 22, R=4, storage=1))


def test_batch_rejects_mixed_radius(env):
    torch, st = env
    (v, dt, src) = shot(0, SHAPES[0])
    d1 = st.make_desc(v, dt, radius=5, src=src)
    d2 = st.make_desc(v, dt, radius=4, src=src)
    with pytest.raises(st.StencilError) as ei:
        st.stencil_batch_create([d1, d2])
    assert ei.value.code == st.STENCIL_EINVAL


def make_server(st, **kw):
    cfg = st.shot_server_cfg_init()
    cfg.radius = kw.pop("radius", 5)
    for k, v in kw.items():
        setattr(cfg, k, v)
    return st.shot_server_create(cfg)


def test_server_results_identical_to_alone_and_mixed_arrivals(env):
    torch, st = env
    server = make_server(st, chunk_steps=7, max_slots=4)
    rng = np.random.default_rng(7)
    jobs = []
    try:
        for i, shape in enumerate(SHAPES + SHAPES[:2]):
            v, dt, src = shot(i, shape)
            steps = int(rng.integers(5, 40))
            out = np.full_like(v, np.nan)
            d = st.make_desc(v, dt, radius=5, src=src)
            t = st.shot_submit(server, d, steps, out)
            jobs.append((t, v, dt, src, steps, out))
            time.sleep(0.002 * (i % 3))            # arrivals while others run
        for t, *_ in jobs:
            assert st.shot_wait(server, t, 120.0) == st.SHOT_DONE
        stats = st.shot_server_get_stats(server)
        assert stats.done == len(jobs) and stats.failed == 0 and stats.running == 0
        for t, v, dt, src, steps, out in jobs:
            state, tm = st.shot_poll(server, t)
            assert state == st.SHOT_DONE and tm.steps_done == steps
            assert 0 <= tm.t_submit <= tm.t_admit <= tm.t_done
    finally:
        st.shot_server_destroy(server)
    for t, v, dt, src, steps, out in jobs:
        assert np.array_equal(out, alone(env, v, dt, src, steps)), t


def test_server_budget_queues_and_rejects(env):
    torch, st = env
    v, dt, src = shot(0, (64, 64, 64))
    one = 64 * 64 * 64 * 12 + 200_000
    server = make_server(st, hbm_budget_bytes=int(1.5 * one), chunk_steps=5)
    try:
        outs, tickets = [], []
        for _ in range(3):                          # only one fits at a time: the rest queue
            out = np.empty_like(v)
            tickets.append(st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src), 12, out))
            outs.append(out)
        big = workloads.constant_velocity(200, 200, 200, 2000.0)
        with pytest.raises(st.StencilError) as ei:
            st.shot_submit(server, st.make_desc(big, dt, radius=5), 3, np.empty_like(big))
        assert ei.value.code == st.STENCIL_EBUDGET
        for t in tickets:
            assert st.shot_wait(server, t, 60.0) == st.SHOT_DONE
        s = st.shot_server_get_stats(server)
        assert s.failed == 1 and s.done == 3 and s.bytes_in_use == 0
    finally:
        st.shot_server_destroy(server)
    ref = alone(env, v, dt, src, 12)
    for out in outs:
        assert np.array_equal(out, ref)


def test_server_unknown_ticket_and_cancel_on_destroy(env):
    torch, st = env
    server = make_server(st, chunk_steps=2, max_slots=1)
    v, dt, src = shot(1, (96, 64, 40))
    outs = [np.empty_like(v) for _ in range(4)]
    tickets = [st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src), 400, o) for o in outs]
    with pytest.raises(st.StencilError) as ei:
        st.shot_poll(server, 987654)
    assert ei.value.code == st.STENCIL_EUNKNOWN_TICKET
    st.shot_server_destroy(server)        # finishes the admitted shot, cancels the queued ones


def test_server_shot_with_invalid_model_fails_cleanly(env):
    torch, st = env
    server = make_server(st)
    try:
        v, dt, src = shot(2, (40, 40, 40))
        bad = v.copy()
        bad[3, 3, 3] = -1.0
        t = st.shot_submit(server, st.make_desc(bad, dt, radius=5, src=src), 10, np.empty_like(v))
        assert st.shot_wait(server, t, 30.0) == st.SHOT_FAILED
        state, tm = st.shot_poll(server, t)
        assert tm.status == st.STENCIL_EINVAL
        good = np.empty_like(v)
        t2 = st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src), 10, good)
        assert st.shot_wait(server, t2, 30.0) == st.SHOT_DONE
    finally:
        st.shot_server_destroy(server)
    assert np.array_equal(good, alone(env, v, dt, src, 10))


# one shape per size lane of a three-lane server: below 2^21 points, 2^21 ..
# 2^23, and above 2^23
LANE_SHAPES = [(64, 64, 40), (160, 128, 120), (256, 160, 208)]


@pytest.mark.parametrize("lanes", [1, 3])
def test_server_lanes_results_identical_to_alone(env, lanes):
    """Shots of all three size classes in the mix, arriving while others
    run: with the lanes stepped independently (or all in one lane) every
    result is bit-identical to the shot run alone."""
    torch, st = env
    server = make_server(st, chunk_steps=6, lanes=lanes)
    jobs = []
    try:
        for i, (shape, steps) in enumerate(zip(LANE_SHAPES * 2, (31, 17, 9, 12, 25, 4))):
            v, dt, src = shot(20 + i, shape)
            out = np.full_like(v, np.nan)
            t = st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src), steps, out)
            jobs.append((t, v, dt, src, steps, out))
            time.sleep(0.001 * (i % 2))
        for t, *_ in jobs:
            assert st.shot_wait(server, t, 120.0) == st.SHOT_DONE
        stats = st.shot_server_get_stats(server)
        assert stats.done == len(jobs) and stats.failed == 0 and stats.bytes_in_use == 0
        assert stats.iterations >= 1
    finally:
        st.shot_server_destroy(server)
    for t, v, dt, src, steps, out in jobs:
        assert np.array_equal(out, alone(env, v, dt, src, steps)), t


def test_server_on_callers_stream_and_bad_lane_count(env):
    torch, st = env
    with pytest.raises(st.StencilError) as ei:
        make_server(st, lanes=7)
    assert ei.value.code == st.STENCIL_EINVAL
    server = make_server(st, chunk_steps=4, cuda_stream=stream(torch))   # one lane, on the given stream
    try:
        v, dt, src = shot(30, (96, 64, 40))
        out = np.empty_like(v)
        t = st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src), 10, out)
        assert st.shot_wait(server, t, 60.0) == st.SHOT_DONE
    finally:
        st.shot_server_destroy(server)
    assert np.array_equal(out, alone(env, v, dt, src, 10))


def test_batch_and_server_with_absorbing_layers_equal_alone(env):
    """Shots with and without an absorbing layer in one batch (the grouped
    absorbing variant) and through the shot server: bit-identical to each
    shot alone, and the layer matches the FP64 oracle."""
    torch, st = env
    layers = [(6, 0.25), (0, 0.0), (9, 0.15), (4, 0.3)]
    shapes = [(67, 45, 33), (96, 64, 40), (40, 40, 40), (130, 20, 51)]
    shots = [shot(40 + i, s) for i, s in enumerate(shapes)]
    descs = [st.make_desc(v, dt, radius=5, src=src, absorb=a, stream=stream(torch))
             for (v, dt, src), a in zip(shots, layers)]
    b = st.stencil_batch_create(descs)
    try:
        st.stencil_batch_run(b, 37)
        st.stencil_batch_sync(b)
        outs = []
        for i, (v, dt, src) in enumerate(shots):
            out = np.empty_like(v)
            st.stencil_get_field(st.stencil_batch_plan(b, i), 0, out)
            outs.append(out)
    finally:
        st.stencil_batch_destroy(b)
    for (v, dt, src), a, out in zip(shots, layers, outs):
        assert np.array_equal(out, alone(env, v, dt, src, 37, absorb=a))
    v, dt, src = shots[0]
    ref, _, _ = oracle.run_ext(v, workloads.DX, dt, 5, 37, src=src, absorb=layers[0])
    assert oracle.rel_l2(outs[0], ref) <= 1e-5
    server = make_server(st, chunk_steps=5)
    jobs = []
    try:
        for (v, dt, src), a in zip(shots, layers):
            out = np.full_like(v, np.nan)
            jobs.append((st.shot_submit(server, st.make_desc(v, dt, radius=5, src=src, absorb=a), 23, out), out))
        for t, _ in jobs:
            assert st.shot_wait(server, t, 60.0) == st.SHOT_DONE
    finally:
        st.shot_server_destroy(server)
    for ((v, dt, src), a), (t, out) in zip(zip(shots, layers), jobs):
        assert np.array_equal(out, alone(env, v, dt, src, 23, absorb=a))


def test_served_migrations_equal_single_plan_migrations(env):
    """Reverse-time migrations through the shot server (forward with record
    and snapshots, then backward with the reversed traces injected and the
    imaging condition, in the lanes beside ordinary shots; snapshots fall in
    the middle of the lane's chunks): image and traces bit-identical to the
    single-plan migration (rtm.migrate) with the server's tile, and the
    ordinary shots to their alone runs."""
    torch, st = env
    from paper_1310_8232_gb300 import rtm
    jobs = [((48, 40, 36), 36, 6, 4, (6, 0.2)), ((56, 30, 44), 30, 5, 7, (0, 0.0)),
            ((70, 66, 40), 24, 4, 3, (5, 0.25))]
    server = make_server(st, chunk_steps=5)
    subs, plain = [], []
    try:
        for i, (shape, T, k, zr, ab) in enumerate(jobs):
            v, dt, src = shot(60 + i, shape)
            img = np.full_like(v, np.nan)
            tr = np.full((T, shape[1], shape[0]), np.nan, dtype=np.float32)
            t = st.shot_submit_rtm(server, st.make_desc(v, dt, radius=5, src=src, absorb=ab), T, zr, k, img, tr)
            subs.append((t, v, dt, src, T, k, zr, ab, img, tr))
            if i == 1:                                     # ordinary shots arriving in between
                for j, s in enumerate(SHAPES[:2]):
                    pv, pdt, psrc = shot(70 + j, s)
                    out = np.full_like(pv, np.nan)
                    plain.append((st.shot_submit(server, st.make_desc(pv, pdt, radius=5, src=psrc), 17, out),
                                  pv, pdt, psrc, out))
        for t, *_ in subs + plain:
            assert st.shot_wait(server, t, 120.0) == st.SHOT_DONE
        state, tm = st.shot_poll(server, subs[0][0])
        assert tm.steps_done == 2 * jobs[0][1]
    finally:
        st.shot_server_destroy(server)
    for t, v, dt, src, T, k, zr, ab, img, tr in subs:
        want_img, want_tr = rtm.migrate(torch, torch.from_numpy(v).cuda(), dt, T, src, zr, k, radius=5,
                                        dx=workloads.DX, absorb=ab, tile=(2, 64, 16, -1))
        assert np.array_equal(tr, want_tr.cpu().numpy())
        assert np.array_equal(img, want_img.cpu().numpy())
        assert np.any(img != 0)
    for t, pv, pdt, psrc, out in plain:
        assert np.array_equal(out, alone(env, pv, pdt, psrc, 17))


def test_served_migration_refusals(env):
    torch, st = env
    v, dt, src = shot(80, (40, 40, 40))
    img = np.zeros_like(v)
    server = make_server(st)
    try:
        for T, k, zr in ((30, 7, 4), (0, 5, 4), (30, 5, 40), (30, 0, 4)):
            with pytest.raises(st.StencilError) as ei:
                st.shot_submit_rtm(server, st.make_desc(v, dt, radius=5, src=src), T, zr, k, img)
            assert ei.value.code == st.STENCIL_EINVAL
    finally:
        st.shot_server_destroy(server)
    cfg = st.shot_server_cfg_init()
    cfg.storage = 1
    half = st.shot_server_create(cfg)
    try:
        with pytest.raises(st.StencilError) as ei:
            st.shot_submit_rtm(half, st.make_desc(v, dt, radius=5, src=src), 30, 4, 5, img)
        assert ei.value.code == st.STENCIL_EUNSUPPORTED
    finally:
        st.shot_server_destroy(half)


def test_server_reads_a_page_locked_model_in_place(env):
    """A page-locked host velocity is read at admission (not copied at
    submit): the result is the shot's alone run."""
    torch, st = env
    v, dt, src = shot(90, (67, 45, 33))
    pinned = torch.from_numpy(v).pin_memory()
    server = make_server(st)
    out = np.full_like(v, np.nan)
    try:
        t = st.shot_submit(server, st.make_desc(pinned, dt, radius=5, src=src), 19, out)
        assert st.shot_wait(server, t, 60.0) == st.SHOT_DONE
    finally:
        st.shot_server_destroy(server)
    assert np.array_equal(out, alone(env, v, dt, src, 19))
