"""The paper's method on the host cores (oracle/host_method.c), a CPU
baseline: the FP32 blocked sweep against the FP64 oracle, blocked = unblocked
bit for bit, and the MWMB selection against oracle/selection.py on the time
table it measured."""
import numpy as np
import pytest

import oracle
from oracle import host_method as hm
from oracle import selection
from paper_1310_8232_gb300 import workloads


def setup(nx, ny, nz, R, seed=11):
    v = workloads.layered_velocity(nx, ny, nz, seed=seed)
    dt = workloads.time_step(oracle.cfl_limit(R), workloads.DX, float(v.max()))
    return v, dt


@pytest.mark.parametrize("R", [4, 5])
def test_fp32_blocked_sweep_matches_oracle(R):
    nx, ny, nz, steps = 26, 21, 19, 14
    v, dt = setup(nx, ny, nz, R)
    src = (nx // 2, ny // 3, nz // 2)
    u = np.zeros((nz, ny, nx), np.float32)
    up = np.zeros_like(u)
    scale = float(v[src[2], src[1], src[0]]) ** 2 * dt * dt
    hm.run(hm.kappa(v, workloads.DX, dt), R, steps, u, up, src=src, src_scale=scale, dt=dt, block=(7, 5, 4))
    ref, ref_prev = oracle.run(v, workloads.DX, dt, R, steps, src=src)
    assert oracle.rel_l2(u, ref) <= 1e-5
    assert oracle.rel_l2(up, ref_prev) <= 1e-5


def test_blocked_equals_unblocked_bit_for_bit():
    nx, ny, nz, R = 30, 17, 23, 5
    v, dt = setup(nx, ny, nz, R, seed=12)
    kap = hm.kappa(v, workloads.DX, dt)
    u0 = workloads.random_field(nx, ny, nz, seed=1)
    um1 = workloads.random_field(nx, ny, nz, seed=2)
    outs = []
    for block in ((0, 0, 0), (1, 1, 1), (15, 15, 143), (7, 5, 3), (30, 2, 23)):
        u, up = u0.copy(), um1.copy()
        hm.run(kap, R, 5, u, up, src=(3, 4, 5), src_scale=1e-3, dt=dt, n0=7, block=block)
        outs.append((u, up))
    for u, up in outs[1:]:
        assert np.array_equal(u, outs[0][0]) and np.array_equal(up, outs[0][1])


def test_candidates_follow_the_paper_example():
    """Sec. 3.7's worked example: S = 200, P = 5 -> 1, 51, 101, 151, 200."""
    assert hm.candidates_1d(200, 5) == [1, 51, 101, 151, 200] == selection.candidates_1d(200, 5)
    for S, P in ((800, 5), (37, 3), (5, 10), (1, 2), (64, 20)):
        assert hm.candidates_1d(S, P) == selection.candidates_1d(S, P)


def test_mwmb_on_host_cores_picks_what_the_stages_say():
    """The block the C selection returns is the one oracle/selection.py's
    three stages (MWMB: stage 2 = max) pick on the same measured table."""
    nx, ny, nz, R = 40, 36, 32, 4
    v, dt = setup(nx, ny, nz, R, seed=13)
    res = hm.select_mwmb(hm.kappa(v, workloads.DX, dt), R, P=3, nI=1, nthreads=4)
    T, nzs = res["cores"], res["slab"]
    ci, cj, ck = (selection.candidates_1d(S, 3) for S in (nx, ny, nzs))
    cands = [(a, b, c) for a in ci for b in cj for c in ck]
    assert res["candidates"] == len(cands) == res["times"].shape[1] and T == 4
    node, c, t = selection.three_stage([res["times"].tolist()], selection.TARGET_OF["MWMB"])
    assert node == 0 and cands[c] == res["block"] and t == res["min_time"]
    assert res["actual_time"] > 0 and np.isfinite(res["quality"])
