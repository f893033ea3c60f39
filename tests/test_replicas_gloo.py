"""The multi-GPU path is replicas only: shots are split over ranks with no
data-path collective, and ranks meet only at a barrier and a max/sum of the
timed region.  This host logic runs here as two gloo ranks on the CPU, with
the FP64 oracle standing in for each rank's sweeps."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1310_8232_gb300.replicas import RankEnv, rank_env, shard_range

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n_units", [0, 1, 2, 5, 7, 64, 65])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_ranges_tile_the_units(n_units, world):
    ranges = [shard_range(n_units, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n_units
    for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
        assert hi == lo2
    sizes = [hi - lo for lo, hi in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)


def test_shard_and_env_reject_bad_arguments(monkeypatch):
    for bad in ((-1, 2, 0), (4, 0, 0), (4, 2, 2), (4, 2, -1)):
        with pytest.raises(ValueError):
            shard_range(*bad)
    monkeypatch.setenv("RANK", "2")
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(ValueError):
        rank_env()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.delenv("LOCAL_RANK", raising=False)
    assert rank_env() == RankEnv(1, 2, 1)


SHOTS = [(12, 10, 9), (9, 9, 9), (14, 8, 11), (10, 13, 8), (11, 11, 12)]


def tiny_shot(i, shape):
    from paper_1310_8232_gb300 import workloads
    import oracle
    nx, ny, nz = shape
    v = workloads.layered_velocity(nx, ny, nz, n_layers=3, seed=40 + i).astype(np.float64)
    dt = workloads.time_step(oracle.cfl_limit(4), workloads.DX, float(v.max()))
    u, _ = oracle.run(v, workloads.DX, dt, 4, 6, src=(nx // 2, ny // 2, nz // 2), nthreads=1)
    return u


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_1310_8232_gb300.replicas import Ranks
    ranks = Ranks(backend="gloo", cuda=False)
    try:
        lo, hi = ranks.shard(len(SHOTS))
        ranks.barrier()
        mine = {i: tiny_shot(i, SHOTS[i]) for i in range(lo, hi)}
        ranks.barrier()
        pooled = ranks.gather(mine)
        assert ranks.max(rank + 1.5) == world + 0.5
        assert ranks.sum(rank + 1.5) == sum(r + 1.5 for r in range(world))
        owners = [set(part) for part in pooled]
        assert set().union(*owners) == set(range(len(SHOTS)))
        assert sum(len(o) for o in owners) == len(SHOTS)
        if ranks.is_root:
            merged = {}
            for part in pooled:
                merged.update(part)
            np.savez(os.path.join(out_dir, "pooled.npz"), **{str(k): v for k, v in merged.items()})
    finally:
        ranks.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_cover_all_shots_once(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    pooled = np.load(tmp_path / "pooled.npz")
    assert sorted(int(k) for k in pooled.files) == list(range(len(SHOTS)))
    for i, shape in enumerate(SHOTS):
        # each rank's result is the shot run alone, bit for bit
        assert np.array_equal(pooled[str(i)], tiny_shot(i, shape))


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
