"""Replicas across GPUs: one process per GPU, independent shots, no exchange.

A shot does not shard: its time steps are sequential and one grid fits a
GB300's HBM many times over, while splitting a grid over GPUs would add a
halo exchange per time step that the method (Sec. 2, 2.5D blocking within
one memory hierarchy) does not have.  Several GPUs therefore run independent
shots ("replicas only"): the units of work (shots) are split over the ranks
in contiguous balanced ranges, each rank sweeps its own with no data-path
collective, and the only communication is a barrier around the timed region
and a max (or sum) over ranks of a scalar.

Launch: one process per GPU (`torchrun --nproc-per-node N`), RANK,
WORLD_SIZE and LOCAL_RANK from the environment.  The process group is NCCL
for device tensors on GPUs and gloo for CPU tensors (tests); with one
process no group is created.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    rank: int
    world: int
    local: int


def rank_env() -> RankEnv:
    """RANK / WORLD_SIZE / LOCAL_RANK as set by torchrun (defaults 0 / 1 / 0)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank environment: RANK={rank} WORLD_SIZE={world}")
    return RankEnv(rank, world, local)


def shard_range(n_units: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous range [lo, hi) of the n_units owned by `rank`: the first
    n_units % world ranks take one unit more, so sizes differ by at most one
    and the ranges tile [0, n_units) in rank order."""
    if n_units < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("shard_range: need n_units >= 0, world >= 1, 0 <= rank < world")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class Ranks:
    """The process group of a replica run, or a stand-in for one process.

    `barrier()` also synchronises the current CUDA device when `cuda` is
    set, so a timed region bracketed by barriers starts and ends with every
    rank's device idle; `max()` and `sum()` reduce one float over ranks."""

    def __init__(self, env: RankEnv | None = None, backend: str | None = None, cuda: bool = True):
        import torch
        self.torch = torch
        self.env = env or rank_env()
        self.cuda = cuda
        self.dist = None
        if self.env.world > 1:
            import torch.distributed as dist
            backend = backend or ("nccl" if cuda else "gloo")
            if not dist.is_initialized():
                kw = {}
                if backend == "nccl":
                    kw["device_id"] = torch.device("cuda", self.env.local)
                dist.init_process_group(backend, rank=self.env.rank, world_size=self.env.world, **kw)
            self.dist = dist
        self.device = torch.device("cuda", self.env.local) if cuda else torch.device("cpu")

    @property
    def is_root(self) -> bool:
        return self.env.rank == 0

    def shard(self, n_units: int) -> tuple[int, int]:
        return shard_range(n_units, self.env.world, self.env.rank)

    def barrier(self) -> None:
        if self.dist:
            self.dist.barrier()
        if self.cuda:
            self.torch.cuda.synchronize()

    def _reduce(self, x: float, op) -> float:
        if not self.dist:
            return float(x)
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)

    def gather(self, obj) -> list:
        """Every rank's `obj` (picklable), in rank order, on every rank."""
        if not self.dist:
            return [obj]
        out = [None] * self.env.world
        self.dist.all_gather_object(out, obj)
        return out

    def close(self) -> None:
        if self.dist and self.dist.is_initialized():
            self.dist.destroy_process_group()
        self.dist = None
