"""The paper's blocksize-selection methodology, plain Python -- TEST INFRASTRUCTURE ONLY.

Written from Sec. 3.2 (two-phase profiling: selection gives MinTime,
verification gives ActualTime), Sec. 3.3 (OB and the three-stage
contention-aware selection with stage-2 target min / max / avg = MMMB / MWMB /
MAMB, Eqs. 1-3), Sec. 3.6 (quality metric MinTime vs ActualTime) and Sec. 3.7
(candidate generation with P parts per axis).

Readings where the paper is garbled or silent:
  * candidate list: b_l[0] = 1 and b_l[m] = min(S, floor(m*S/(P-1)) + 1) for
    m >= 1.  The printed formula ends at (P-1)S/(P-1)+1 = S+1, but the worked
    example for S = 200, P = 5 lists 200 as the last value, so the top value is
    clamped to S.  Duplicates (small S) are dropped, order kept.
  * Eq. 3 (MAMB) divides a sum over j = 1..i by the node index i; read as: the
    core of node i whose best time is closest to the mean of the best times of
    the cores of node i.
  * Stage 3: b_best is the stage-2 block of the node whose recorded stage-2
    time is smallest.
  * Ties (equal times) go to the lowest index: lowest candidate index in
    stage 1, lowest core index in stage 2, lowest node index in stage 3.
"""
from __future__ import annotations

import math


def candidates_1d(S: int, P: int) -> list[int]:
    """Values of one block axis of extent S split into P parts (Sec. 3.7)."""
    if S < 1 or P < 2:
        raise ValueError("need S >= 1 and P >= 2")
    out = [1]
    for m in range(1, P):
        b = min(S, (m * S) // (P - 1) + 1)
        if b not in out:
            out.append(b)
    return out


def candidates(extents, P: int) -> list[tuple[int, ...]]:
    """Cartesian product of candidates_1d over the axes, first axis slowest."""
    axes = [candidates_1d(S, P) for S in extents]
    combos = [()]
    for ax in axes:
        combos = [c + (b,) for c in combos for b in ax]
    return combos


def _argmin(xs):
    best = 0
    for i, x in enumerate(xs):
        if x < xs[best]:
            best = i
    return best


def _argmax(xs):
    best = 0
    for i, x in enumerate(xs):
        if x > xs[best]:
            best = i
    return best


def stage1(times_core):
    """Stage 1: a core's best candidate.  times_core[c] = t(b_c, P_k,i)."""
    c = _argmin(times_core)
    return c, times_core[c]


def stage2(best_times, target: str) -> int:
    """Stage 2 over the cores of one node (Eqs. 1-3); returns the chosen core."""
    if target == "min":
        return _argmin(best_times)
    if target == "max":
        return _argmax(best_times)
    if target == "avg":
        mean = sum(best_times) / len(best_times)
        return _argmin([abs(t - mean) for t in best_times])
    raise ValueError(target)


def three_stage(times, target: str):
    """Contention-aware selection (Sec. 3.3).

    times[i][k][c] = time of node i's c-th candidate on core k of node i (all
    cores of a node run the same candidates in the same order).  Returns
    (node i*, candidate index c* within node i*'s list, its stage-2 time).
    """
    per_node = []
    for node in times:
        s1 = [stage1(core) for core in node]              # (cand, time) per core
        k = stage2([t for _, t in s1], target)
        per_node.append((s1[k][0], s1[k][1]))
    i = _argmin([t for _, t in per_node])
    return i, per_node[i][0], per_node[i][1]


def original_block(times_per_process):
    """OB (Sec. 3.3): each process times its own distinct candidates; global min.

    times_per_process[p][c] = time of process p's c-th candidate.  Returns
    (p*, c*, time).
    """
    best = None
    for p, ts in enumerate(times_per_process):
        for c, t in enumerate(ts):
            if best is None or t < best[2]:
                best = (p, c, t)
    return best


TARGET_OF = {"MMMB": "min", "MWMB": "max", "MAMB": "avg"}


def quality(min_time: float, actual_time: float) -> float:
    """(ActualTime - MinTime) / MinTime, the blocksize quality metric (Sec. 3.6)."""
    if min_time <= 0 or not math.isfinite(min_time):
        raise ValueError("MinTime must be positive")
    return (actual_time - min_time) / min_time
