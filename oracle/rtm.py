"""Reverse-time migration of one shot with the FP64 oracle.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the reference the
GPU migration is checked against.  The paper's kernel is the "3D model"
step of an RTM code (Sec. 2, Algorithm 1); the paper does not spell out the
migration around it, so this follows the textbook zero-lag
cross-correlation scheme, in the same steps and time pairing as the GPU
workflow (readings in the design notes):

1. forward: from u^0 = u^{-1} = 0, T steps with the point source and the
   absorbing layer; after step n (producing u^{n+1}) record the receiver
   plane, d[n] = u^{n+1}|_{z = z_r}; keep the snapshots S(t) = u^t for
   t = k, 2k, ..., T;
2. backward: from r^0 = r^{-1} = 0, no point source, the same absorbing
   layer; backward step m injects d[T-1-m] on the receiver plane (the
   traces reversed in time), so r^j (j steps done) belongs to forward time
   T + 1 - j;
3. image: I = sum over t = k, 2k, ..., T of S(t) * r^{T+1-t}.
"""
from __future__ import annotations

import numpy as np

from . import run_ext


def migrate(v, dx: float, dt: float, R: int, steps: int, src, receiver_z: int, snap_every: int,
            absorb=(0, 0.0), f: float = 15.0, t0: float | None = None, amp: float = 1.0):
    """Image, traces and snapshots of one shot (all FP64)."""
    T, k = int(steps), int(snap_every)
    if T < 1 or k < 1 or T % k:
        raise ValueError("steps must be a positive multiple of snap_every")
    v = np.ascontiguousarray(v, dtype=np.float64)
    # 1. forward, k steps at a time
    u = um1 = None
    traces, snaps = [], {}
    for n0 in range(0, T, k):
        u, um1, tr = run_ext(v, dx, dt, R, k, src=src, f=f, t0=t0, amp=amp, u0=u, um1=um1, n0=n0,
                             absorb=absorb, record=(receiver_z, -1))
        traces.append(tr)
        snaps[n0 + k] = u.copy()
    d = np.concatenate(traces)                       # (T, ny, nx)
    # 2./3. backward; stop at j = T + 1 - t for every snapshot time t
    stops = sorted(T + 1 - t for t in snaps)         # 1, k+1, ..., T+1-k
    image = np.zeros_like(v)
    r = rm1 = None
    j = 0
    for stop in stops:
        c = stop - j                                 # backward steps j .. stop-1 inject d[T-1-j] ...
        chunk = d[T - stop: T - j]                   # ascending time, read reversed
        r, rm1, _ = run_ext(v, dx, dt, R, c, amp=0.0, u0=r, um1=rm1, absorb=absorb,
                            inject=(receiver_z, -1, chunk, True, 1.0))
        j = stop
        image += snaps[T + 1 - j] * r
    return image, d, snaps
