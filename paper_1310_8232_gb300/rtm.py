"""Reverse-time migration of a shot through the C-ABI.

The paper's kernel is the "3D model" step of an RTM code (Sec. 2,
Algorithm 1).  This workflow runs the migration around it on the GPU with
the library's own calls; every step of the arithmetic happens in the
library's kernels:

1. forward plan (point source, absorbing layer): T sweeps recording the
   receiver plane z_r after every step (`stencil_record_*`, traces stay on
   the device) and copying the source wavefield u^t into device snapshots at
   t = k, 2k, ..., T (`stencil_get_field`, device to device);
2. backward plan (no point source, same layer): the traces injected on the
   receiver plane in reverse time order (`stencil_inject_start`, reverse),
   so the field after j backward steps belongs to forward time T + 1 - j;
3. the imaging condition I += S(t) * r^{T+1-t} at each snapshot time
   (`stencil_image_accumulate`, zero-lag cross-correlation).

Snapshots are kept in HBM: T/k fields of nx*ny*nz FP32.
"""
from __future__ import annotations

from . import binding as st


def migrate(torch, velocity, dt: float, steps: int, src, receiver_z: int, snap_every: int,
            radius: int = 5, dx: float = 10.0, absorb=(0, 0.0), f: float = 15.0, tile=None,
            graph_steps: int = 0, stream=None):
    """Returns (image, traces) as CUDA float32 tensors, shapes (nz, ny, nx)
    and (steps, ny, nx).  ``velocity``: CUDA float32 tensor (nz, ny, nx)."""
    T, k = int(steps), int(snap_every)
    if T < 1 or k < 1 or T % k:
        raise ValueError("steps must be a positive multiple of snap_every")
    nz, ny, nx = (int(s) for s in velocity.shape)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    common = dict(radius=radius, dx=dx, absorb=absorb, f=f, tile=tile, graph_steps=graph_steps, stream=s)
    fwd = st.stencil_plan(st.make_desc(velocity, dt, src=src, **common))
    traces = torch.empty((T, ny, nx), dtype=torch.float32, device=velocity.device)
    snaps = {}
    try:
        st.stencil_record_start(fwd, receiver_z=receiver_z, capacity=T)
        for n0 in range(0, T, k):
            st.stencil_step(fwd, k)
            snap = torch.empty((nz, ny, nx), dtype=torch.float32, device=velocity.device)
            st.stencil_get_field(fwd, 0, snap)
            snaps[n0 + k] = snap
        st.stencil_record_read(fwd, traces)
    finally:
        st.stencil_destroy(fwd)
    image = torch.zeros((nz, ny, nx), dtype=torch.float32, device=velocity.device)
    bwd = st.stencil_plan(st.make_desc(velocity, dt, src=src, amp=0.0, **common))
    try:
        st.stencil_inject_start(bwd, receiver_z, traces, reverse=True)
        j = 0
        for stop in sorted(T + 1 - t for t in snaps):
            st.stencil_step(bwd, stop - j)
            j = stop
            st.stencil_image_accumulate(bwd, snaps[T + 1 - j], image)
        st.stencil_sync(bwd)
    finally:
        st.stencil_destroy(bwd)
    return image, traces
