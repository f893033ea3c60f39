"""A grid of more than 2^31 points (2048 x 1024 x 1040; 61 GB on the device):
every index the sweep, the plan set-up and the field copies form must be
64-bit.  Fields and model are made on the device; sampled points are
checked against the oracle evaluated point by point on the sub-cube that can
reach them."""
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
    free, _ = torch.cuda.mem_get_info()
    if free < 80 * 2**30:
        pytest.skip("needs 80 GB of free device memory")
    return torch, st


def test_more_than_2_31_points_sampled_against_oracle(env):
    torch, st = env
    nx, ny, nz, R, k = 2048, 1024, 1040, 5, 2
    assert nx * ny * nz > 2**31
    layers = workloads.layer_velocities(8, seed=1310)
    dt = workloads.time_step(st.stencil_cfl_limit(R), workloads.DX, float(layers.max()))
    vl = torch.from_numpy(layers).cuda()
    z = torch.arange(nz, device="cuda")
    v = vl[(8 * z) // nz].view(nz, 1, 1).expand(nz, ny, nx).contiguous()
    g = torch.Generator(device="cuda")
    g.manual_seed(2031)
    u0 = torch.rand((nz, ny, nx), generator=g, device="cuda") - 0.5
    um1 = torch.rand((nz, ny, nx), generator=g, device="cuda") - 0.5
    src = (nx // 2, ny // 2, nz // 2)
    plan = st.stencil_plan(st.make_desc(v, dt, radius=R, src=src, graph_steps=2,
                                        stream=torch.cuda.current_stream().cuda_stream))
    try:
        assert st.stencil_get_stats(plan).tile.kernel == st.STENCIL_KERNEL_TILED
        st.stencil_set_fields(plan, u0, um1, step=40)
        out = torch.empty_like(u0)
        st.stencil_run(plan, k, out)
        torch.cuda.synchronize()
    finally:
        st.stencil_destroy(plan)
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz - 1), (5, ny - 3, nz - 2), src]
    pts += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(40)]
    W = k * R
    worst = 0.0
    for x, y, zz in pts:
        zs = slice(max(0, zz - W), min(nz, zz + W + 1))
        ys = slice(max(0, y - W), min(ny, y + W + 1))
        xs = slice(max(0, x - W), min(nx, x + W + 1))
        cut = lambda a: a[zs, ys, xs].cpu().numpy().astype(np.float64)
        ls = (src[0] - xs.start, src[1] - ys.start, src[2] - zs.start)
        inside = all(0 <= ls[i] < (xs, ys, zs)[i].stop - (xs, ys, zs)[i].start for i in range(3))
        ref, _ = oracle.run(cut(v), workloads.DX, dt, R, k, src=ls if inside else (0, 0, 0),
                            amp=1.0 if inside else 0.0, u0=cut(u0), um1=cut(um1), n0=40)
        got = float(out[zz, y, x])
        want = ref[zz - zs.start, y - ys.start, x - xs.start]
        worst = max(worst, abs(got - want) / max(1.0, abs(want)))
    assert worst < 1e-5, worst
