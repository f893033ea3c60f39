"""The allocation-free reduction entry point (stencil_sqdiff_noalloc) against
the plan-based one (stencil_rel_l2) on the same data, two calls in a row.

It exists for callers that cannot allocate device memory (all of it held by
a caching allocator, or a path that must not stall on cudaMalloc/cudaFree);
its partial sums live in the library's static device memory.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import math

import numpy as np
import pytest

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


def test_noalloc_matches_plan_reduction_two_calls(env):
    torch, st = env
    nx, ny, nz = 97, 83, 71
    a = workloads.random_field(nx, ny, nz, seed=41)
    b = a.astype(np.float64) + 1e-3 * workloads.random_field(nx, ny, nz, seed=42).astype(np.float64)
    stream = torch.cuda.current_stream()
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    v = workloads.constant_velocity(nx, ny, nz, 2000.0)
    plan = st.stencil_plan(st.make_desc(v, 1e-3, radius=4, stream=stream.cuda_stream))
    try:
        st.stencil_set_fields(plan, da, None)
        want = st.stencil_rel_l2(plan, db)
    finally:
        st.stencil_destroy(plan)
    host = math.sqrt(np.sum((a.astype(np.float64) - b) ** 2) / np.sum(b * b))
    assert want == pytest.approx(host, rel=1e-9)
    for _ in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st.stencil_sqdiff_noalloc(da, nx, db, nx, ny, nz, out, stream.cuda_stream)
        stream.synchronize()
        d2, r2 = out.cpu().tolist()
        assert math.sqrt(d2 / r2) == pytest.approx(want, rel=1e-9)


def test_noalloc_reads_pitched_rows(env):
    torch, st = env
    nx, ny, nz, pitch = 50, 7, 9, 64
    a = workloads.random_field(pitch, ny, nz, seed=43)
    b = workloads.random_field(nx, ny, nz, seed=44).astype(np.float64)
    stream = torch.cuda.current_stream()
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st.stencil_sqdiff_noalloc(da, pitch, db, nx, ny, nz, out, stream.cuda_stream)
    stream.synchronize()
    dense = a[:, :, :nx].astype(np.float64)
    d2, r2 = out.cpu().tolist()
    assert d2 == pytest.approx(np.sum((dense - b) ** 2), rel=1e-12)
    assert r2 == pytest.approx(np.sum(b * b), rel=1e-12)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(env):
    """2^28 + 2^20 elements, one block of partials more than the static array
    holds: refused.  The buffers have the declared sizes (1.1 GB FP32, 2.2 GB
    FP64), so even a launch that got past the check would stay in bounds."""
    torch, st = env
    nx, ny, nz = 1024, 1024, 257
    t = torch.zeros(nx * ny * nz, dtype=torch.float32, device="cuda")
    d = torch.zeros(nx * ny * nz, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(st.StencilError) as ei:
            st.stencil_sqdiff_noalloc(t, nx, d, nx, ny, nz, out)
        assert ei.value.code == st.STENCIL_EINVAL
        assert "2^28" in str(ei.value)
    finally:
        del t, d
        torch.cuda.empty_cache()


def test_noalloc_binding_checks_types_and_sizes(env):
    """The bare C entry point cannot see buffer sizes: the binding refuses
    wrong dtypes and buffers too small for the stated grid before calling it."""
    torch, st = env
    nx, ny, nz = 16, 8, 4
    a = torch.zeros(nx * ny * nz, dtype=torch.float32, device="cuda")
    b = torch.zeros(nx * ny * nz, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for args in ((a.double(), nx, b, out), (a, nx, b.float(), out), (a, nx, b, out[:1]),
                 (a[:-1], nx, b, out), (a, nx + 1, b, out), (a, nx - 1, b, out), (a, nx, b[:-1], out)):
        with pytest.raises(ValueError):
            st.stencil_sqdiff_noalloc(args[0], args[1], args[2], nx, ny, nz, args[3])
    st.stencil_sqdiff_noalloc(a, nx, b, nx, ny, nz, out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0]
