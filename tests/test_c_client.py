"""The library used from plain C: tests/c/abi_client.c is compiled with gcc
-std=c11 against include/stencil.h and linked to libstencil.so.  The host
checks run anywhere; on a GPU its 12-step shot must equal, bit for bit, the
same shot through the Python binding."""
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import __graft_entry__
    lib = __graft_entry__.build_library()
    exe = str(tmp_path_factory.mktemp("c") / "abi_client")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_client.c"), "-L", libdir, "-lstencil",
           f"-Wl,-rpath,{libdir}", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_host_calls(client):
    r = subprocess.run([client, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "host ok" in r.stdout


def test_binding_structs_match_the_c_layout(client):
    """Every ctypes mirror in the binding has the size and field offsets the
    C compiler gives the header's struct (an added, dropped or reordered
    field on either side fails here)."""
    import ctypes
    from paper_1310_8232_gb300 import binding as st
    r = subprocess.run([client, "layout"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    c = dict(line.rsplit(" ", 1) for line in r.stdout.strip().splitlines())
    seen = 0
    for key, value in c.items():
        name, _, field = key.partition(".")
        cls = getattr(st, name)
        got = ctypes.sizeof(cls) if not field else getattr(cls, field).offset
        assert got == int(value), (key, got, value)
        seen += 1
    assert seen > 90


@pytest.mark.gpu
def test_c_client_shot_equals_python_binding(client, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out_path = str(tmp_path / "u.bin")
    r = subprocess.run([client, "run", out_path], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    dt = float(r.stdout.split()[1])
    got = np.fromfile(out_path, dtype=np.float32).reshape(30, 36, 40)
    from paper_1310_8232_gb300 import binding as st
    nx, ny, nz = 40, 36, 30
    v = np.empty((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        v[k] = 1800.0 + 500.0 * ((4 * k) // nz)
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    plan = st.stencil_plan(st.make_desc(v, dt, radius=5, dx=10.0, src=(nx // 2, ny // 2, nz // 2),
                                        tile=(st.STENCIL_KERNEL_TILED, 64, 16, -1), graph_steps=4,
                                        stream=s.cuda_stream))
    try:
        want = np.empty_like(v)
        st.stencil_run(plan, 12, want)
    finally:
        st.stencil_destroy(plan)
    assert np.array_equal(got, want)
    assert np.max(np.abs(got)) > 0
