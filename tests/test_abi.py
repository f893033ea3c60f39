"""The C-ABI library loads and exports every declared symbol; host-side
validation and helpers behave (CPU only, no compute calls)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT

import oracle


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"STENCIL_API\s+[\w\s\*]*?\b((?:stencil|shot)_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1310_8232_gb300 import binding
    return binding


def test_library_exports_every_declared_symbol(st):
    lib = ctypes.CDLL(st.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(st):
    for n in declared_symbols():
        assert hasattr(st, n), n


def test_version(st):
    assert "sm_103a" in st.stencil_version()


@pytest.mark.parametrize("R", [4, 5])
def test_cfl_limit_agrees_with_oracle(st, R):
    # Independent implementations (library weights table vs oracle closed form).
    assert st.stencil_cfl_limit(R) == pytest.approx(oracle.cfl_limit(R), rel=1e-14)


def test_cfl_limit_rejects_unsupported_radius(st):
    assert st.stencil_cfl_limit(3) < 0


def test_desc_init_defaults(st):
    d = st.stencil_desc_init()
    assert d.radius == 5 and d.dx == 10.0 and d.src_freq_hz == 15.0
    assert d.src_t0 < 0 and d.src_amp == 1.0
    assert d.storage == st.STENCIL_FP32 and d.tune_mode == st.STENCIL_TUNE_NONE
    assert d.tune.parts == 5 and d.graph_steps == 0


def test_server_cfg_defaults(st):
    c = st.shot_server_cfg_init()
    assert c.hbm_budget_frac == 0.8 and c.max_slots == 64 and c.chunk_steps == 20
    assert c.radius == 5 and c.storage == st.STENCIL_FP32 and c.lanes == 3 and not c.cuda_stream
    import ctypes
    assert ctypes.sizeof(c) == 64            # the C struct: 8 + 8 + 4 * 4 + 8 + 16 + 4 + 4 bytes


def _desc(st, **kw):
    v = np.full((8, 8, 8), 2000.0, dtype=np.float32)
    d = st.make_desc(v, dt=1e-3, radius=4)
    for k, val in kw.items():
        setattr(d, k, val)
    return d, v


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("ny", -1), ("radius", 3), ("radius", 6), ("dx", 0.0), ("dt", -1.0),
    ("src_x", 8), ("src_z", -1), ("graph_steps", 3), ("tune_mode", 9),
    ("absorb_width", -1), ("absorb_width", 256),
    ("nz", 0), ("ny", 65536), ("nz", 65536), ("nx", (1 << 24) + 1), ("dx", float("inf")), ("dt", float("nan")),
    ("src_y", 8), ("src_x", -1), ("src_freq_hz", 0.0), ("storage", 3), ("graph_steps", -2),
    ("absorb_eta", -0.1), ("absorb_eta", float("nan")), ("absorb_eta", float("inf")), ("tune_mode", -1),
])
def test_invalid_descriptors_rejected_before_device(st, field, value):
    d, v = _desc(st, **{field: value})
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == st.STENCIL_EINVAL


def test_null_velocity_rejected(st):
    d, v = _desc(st)
    d.velocity = None
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == st.STENCIL_EINVAL


def test_null_handles_rejected(st):
    for fn, args in ((st._lib.stencil_step, (None, 1)), (st._lib.stencil_sync, (None,)),
                     (st._lib.stencil_destroy, (None,))):
        assert fn(*args) == st.STENCIL_EINVAL


# ---- blocksize-selection building blocks vs the selection oracle ----------
from oracle import selection  # noqa: E402


@pytest.mark.parametrize("S,P", [(200, 5), (800, 5), (250, 10), (1500, 20), (3, 5), (1, 2), (7, 7),
                                 (512, 5), (13, 4)])
def test_candidates_1d_matches_oracle(st, S, P):
    assert st.stencil_candidates_1d(S, P) == selection.candidates_1d(S, P)


def test_candidates_1d_paper_example(st):
    from conftest import read_golden
    for row in read_golden("paper_candidates.txt"):
        assert st.stencil_candidates_1d(int(row[0]), int(row[1])) == [int(x) for x in row[2:]]


@pytest.mark.parametrize("seed", range(20))
@pytest.mark.parametrize("target,name", [(0, "min"), (1, "max"), (2, "avg")])
def test_three_stage_matches_oracle(st, seed, target, name):
    rng = np.random.default_rng(seed)
    G, C, K = rng.integers(1, 4), rng.integers(1, 6), rng.integers(1, 7)
    # coarse values so that ties happen
    t = rng.integers(1, 6, size=(G, C, K)).astype(np.float64)
    g, s, c, tt = st.stencil_select(t, target)
    og, oc, ot = selection.three_stage(t.tolist(), name)
    assert (g, c, tt) == (og, oc, ot)
    # the chosen stream's stage-1 pick is that candidate
    assert t[g, s, c] == tt


@pytest.mark.parametrize("seed", range(10))
def test_original_block_matches_oracle(st, seed):
    rng = np.random.default_rng(100 + seed)
    C, K = rng.integers(1, 6), rng.integers(1, 7)
    t = rng.integers(1, 9, size=(C, K)).astype(np.float64)
    assert st.stencil_select_ob(t) == selection.original_block(t.tolist())


def test_three_stage_skips_missing_entries(st):
    t = np.full((2, 2, 3), np.inf)
    t[0, :, :2] = [[3.0, 2.0], [4.0, 5.0]]
    t[1, :, :1] = [[6.0], [1.0]]
    g, s, c, tt = st.stencil_select(t, 1)       # MWMB: node0 max(2,4)=4; node1 max(6,1)=6
    assert (g, s, c, tt) == (0, 1, 0, 4.0)


def test_selection_rejects_bad_arguments(st):
    with pytest.raises(st.StencilError):
        st.stencil_select(np.ones((1, 1, 1)), 3)
    with pytest.raises(st.StencilError):
        st.stencil_candidates_1d(0, 5)


def test_tile_info_reports_built_tiles(st):
    built = [(tx, ty) for tx in (32, 64, 128) for ty in (4, 8, 16, 32)
             if st.stencil_tile_info(5, tx, ty) is not None]
    assert (64, 16) in built
    smem, threads = st.stencil_tile_info(5, 64, 16)
    assert 0 < smem <= 227 * 1024 and threads % 32 == 0
    assert st.stencil_tile_info(5, 48, 16) is None
    assert st.stencil_tile_info(3, 64, 16) is None


@pytest.mark.parametrize("bufs,code", [
    ((0x10000, 0, 0), "EINVAL"),                     # one of three
    ((0x10000, 0x20000, 0x20000), "EINVAL"),         # the same buffer twice
    ((0x10008, 0x20000, 0x30000), "EINVAL"),         # not 16-byte aligned
])
def test_user_buffer_descriptors_rejected_before_device(st, bufs, code):
    """The caller-owned buffer rules are checked on the pointers alone, before
    any device call (the addresses here are never dereferenced)."""
    d, v = _desc(st)
    for i, b in enumerate(bufs):
        d.user_buffers[i] = b if b else None
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == getattr(st, "STENCIL_" + code)


def test_user_buffers_need_whole_16_byte_rows_and_fp32(st):
    v = np.full((8, 8, 6), 2000.0, dtype=np.float32)      # nx = 6: rows of 24 bytes
    d = st.make_desc(v, dt=1e-3, radius=4)
    for i, b in enumerate((0x10000, 0x20000, 0x30000)):
        d.user_buffers[i] = b
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == st.STENCIL_EINVAL
    d, v = _desc(st)
    for i, b in enumerate((0x10000, 0x20000, 0x30000)):
        d.user_buffers[i] = b
    d.storage = st.STENCIL_FP16
    with pytest.raises(st.StencilError) as ei:
        st.stencil_plan(d)
    assert ei.value.code == st.STENCIL_EUNSUPPORTED
