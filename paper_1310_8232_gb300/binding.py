"""ctypes binding of libstencil (include/stencil.h): same names, argument marshalling only.

Every step of the sweep runs in the CUDA library; this module only converts
Python values to the C structures and pointers and turns negative status
codes into ``StencilError``.  Importing it fails loudly if the library has not
been built (``python -m paper_1310_8232_gb300.build``); there is no fallback.

Arrays: numpy arrays are passed as host pointers; torch CUDA tensors are
passed as device pointers (PyTorch provides device memory and streams only).
All arrays are float32 (velocity, fields) or float64 (reference fields) of
shape (nz, ny, nx), C-contiguous.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstencil.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1310_8232_gb300.build` "
                      "(or __graft_entry__.build()); the sweep has no non-CUDA fallback")

_lib = ctypes.CDLL(LIB_PATH)

# ---- constants (mirror include/stencil.h) ----------------------------------
STENCIL_OK = 0
STENCIL_EINVAL = -1
STENCIL_ECFL = -2
STENCIL_ENOMEM = -3
STENCIL_EBUDGET = -4
STENCIL_ETIMEOUT = -5
STENCIL_ECUDA = -6
STENCIL_ENOTREADY = -7
STENCIL_EUNKNOWN_TICKET = -8
STENCIL_ENODEV = -9
STENCIL_EUNSUPPORTED = -10
STENCIL_ECANCELLED = -11
SHOT_QUEUED, SHOT_RUNNING, SHOT_DONE, SHOT_FAILED = 0, 1, 2, 3

STENCIL_FP32, STENCIL_FP16, STENCIL_BF16 = 0, 1, 2
STENCIL_KERNEL_AUTO, STENCIL_KERNEL_NAIVE, STENCIL_KERNEL_TILED, STENCIL_KERNEL_TWO_STEP = 0, 1, 2, 3
(STENCIL_TUNE_NONE, STENCIL_TUNE_OWN, STENCIL_TUNE_MWMB, STENCIL_TUNE_OB, STENCIL_TUNE_MMMB,
 STENCIL_TUNE_MAMB, STENCIL_TUNE_EXHAUSTIVE) = range(7)

_CODE_NAMES = {v: k for k, v in globals().items() if k.startswith("STENCIL_E")}


class StencilError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODE_NAMES.get(code, code)}: {msg}")
        self.code = code


# ---- structures --------------------------------------------------------------
class stencil_tile(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("tx", ctypes.c_int32), ("ty", ctypes.c_int32),
                ("zchunk", ctypes.c_int32)]


class stencil_tune_params(ctypes.Structure):
    _fields_ = [("parts", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("groups", ctypes.c_int32)]


class stencil_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("radius", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("velocity", ctypes.c_void_p), ("velocity_on_device", ctypes.c_int32),
        ("src_x", ctypes.c_int32), ("src_y", ctypes.c_int32), ("src_z", ctypes.c_int32),
        ("src_freq_hz", ctypes.c_double), ("src_t0", ctypes.c_double), ("src_amp", ctypes.c_double),
        ("storage", ctypes.c_int32), ("tune_mode", ctypes.c_int32),
        ("tile", stencil_tile), ("tune", stencil_tune_params),
        ("cuda_stream", ctypes.c_void_p), ("graph_steps", ctypes.c_int32),
        ("user_buffers", ctypes.c_void_p * 3),
        ("absorb_width", ctypes.c_int32), ("absorb_eta", ctypes.c_double),
    ]


class stencil_stats(ctypes.Structure):
    _fields_ = [
        ("steps_done", ctypes.c_int64), ("tile", stencil_tile),
        ("vmax", ctypes.c_double), ("cfl", ctypes.c_double), ("cfl_limit", ctypes.c_double),
        ("pitch", ctypes.c_int64), ("field_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("min_time_ms", ctypes.c_double), ("actual_time_ms", ctypes.c_double),
        ("full_time_ms", ctypes.c_double),
        ("quality", ctypes.c_double), ("selection_ms", ctypes.c_double),
        ("n_candidates", ctypes.c_int32), ("tune_mode", ctypes.c_int32),
        ("current_buffer", ctypes.c_int32), ("user_buffers", ctypes.c_int32),
    ]


class stencil_record_cfg(ctypes.Structure):
    _fields_ = [("receiver_z", ctypes.c_int32), ("receiver_y", ctypes.c_int32),
                ("energy", ctypes.c_int32), ("capacity", ctypes.c_int32)]


class stencil_inject_cfg(ctypes.Structure):
    _fields_ = [("z", ctypes.c_int32), ("y", ctypes.c_int32), ("data", ctypes.c_void_p),
                ("steps", ctypes.c_int32), ("reverse", ctypes.c_int32), ("scale", ctypes.c_float)]


class shot_server_cfg(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_frac", ctypes.c_double), ("hbm_budget_bytes", ctypes.c_int64),
        ("max_slots", ctypes.c_int32), ("chunk_steps", ctypes.c_int32),
        ("radius", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p), ("tile", stencil_tile),
        ("lanes", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


class shot_rtm_cfg(ctypes.Structure):
    _fields_ = [("receiver_z", ctypes.c_int32), ("receiver_y", ctypes.c_int32),
                ("snap_every", ctypes.c_int32), ("image_scale", ctypes.c_float)]


class shot_timing(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("steps_done", ctypes.c_int64), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


class shot_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("done", ctypes.c_int64),
        ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
        ("bytes_in_use", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
        ("iterations", ctypes.c_int64), ("point_updates", ctypes.c_int64), ("busy_s", ctypes.c_double),
        ("admit_s", ctypes.c_double), ("build_s", ctypes.c_double), ("retire_s", ctypes.c_double),
    ]


# ---- prototypes ----------------------------------------------------------------
_P = ctypes.c_void_p
_I = ctypes.c_int32
_lib.stencil_desc_init.argtypes = [ctypes.POINTER(stencil_desc)]
_lib.stencil_desc_init.restype = None
_lib.stencil_plan.argtypes = [ctypes.POINTER(stencil_desc), ctypes.POINTER(_P)]
_lib.stencil_destroy.argtypes = [_P]
_lib.stencil_step.argtypes = [_P, _I]
_lib.stencil_run.argtypes = [_P, _I, _P, _I]
_lib.stencil_sync.argtypes = [_P]
_lib.stencil_get_field.argtypes = [_P, _I, _P, _I]
_lib.stencil_set_fields.argtypes = [_P, _P, _P, _I, ctypes.c_int64]
_lib.stencil_set_velocity.argtypes = [_P, _P, _I]
_lib.stencil_get_stats.argtypes = [_P, ctypes.POINTER(stencil_stats)]
_lib.stencil_record_cfg_init.argtypes = [ctypes.POINTER(stencil_record_cfg)]
_lib.stencil_record_cfg_init.restype = None
_lib.stencil_record_start.argtypes = [_P, ctypes.POINTER(stencil_record_cfg)]
_lib.stencil_record_read.argtypes = [_P, _P, _I, _P, ctypes.POINTER(_I)]
_lib.stencil_record_stop.argtypes = [_P]
_lib.stencil_inject_start.argtypes = [_P, ctypes.POINTER(stencil_inject_cfg)]
_lib.stencil_inject_stop.argtypes = [_P]
_lib.stencil_image_accumulate.argtypes = [_P, _P, _P, ctypes.c_float]
_lib.stencil_debug_wait_fault.argtypes = [_P, _I, ctypes.c_uint32]
_lib.stencil_checkpoint_size.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64)]
_lib.stencil_checkpoint.argtypes = [_P, _P, ctypes.c_uint64, _I]
_lib.stencil_restore.argtypes = [_P, _P, ctypes.c_uint64, _I]
_lib.stencil_energy.argtypes = [_P, ctypes.POINTER(ctypes.c_double)]
_lib.stencil_rel_l2.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_double)]
_lib.stencil_candidates_1d.argtypes = [_I, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I)]
_lib.stencil_select.argtypes = [ctypes.POINTER(ctypes.c_double), _I, _I, _I, _I, ctypes.POINTER(_I),
                                ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]
_lib.stencil_select_ob.argtypes = [ctypes.POINTER(ctypes.c_double), _I, _I, ctypes.POINTER(_I),
                                   ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]
_lib.stencil_batch_create.argtypes = [ctypes.POINTER(stencil_desc), _I, _I, ctypes.POINTER(_P)]
_lib.stencil_batch_run.argtypes = [_P, _I]
_lib.stencil_batch_sync.argtypes = [_P]
_lib.stencil_batch_size.argtypes = [_P, ctypes.POINTER(_I)]
_lib.stencil_batch_plan.argtypes = [_P, _I, ctypes.POINTER(_P)]
_lib.stencil_batch_zchunk.argtypes = [_P, ctypes.POINTER(_I)]
_lib.stencil_batch_destroy.argtypes = [_P]
_lib.shot_server_cfg_init.argtypes = [ctypes.POINTER(shot_server_cfg)]
_lib.shot_server_cfg_init.restype = None
_lib.shot_server_create.argtypes = [ctypes.POINTER(shot_server_cfg), ctypes.POINTER(_P)]
_lib.shot_submit.argtypes = [_P, ctypes.POINTER(stencil_desc), _I, _P, ctypes.POINTER(ctypes.c_uint64)]
_lib.shot_rtm_cfg_init.argtypes = [ctypes.POINTER(shot_rtm_cfg)]
_lib.shot_rtm_cfg_init.restype = None
_lib.shot_submit_rtm.argtypes = [_P, ctypes.POINTER(stencil_desc), _I, ctypes.POINTER(shot_rtm_cfg), _P, _P,
                                 ctypes.POINTER(ctypes.c_uint64)]
_lib.shot_poll.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(shot_timing)]
_lib.shot_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_I)]
_lib.shot_server_get_stats.argtypes = [_P, ctypes.POINTER(shot_server_stats)]
_lib.shot_server_destroy.argtypes = [_P]
_lib.stencil_sqdiff_noalloc.argtypes = [_P, ctypes.c_int64, _P, _I, _I, _I, _P, _P]
_lib.stencil_tile_info.argtypes = [_I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]
_lib.stencil_tile_info.restype = ctypes.c_int
_lib.stencil_cfl_limit.argtypes = [_I]
_lib.stencil_cfl_limit.restype = ctypes.c_double
_lib.stencil_last_error.restype = ctypes.c_char_p
_lib.stencil_version.restype = ctypes.c_char_p
for _name in ("stencil_plan", "stencil_destroy", "stencil_step", "stencil_run", "stencil_sync",
              "stencil_get_field", "stencil_set_fields", "stencil_get_stats", "stencil_energy",
              "stencil_rel_l2", "stencil_set_velocity", "stencil_candidates_1d", "stencil_select",
              "stencil_select_ob", "stencil_sqdiff_noalloc", "stencil_batch_create", "stencil_batch_run",
              "stencil_batch_sync", "stencil_batch_size", "stencil_batch_plan", "stencil_batch_zchunk",
              "stencil_batch_destroy", "shot_server_create", "shot_submit", "shot_submit_rtm", "shot_poll",
              "shot_wait", "shot_server_get_stats", "shot_server_destroy"):
    getattr(_lib, _name).restype = ctypes.c_int


def _check(rc: int) -> int:
    if rc < 0:
        raise StencilError(rc, (_lib.stencil_last_error() or b"").decode())
    return rc


def _ptr(a) -> tuple[int, int]:
    """(address, on_device) of a numpy array or a torch tensor; None -> (0, 0)."""
    if a is None:
        return 0, 0
    if hasattr(a, "data_ptr"):          # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(a.data_ptr()), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return int(a.ctypes.data), 0


# ---- C-ABI calls, same names --------------------------------------------------
def stencil_desc_init() -> stencil_desc:
    d = stencil_desc()
    _lib.stencil_desc_init(ctypes.byref(d))
    return d


def stencil_plan(desc: stencil_desc, velocity=None) -> int:
    """Create a plan; ``velocity`` (numpy float32 or CUDA tensor) overrides desc.velocity.
    Returns the opaque plan handle (an int)."""
    if velocity is not None:
        addr, dev = _ptr(velocity)
        desc.velocity = addr
        desc.velocity_on_device = dev
    h = _P()
    _check(_lib.stencil_plan(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def stencil_destroy(plan: int) -> None:
    _check(_lib.stencil_destroy(plan))


def stencil_step(plan: int, nsteps: int) -> None:
    _check(_lib.stencil_step(plan, nsteps))


def stencil_run(plan: int, nsteps: int, out=None) -> None:
    addr, dev = _ptr(out)
    _check(_lib.stencil_run(plan, nsteps, addr or None, dev))


def stencil_sync(plan: int) -> None:
    _check(_lib.stencil_sync(plan))


def stencil_get_field(plan: int, which: int, out) -> None:
    addr, dev = _ptr(out)
    _check(_lib.stencil_get_field(plan, which, addr, dev))


def stencil_set_fields(plan: int, u=None, u_prev=None, step: int = 0) -> None:
    au, du = _ptr(u)
    ap, dp = _ptr(u_prev)
    if u is not None and u_prev is not None and du != dp:
        raise ValueError("u and u_prev must both be host or both be device arrays")
    _check(_lib.stencil_set_fields(plan, au or None, ap or None, du or dp, step))


def stencil_set_velocity(plan: int, velocity) -> None:
    addr, dev = _ptr(velocity)
    _check(_lib.stencil_set_velocity(plan, addr, dev))


def stencil_get_stats(plan: int) -> stencil_stats:
    s = stencil_stats()
    _check(_lib.stencil_get_stats(plan, ctypes.byref(s)))
    return s


def stencil_record_cfg_init() -> stencil_record_cfg:
    c = stencil_record_cfg()
    _lib.stencil_record_cfg_init(ctypes.byref(c))
    return c


def stencil_record_start(plan: int, receiver_z: int = -1, receiver_y: int = -1, energy: bool = False,
                         capacity: int = 0) -> None:
    c = stencil_record_cfg_init()
    c.receiver_z, c.receiver_y, c.energy, c.capacity = receiver_z, receiver_y, int(bool(energy)), capacity
    _check(_lib.stencil_record_start(plan, ctypes.byref(c)))


def stencil_record_read(plan: int, traces=None, energy=None) -> int:
    """Copy the records made so far into ``traces`` (float32, numpy or CUDA
    tensor, [capacity][ny or 1][nx]) and ``energy`` (numpy float64,
    [capacity]); returns how many records there are."""
    at, dt_ = _ptr(traces)
    ae, de = _ptr(energy)
    if de:
        raise ValueError("energy must be a host array")
    n = _I()
    _check(_lib.stencil_record_read(plan, at or None, dt_, ae or None, ctypes.byref(n)))
    return n.value


def stencil_record_stop(plan: int) -> None:
    _check(_lib.stencil_record_stop(plan))


def stencil_inject_start(plan: int, z: int, data, y: int = -1, reverse: bool = False, scale: float = 1.0) -> None:
    """Inject ``data`` (CUDA float32 tensor, [steps][ny or 1][nx]) on plane z
    after every step from now on (reversed in time when ``reverse``)."""
    addr, dev = _ptr(data)
    if not dev:
        raise ValueError("injection data must be a CUDA tensor")
    c = stencil_inject_cfg(int(z), int(y), addr, int(data.shape[0]), int(bool(reverse)), float(scale))
    _check(_lib.stencil_inject_start(plan, ctypes.byref(c)))


def stencil_inject_stop(plan: int) -> None:
    _check(_lib.stencil_inject_stop(plan))


def stencil_image_accumulate(plan: int, snapshot, image, scale: float = 1.0) -> None:
    """image += scale * snapshot * u^n (CUDA float32 tensors of the grid's shape)."""
    a, da = _ptr(snapshot)
    b, db = _ptr(image)
    if not (da and db):
        raise ValueError("snapshot and image must be CUDA tensors")
    _check(_lib.stencil_image_accumulate(plan, a, b, float(scale)))


def stencil_debug_wait_fault(plan: int, enable: bool, wait_ns: int = 0) -> None:
    _check(_lib.stencil_debug_wait_fault(plan, int(bool(enable)), int(wait_ns)))


def stencil_checkpoint_size(plan: int) -> int:
    n = ctypes.c_uint64()
    _check(_lib.stencil_checkpoint_size(plan, ctypes.byref(n)))
    return n.value


def stencil_checkpoint(plan: int, out=None):
    """Write the plan's state into ``out`` (a uint8 numpy array or CUDA
    tensor of at least stencil_checkpoint_size bytes); with no ``out`` a new
    numpy uint8 array is returned."""
    if out is None:
        import numpy as np
        out = np.empty(stencil_checkpoint_size(plan), dtype=np.uint8)
    addr, dev = _ptr(out)
    nbytes = out.nbytes if hasattr(out, "nbytes") else out.numel() * out.element_size()
    _check(_lib.stencil_checkpoint(plan, addr, nbytes, dev))
    return out


def stencil_restore(plan: int, ckpt) -> None:
    addr, dev = _ptr(ckpt)
    nbytes = ckpt.nbytes if hasattr(ckpt, "nbytes") else ckpt.numel() * ckpt.element_size()
    _check(_lib.stencil_restore(plan, addr, nbytes, dev))


def stencil_energy(plan: int) -> float:
    v = ctypes.c_double()
    _check(_lib.stencil_energy(plan, ctypes.byref(v)))
    return v.value


def stencil_rel_l2(plan: int, ref_device) -> float:
    addr, dev = _ptr(ref_device)
    if not dev:
        raise ValueError("reference must be a CUDA float64 tensor")
    v = ctypes.c_double()
    _check(_lib.stencil_rel_l2(plan, addr, ctypes.byref(v)))
    return v.value


def stencil_candidates_1d(S: int, P: int) -> list[int]:
    out = (_I * max(P, 1))()
    n = _I()
    _check(_lib.stencil_candidates_1d(S, P, out, max(P, 1), ctypes.byref(n)))
    return list(out[: n.value])


def _times_array(times):
    import numpy as np
    a = np.ascontiguousarray(times, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def stencil_select(times, target: int) -> tuple[int, int, int, float]:
    """times: array [groups][streams][cands]; returns (group, stream, cand, time)."""
    a, p = _times_array(times)
    g, s, c = _I(), _I(), _I()
    t = ctypes.c_double()
    G, C, K = a.shape
    _check(_lib.stencil_select(p, G, C, K, target, ctypes.byref(g), ctypes.byref(s), ctypes.byref(c),
                               ctypes.byref(t)))
    return g.value, s.value, c.value, t.value


def stencil_select_ob(times) -> tuple[int, int, float]:
    """times: array [streams][cands]; returns (stream, cand, time)."""
    a, p = _times_array(times)
    s, c = _I(), _I()
    t = ctypes.c_double()
    C, K = a.shape
    _check(_lib.stencil_select_ob(p, C, K, ctypes.byref(s), ctypes.byref(c), ctypes.byref(t)))
    return s.value, c.value, t.value


def stencil_sqdiff_noalloc(a, a_pitch: int, b, nx: int, ny: int, nz: int, out, stream=None) -> None:
    """out[0] = sum (a-b)^2, out[1] = sum b^2 (FP64, device), with no device allocation.
    a: FP32 CUDA tensor (row pitch a_pitch), b: FP64 CUDA tensor, out: 2-element FP64 CUDA tensor.

    The C entry point receives bare pointers and cannot see how large the
    buffers are, so the types and sizes are checked here: a holds at least
    (ny*nz - 1) * a_pitch + nx FP32 values, b at least nx*ny*nz FP64 values,
    out at least 2 FP64 values, all contiguous."""
    pa, da = _ptr(a)
    pb, db = _ptr(b)
    po, do = _ptr(out)
    if not (da and db and do):
        raise ValueError("a, b and out must be CUDA tensors")
    import torch
    if nx <= 0 or ny <= 0 or nz <= 0 or a_pitch < nx:
        raise ValueError("need nx, ny, nz > 0 and a_pitch >= nx")
    rows = ny * nz
    for name, t, dtype, need in (("a", a, torch.float32, (rows - 1) * a_pitch + nx),
                                 ("b", b, torch.float64, nx * rows), ("out", out, torch.float64, 2)):
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} values, the sizes need {need}")
    _check(_lib.stencil_sqdiff_noalloc(pa, a_pitch, pb, nx, ny, nz, po, int(stream) if stream else None))


def stencil_tile_info(radius: int, tx: int, ty: int, storage: int = STENCIL_FP32):
    """(smem_bytes, threads) if the tiled kernel is built for this tile, else None."""
    smem, nt = _I(), _I()
    if _lib.stencil_tile_info(radius, storage, tx, ty, ctypes.byref(smem), ctypes.byref(nt)):
        return smem.value, nt.value
    return None


def stencil_batch_create(descs, graph_steps: int = 0) -> int:
    """Batch of shots from a list of stencil_desc (their velocity arrays must
    stay alive until this returns).  Returns the batch handle."""
    arr = (stencil_desc * len(descs))(*descs)
    h = _P()
    _check(_lib.stencil_batch_create(arr, len(descs), graph_steps, ctypes.byref(h)))
    return h.value


def stencil_batch_run(batch: int, nsteps: int) -> None:
    _check(_lib.stencil_batch_run(batch, nsteps))


def stencil_batch_sync(batch: int) -> None:
    _check(_lib.stencil_batch_sync(batch))


def stencil_batch_size(batch: int) -> int:
    n = _I()
    _check(_lib.stencil_batch_size(batch, ctypes.byref(n)))
    return n.value


def stencil_batch_plan(batch: int, shot: int) -> int:
    h = _P()
    _check(_lib.stencil_batch_plan(batch, shot, ctypes.byref(h)))
    return h.value


def stencil_batch_zchunk(batch: int) -> int:
    z = _I()
    _check(_lib.stencil_batch_zchunk(batch, ctypes.byref(z)))
    return z.value


def stencil_batch_destroy(batch: int) -> None:
    _check(_lib.stencil_batch_destroy(batch))


def shot_server_cfg_init() -> shot_server_cfg:
    c = shot_server_cfg()
    _lib.shot_server_cfg_init(ctypes.byref(c))
    return c


def shot_server_create(cfg: shot_server_cfg) -> int:
    h = _P()
    _check(_lib.shot_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def shot_submit(server: int, desc: stencil_desc, nsteps: int, out_host=None) -> int:
    """Queue a shot; out_host (numpy float32, nz x ny x nx) must stay alive until it finishes."""
    t = ctypes.c_uint64()
    addr, dev = _ptr(out_host)
    if dev:
        raise ValueError("out_host must be host memory")
    _check(_lib.shot_submit(server, ctypes.byref(desc), nsteps, addr or None, ctypes.byref(t)))
    return t.value


def shot_rtm_cfg_init() -> shot_rtm_cfg:
    """A migration request's defaults: every row of the receiver plane, a
    snapshot every 10 steps, image scale 1."""
    c = shot_rtm_cfg()
    _lib.shot_rtm_cfg_init(ctypes.byref(c))
    return c


def shot_submit_rtm(server: int, desc: stencil_desc, nsteps: int, receiver_z: int, snap_every: int,
                    image_host, traces_host=None, receiver_y: int = -1, image_scale: float = 1.0) -> int:
    """Queue a served migration (nsteps forward + nsteps backward steps).
    image_host: numpy float32 (nz, ny, nx); traces_host: numpy float32
    (nsteps, ny or 1, nx) or None; both must stay alive until it finishes."""
    c = shot_rtm_cfg_init()
    c.receiver_z, c.receiver_y, c.snap_every, c.image_scale = int(receiver_z), int(receiver_y), int(snap_every), \
        float(image_scale)
    t = ctypes.c_uint64()
    ia, idev = _ptr(image_host)
    ta, tdev = _ptr(traces_host)
    if idev or tdev or not ia:
        raise ValueError("image_host (required) and traces_host must be host memory")
    _check(_lib.shot_submit_rtm(server, ctypes.byref(desc), nsteps, ctypes.byref(c), ia, ta or None,
                                ctypes.byref(t)))
    return t.value


def shot_poll(server: int, ticket: int) -> tuple[int, shot_timing]:
    st_ = _I()
    tm = shot_timing()
    _check(_lib.shot_poll(server, ticket, ctypes.byref(st_), ctypes.byref(tm)))
    return st_.value, tm


def shot_wait(server: int, ticket: int, timeout_s: float = 60.0) -> int:
    st_ = _I()
    _check(_lib.shot_wait(server, ticket, timeout_s, ctypes.byref(st_)))
    return st_.value


def shot_server_get_stats(server: int) -> shot_server_stats:
    s_ = shot_server_stats()
    _check(_lib.shot_server_get_stats(server, ctypes.byref(s_)))
    return s_


def shot_server_destroy(server: int) -> None:
    _check(_lib.shot_server_destroy(server))


def stencil_cfl_limit(radius: int) -> float:
    return float(_lib.stencil_cfl_limit(radius))


def stencil_last_error() -> str:
    return (_lib.stencil_last_error() or b"").decode()


def stencil_version() -> str:
    return (_lib.stencil_version() or b"").decode()


# ---- convenience -----------------------------------------------------------------
def make_desc(velocity, dt: float, radius: int = 5, dx: float = 10.0, src=None, f: float = 15.0,
              t0: float = -1.0, amp: float = 1.0, tile=None, graph_steps: int = 0, stream=None,
              tune_mode: int = STENCIL_TUNE_NONE, storage: int = STENCIL_FP32,
              buffers=None, absorb=(0, 0.0)) -> stencil_desc:
    """Descriptor for a velocity array of shape (nz, ny, nx); src defaults to the centre.
    ``buffers``: three contiguous CUDA float32 tensors (field 0, field 1, kappa)
    the plan runs on in place of its own allocations."""
    nz, ny, nx = (int(s) for s in velocity.shape)
    d = stencil_desc_init()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.radius = radius
    d.dx, d.dt = float(dx), float(dt)
    sx, sy, sz = src if src is not None else (nx // 2, ny // 2, nz // 2)
    d.src_x, d.src_y, d.src_z = int(sx), int(sy), int(sz)
    d.src_freq_hz, d.src_t0, d.src_amp = float(f), float(t0), float(amp)
    d.storage = storage
    d.tune_mode = tune_mode
    if tile is not None:
        kernel, tx, ty, zc = tile
        d.tile = stencil_tile(kernel, tx, ty, zc)
    d.graph_steps = graph_steps
    d.absorb_width, d.absorb_eta = int(absorb[0]), float(absorb[1])
    if stream is not None:
        d.cuda_stream = int(stream)
    addr, dev = _ptr(velocity)
    d.velocity = addr
    d.velocity_on_device = dev
    if buffers is not None:
        if len(buffers) != 3:
            raise ValueError("buffers: field 0, field 1 and kappa")
        for i, b in enumerate(buffers):
            a, on_dev = _ptr(b)
            if not on_dev:
                raise ValueError("buffers must be CUDA tensors")
            d.user_buffers[i] = a
    return d


EXPORTED = [
    "stencil_desc_init", "stencil_plan", "stencil_destroy", "stencil_step", "stencil_run",
    "stencil_sync", "stencil_get_field", "stencil_set_fields", "stencil_set_velocity",
    "stencil_get_stats", "stencil_checkpoint_size", "stencil_checkpoint", "stencil_restore",
    "stencil_record_cfg_init", "stencil_record_start", "stencil_record_read", "stencil_record_stop",
    "stencil_inject_start", "stencil_inject_stop", "stencil_image_accumulate", "stencil_debug_wait_fault",
    "stencil_energy", "stencil_rel_l2", "stencil_cfl_limit", "stencil_last_error",
    "stencil_candidates_1d", "stencil_select", "stencil_select_ob", "stencil_sqdiff_noalloc",
    "stencil_tile_info", "stencil_batch_create", "stencil_batch_run", "stencil_batch_sync",
    "stencil_batch_size", "stencil_batch_plan", "stencil_batch_zchunk", "stencil_batch_destroy",
    "shot_server_cfg_init", "shot_server_create", "shot_submit", "shot_rtm_cfg_init", "shot_submit_rtm",
    "shot_poll", "shot_wait", "shot_server_get_stats", "shot_server_destroy",
    "stencil_version",
]
