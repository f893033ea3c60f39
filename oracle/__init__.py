"""FP64 CPU oracle for the acoustic stencil sweep -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and nothing
here imports the product package.

The numerical work is in ``stencil_oracle.c`` (plain C, FP64, OpenMP only
over independent k-blocks); this module builds it with gcc on first use and
wraps it with ctypes.  ``selection.py`` holds the paper's blocksize-selection
methodology (Sec. 3.2-3.7) in plain Python.  ``host_method.py`` wraps
``host_method.c``, the paper's method run on the host cores (an FP32 blocked
sweep with an MWMB-selected block): a reported CPU baseline, not a checker.

Arrays are numpy float64 of shape (nz, ny, nx), C order (x fastest).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/liboracle.so (gcc, -O2, no FP contraction),
    and the host-method baseline (host_method.c) beside it."""
    from . import host_method
    host_method.build(force)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("R", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("v", ctypes.c_void_p),
        ("sx", ctypes.c_int32), ("sy", ctypes.c_int32), ("sz", ctypes.c_int32),
        ("f", ctypes.c_double), ("t0", ctypes.c_double), ("amp", ctypes.c_double),
        ("n0", ctypes.c_int64),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_fd_coeffs_rational.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_fd_coeffs.argtypes = [ctypes.c_int, ctypes.c_void_p]
            lib.oracle_cfl_limit.argtypes = [ctypes.c_int]
            lib.oracle_cfl_limit.restype = ctypes.c_double
            lib.oracle_ricker.argtypes = [ctypes.c_double] * 3
            lib.oracle_ricker.restype = ctypes.c_double
            lib.oracle_laplacian.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 2
            lib.oracle_run.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int]
            lib.oracle_energy.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 2 + [ctypes.c_void_p] * 3
            lib.oracle_energy.restype = ctypes.c_double
            lib.oracle_sq_diff.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_run_ext.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Ext), ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_eta.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_long, ctypes.c_long,
                                                            ctypes.c_long]
            lib.oracle_eta.restype = ctypes.c_double
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def fd_coeffs_rational(R: int) -> list[tuple[int, int]]:
    """Exact weights c_0..c_R of the order-2R central 2nd difference as (num, den)."""
    num = np.zeros(R + 1, dtype=np.int64)
    den = np.zeros(R + 1, dtype=np.int64)
    if _load().oracle_fd_coeffs_rational(R, num.ctypes.data, den.ctypes.data):
        raise ValueError(f"radius {R} out of range")
    return [(int(n), int(d)) for n, d in zip(num, den)]


def fd_coeffs(R: int) -> np.ndarray:
    c = np.zeros(R + 1, dtype=np.float64)
    if _load().oracle_fd_coeffs(R, c.ctypes.data):
        raise ValueError(f"radius {R} out of range")
    return c


def cfl_limit(R: int) -> float:
    """Largest stable Courant number v*dt/dx of the 3D leapfrog scheme."""
    return float(_load().oracle_cfl_limit(R))


def ricker(f: float, t0: float, t: float) -> float:
    return float(_load().oracle_ricker(f, t0, t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def laplacian(u, R: int) -> np.ndarray:
    """Lambda(u) on unit spacing with ghost zeros."""
    u = _f64(u)
    if u.ndim != 3:
        raise ValueError("u must be (nz, ny, nx)")
    out = np.empty_like(u)
    nz, ny, nx = u.shape
    if _load().oracle_laplacian(nx, ny, nz, R, u.ctypes.data, out.ctypes.data):
        raise ValueError("bad arguments")
    return out


def run(v, dx: float, dt: float, R: int, steps: int, src=None, f: float = 15.0,
        t0: float | None = None, amp: float = 1.0, u0=None, um1=None, n0: int = 0,
        block=(0, 0, 0), nthreads: int = 0):
    """Advance ``steps`` leapfrog steps from (u0, um1) (zeros if None).

    ``src`` is the source grid index (x, y, z), default the grid centre by
    integer division; ``t0`` defaults to 1/f; ``block`` = (bi, bj, bk) with 0
    meaning the full extent.  Returns (u^{n0+steps}, u^{n0+steps-1}).
    """
    v = _f64(v)
    nz, ny, nx = v.shape
    if src is None:
        src = (nx // 2, ny // 2, nz // 2)
    if t0 is None:
        t0 = 1.0 / f
    u = np.zeros_like(v) if u0 is None else _f64(u0).copy()
    up = np.zeros_like(v) if um1 is None else _f64(um1).copy()
    p = _Problem(nx, ny, nz, R, float(dx), float(dt), v.ctypes.data,
                 int(src[0]), int(src[1]), int(src[2]), float(f), float(t0), float(amp),
                 int(n0))
    rc = _load().oracle_run(ctypes.byref(p), int(steps), int(block[0]), int(block[1]),
                            int(block[2]), u.ctypes.data, up.ctypes.data, int(nthreads))
    if rc:
        raise ValueError("oracle_run: bad arguments")
    return u, up


class _Ext(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("eta_max", ctypes.c_double),
                ("inj_z", ctypes.c_int32), ("inj_y", ctypes.c_int32), ("inj", ctypes.c_void_p),
                ("inj_steps", ctypes.c_int32), ("inj_reverse", ctypes.c_int32), ("inj_scale", ctypes.c_double),
                ("rec_z", ctypes.c_int32), ("rec_y", ctypes.c_int32), ("rec", ctypes.c_void_p),
                ("rec_steps", ctypes.c_int32)]


def run_ext(v, dx: float, dt: float, R: int, steps: int, src=None, f: float = 15.0,
            t0: float | None = None, amp: float = 1.0, u0=None, um1=None, n0: int = 0,
            absorb=(0, 0.0), inject=None, record=None, nthreads: int = 0):
    """The time loop with an absorbing layer, a plane injection and a plane
    record (the RTM pieces around the 3D-model step).

    absorb = (width, eta_max); inject = (z, y, data, reverse, scale) with data
    shaped (steps, rows, nx), rows = ny when y < 0 else 1; record = (z, y).
    Returns (u, u_prev, traces) with traces shaped (steps, rows, nx) or None.
    """
    v = _f64(v)
    nz, ny, nx = v.shape
    if src is None:
        src = (nx // 2, ny // 2, nz // 2)
    if t0 is None:
        t0 = 1.0 / f
    u = np.zeros_like(v) if u0 is None else _f64(u0).copy()
    up = np.zeros_like(v) if um1 is None else _f64(um1).copy()
    p = _Problem(nx, ny, nz, R, float(dx), float(dt), v.ctypes.data,
                 int(src[0]), int(src[1]), int(src[2]), float(f), float(t0), float(amp), int(n0))
    e = _Ext()
    e.width, e.eta_max = int(absorb[0]), float(absorb[1])
    e.inj_z, e.rec_z = -1, -1
    keep = []
    if inject is not None:
        z, y, data, reverse, scale = inject
        data = _f64(data)
        keep.append(data)
        e.inj_z, e.inj_y, e.inj = int(z), int(y), data.ctypes.data
        e.inj_steps, e.inj_reverse, e.inj_scale = int(data.shape[0]), int(bool(reverse)), float(scale)
    traces = None
    if record is not None:
        z, y = record
        traces = np.zeros((steps, ny if y < 0 else 1, nx))
        e.rec_z, e.rec_y, e.rec, e.rec_steps = int(z), int(y), traces.ctypes.data, int(steps)
    rc = _load().oracle_run_ext(ctypes.byref(p), ctypes.byref(e), int(steps), u.ctypes.data, up.ctypes.data,
                                int(nthreads))
    if rc:
        raise ValueError("oracle_run_ext: bad arguments")
    return u, up, traces


def eta(shape, width: int, eta_max: float) -> np.ndarray:
    """The absorbing layer's eta at every point, (nz, ny, nx)."""
    nz, ny, nx = shape
    out = np.empty(shape)
    lib = _load()
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                out[k, j, i] = lib.oracle_eta(nx, ny, nz, width, eta_max, i, j, k)
    return out


def energy(v, dx: float, dt: float, R: int, u1, u0) -> float:
    """Conserved discrete energy between levels n (u0) and n+1 (u1)."""
    v, u1, u0 = _f64(v), _f64(u1), _f64(u0)
    nz, ny, nx = v.shape
    return float(_load().oracle_energy(nx, ny, nz, R, dx, dt, v.ctypes.data,
                                       u1.ctypes.data, u0.ctypes.data))


def rel_l2(a, b) -> float:
    """||a - b|| / ||b|| in FP64 (per-plane partials, planes in order)."""
    a, b = _f64(a), _f64(b)
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    d2 = ctypes.c_double()
    r2 = ctypes.c_double()
    planes = a.shape[0] if a.ndim == 3 else 1
    plane = a.size // planes
    _load().oracle_sq_diff(planes, plane, a.ctypes.data, b.ctypes.data,
                           ctypes.byref(d2), ctypes.byref(r2))
    if r2.value == 0.0:
        return 0.0 if d2.value == 0.0 else float("inf")
    return float(np.sqrt(d2.value / r2.value))
