"""The paper's method on the host cores (``host_method.c``) -- a CPU BASELINE.

Only ``bench.py``'s host-method leg and the tests use this module.  It wraps
the FP32 blocked sweep (Sec. 3's loop tiling of Sec. 2's "3D model" step) and
the MWMB blocksize selection across the host's cores (Sec. 3.2-3.3, with the
Sec. 3.7 candidate rule).  The library is built with gcc -O3 -fopenmp, FP
contraction off; arrays are numpy float32 of shape (nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "host_method.c")
_LIB_PATH = os.path.join(_HERE, "libhostmethod.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            I, D, P, L, F = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_long, ctypes.c_float
            lib.hm_run.argtypes = [I, I, I, I, P, I, I, I, F, D, D, D, I, L, I, I, I, P, P, I]
            lib.hm_run.restype = D
            lib.hm_candidates_1d.argtypes = [I, I, P]
            lib.hm_candidates_1d.restype = I
            lib.hm_select_mwmb.argtypes = [I, I, I, I, P, I, I, I, P, P, L, P, P, P]
            lib.hm_select_mwmb.restype = I
            lib.hm_max_threads.restype = I
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().hm_max_threads())


def kappa(v, dx: float, dt: float) -> np.ndarray:
    """kappa = v^2 dt^2 / dx^2 in FP32 (FP64 product, rounded once)."""
    v = np.asarray(v, dtype=np.float64)
    return np.ascontiguousarray((v * v * (dt * dt / (dx * dx))).astype(np.float32))


def run(kap, R: int, steps: int, u, up, src=None, src_scale: float = 0.0, f: float = 15.0,
        t0: float | None = None, dt: float = 0.0, n0: int = 0, block=(0, 0, 0), nthreads: int = 0):
    """FP32 blocked leapfrog steps in place on float32 arrays u (u^n) and up
    (u^{n-1}); returns the wall seconds."""
    kap = np.ascontiguousarray(kap, dtype=np.float32)
    for a in (u, up):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"] or a.shape != kap.shape:
            raise ValueError("u and up must be C-contiguous float32 arrays shaped like kappa")
    nz, ny, nx = kap.shape
    sx, sy, sz = src if src is not None else (-1, 0, 0)
    if t0 is None:
        t0 = 1.0 / f
    el = _load().hm_run(nx, ny, nz, R, kap.ctypes.data, int(sx), int(sy), int(sz), float(src_scale), float(f),
                        float(t0), float(dt), int(steps), int(n0), int(block[0]), int(block[1]), int(block[2]),
                        u.ctypes.data, up.ctypes.data, int(nthreads))
    if el < 0:
        raise ValueError("hm_run: bad arguments")
    return el


def candidates_1d(S: int, P: int) -> list[int]:
    out = (ctypes.c_int * 64)()
    n = _load().hm_candidates_1d(int(S), int(P), out)
    return [out[i] for i in range(n)]


def select_mwmb(kap, R: int, P: int = 3, nI: int = 1, nthreads: int = 0):
    """MWMB on the host cores.  Returns a dict: block (bi, bj, bk), times
    [cores][candidates] (s per nI sweeps), min_time, actual_time, quality,
    candidates, cores, slab depth."""
    kap = np.ascontiguousarray(kap, dtype=np.float32)
    nz, ny, nx = kap.shape
    T = nthreads if nthreads > 0 else max_threads()
    T = min(T, nz)
    nzs = nz // T
    nC = len(candidates_1d(nx, P)) * len(candidates_1d(ny, P)) * len(candidates_1d(nzs, P))
    times = np.zeros(T * nC)
    block = (ctypes.c_int * 3)()
    mt, at, nc = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    rc = _load().hm_select_mwmb(nx, ny, nz, R, kap.ctypes.data, int(P), int(nI), int(T), block,
                                times.ctypes.data, times.size, ctypes.byref(mt), ctypes.byref(at),
                                ctypes.byref(nc))
    if rc:
        raise ValueError("hm_select_mwmb failed")
    return {"block": (block[0], block[1], block[2]), "times": times.reshape(T, nC), "min_time": mt.value,
            "actual_time": at.value, "quality": (at.value - mt.value) / mt.value, "candidates": nc.value,
            "cores": T, "slab": nzs}
