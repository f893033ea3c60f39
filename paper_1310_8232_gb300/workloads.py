"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no stencil arithmetic: only random draws and the input
recipes (velocity models, grid sizes of a batch of shots, arrival times).
The time step is derived by the caller from a stability bound that it passes
in, so that each side uses its own implementation of that bound.
"""
from __future__ import annotations

import numpy as np

#: RTM source peak frequency used by every workload (Hz).
RICKER_HZ = 15.0
#: Grid spacing used by every workload (m).
DX = 10.0


def constant_velocity(nx: int, ny: int, nz: int, v: float = 2000.0) -> np.ndarray:
    """v(x,y,z) = v, float32 array of shape (nz, ny, nx)."""
    return np.full((nz, ny, nx), v, dtype=np.float32)


def layer_velocities(n_layers: int = 8, vmin: float = 1500.0, vmax: float = 4500.0,
                     seed: int = 1310) -> np.ndarray:
    """Per-layer velocities drawn uniform in [vmin, vmax) (float32)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(vmin, vmax, n_layers).astype(np.float32)


def layered_velocity(nx: int, ny: int, nz: int, n_layers: int = 8, vmin: float = 1500.0,
                     vmax: float = 4500.0, seed: int = 1310) -> np.ndarray:
    """Horizontal layers of equal thickness along z: layer(z) = floor(n_layers * z / nz)."""
    vl = layer_velocities(n_layers, vmin, vmax, seed)
    z = np.arange(nz)
    layer = (n_layers * z) // nz
    v = np.empty((nz, ny, nx), dtype=np.float32)
    v[:] = vl[layer][:, None, None]
    return v


def time_step(cfl_limit: float, dx: float, vmax: float, frac: float = 0.5) -> float:
    """dt = frac * (stable Courant number) * dx / vmax."""
    return frac * cfl_limit * dx / vmax


def batch_dims(n_shots: int = 64, lo: int = 96, hi: int = 320, step: int = 32,
               seed: int = 4064) -> list[tuple[int, int, int]]:
    """Grid sizes (nx, ny, nz) of a batch: each dim uniform over {lo, lo+step, ..., hi}."""
    rng = np.random.default_rng(seed)
    choices = np.arange(lo, hi + 1, step)
    d = rng.choice(choices, size=(n_shots, 3))
    return [tuple(int(x) for x in row) for row in d]


def batch_layer_seeds(n_shots: int, seed: int = 4064) -> list[int]:
    """One velocity-model seed per shot of a batch."""
    rng = np.random.default_rng(seed + 1)
    return [int(s) for s in rng.integers(0, 2**31 - 1, size=n_shots)]


def poisson_arrivals(rate_hz: float = 20.0, window_s: float = 60.0, side_lo: int = 64,
                     side_hi: int = 400, steps_lo: int = 50, steps_hi: int = 500,
                     seed: int = 5020):
    """Open-loop shot stream: Poisson arrivals over a window.

    Returns a list of dicts {t, side, steps, seed}: arrival time (s), cube side
    log-uniform on [side_lo, side_hi] rounded to an integer, step count uniform
    on [steps_lo, steps_hi], and a per-shot velocity seed.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= window_s:
            break
        side = int(round(float(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi))))))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        out.append({"t": t, "side": side, "steps": steps,
                    "seed": int(rng.integers(0, 2**31 - 1))})
    return out


def gaussian_bump(nx: int, ny: int, nz: int, width: float = 3.0, centre=None) -> np.ndarray:
    """exp(-|p - centre|^2 / width^2) on the grid (float32), a smooth start state."""
    if centre is None:
        centre = (nx // 2, ny // 2, nz // 2)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return np.exp(-r2 / width**2).astype(np.float32)


def random_field(nx: int, ny: int, nz: int, seed: int = 7) -> np.ndarray:
    """Standard-normal field (float32), for stencil tests that need every point non-zero."""
    return np.random.default_rng(seed).standard_normal((nz, ny, nx)).astype(np.float32)
