"""Pins of the oracle's RTM pieces: the absorbing layer, the plane
injection and record, and the migration's time pairing."""
import numpy as np
import pytest

import oracle
from oracle import rtm
from paper_1310_8232_gb300 import workloads

DX = 10.0


def model(shape, R, seed=3, layers=3):
    nx, ny, nz = shape
    v = workloads.layered_velocity(nx, ny, nz, n_layers=layers, seed=seed).astype(np.float64)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, float(v.max()))
    return v, dt


@pytest.mark.parametrize("R", [4, 5])
@pytest.mark.parametrize("steps", [1, 2, 3, 7])
def test_plain_extension_is_the_plain_run_bit_for_bit(R, steps):
    v, dt = model((17, 13, 15), R)
    u0 = workloads.random_field(17, 13, 15, seed=2).astype(np.float64)
    a, ap = oracle.run(v, DX, dt, R, steps, u0=u0, um1=0.5 * u0, n0=4, src=(3, 4, 5))
    b, bp, _ = oracle.run_ext(v, DX, dt, R, steps, u0=u0, um1=0.5 * u0, n0=4, src=(3, 4, 5), absorb=(4, 0.0))
    assert np.array_equal(a, b) and np.array_equal(ap, bp)


def test_eta_profile():
    W, emax = 4, 0.3
    e = oracle.eta((11, 12, 13), W, emax)
    assert e[0, 6, 6] == emax and e[10, 6, 6] == emax and e[6, 0, 6] == emax and e[6, 6, 12] == emax
    assert e[5, 6, 6] == 0.0                              # centre, > W from every face
    assert np.all(e >= 0) and np.all(e <= emax)
    # a ray from a face inwards: (W - d)^2 / W^2, zero from d = W on
    ray = e[5, 6, :7]
    want = [emax * ((W - d) / W) ** 2 if d < W else 0.0 for d in range(7)]
    assert np.allclose(ray, want, rtol=0, atol=1e-15)
    assert np.array_equal(e, e[::-1, ::-1, ::-1])          # symmetric under reflection of all axes


@pytest.mark.parametrize("R", [4, 5])
def test_damped_energy_drops_by_exactly_the_dissipation(R):
    """Centred damping: E^{n+1/2} - E^{n-1/2} = - sum eta (u^{n+1} - u^{n-1})^2 / kappa."""
    shape = (20, 18, 16)
    v, dt = model(shape, R)
    W, emax = 5, 0.25
    eta = oracle.eta(shape[::-1], W, emax)
    kappa = v * v * dt * dt / (DX * DX)
    u = workloads.gaussian_bump(*shape, width=2.5, centre=(4, 9, 8)).astype(np.float64)
    um1 = u.copy()
    e_prev = oracle.energy(v, DX, dt, R, u, um1)
    for _ in range(10):
        u1, u0, _ = oracle.run_ext(v, DX, dt, R, 1, amp=0.0, u0=u, um1=um1, absorb=(W, emax))
        e_now = oracle.energy(v, DX, dt, R, u1, u0)
        loss = float(np.sum(eta * (u1 - um1) ** 2 / kappa))
        assert loss > 0
        assert abs((e_now - e_prev) + loss) <= 1e-9 * abs(e_prev)
        e_prev, u, um1 = e_now, u1, u0


def test_layer_absorbs_what_the_plain_boundary_reflects():
    shape, R = (40, 40, 40), 4
    v = np.full(shape[::-1], 2000.0)
    dt = workloads.time_step(oracle.cfl_limit(R), DX, 2000.0)
    u0 = workloads.gaussian_bump(*shape, width=2.0).astype(np.float64)
    steps = 160                                         # the pulse reaches the faces and comes back
    inner = (slice(12, 28),) * 3
    out = {}
    for absorb in ((0, 0.0), (10, 0.3)):
        u, up, _ = oracle.run_ext(v, DX, dt, R, steps, amp=0.0, u0=u0, um1=u0, absorb=absorb)
        out[absorb] = float(np.sum(u[inner] ** 2))
    assert out[(10, 0.3)] < 0.1 * out[(0, 0.0)]


def test_injection_is_adding_after_each_step():
    shape, R = (14, 11, 12), 5
    v, dt = model(shape, R)
    nx, ny, nz = shape
    rng = np.random.default_rng(8)
    data = rng.standard_normal((5, 1, nx))
    z, y = 3, 7
    got, gotp, _ = oracle.run_ext(v, DX, dt, R, 5, src=(6, 5, 6), inject=(z, y, data, False, 0.5))
    u = up = None
    for m in range(5):                                   # by hand: one plain step, then the addition
        u, up = oracle.run(v, DX, dt, R, 1, src=(6, 5, 6), u0=u, um1=up, n0=m)
        u[z, y, :] += 0.5 * data[m, 0]
    assert np.array_equal(got, u) and np.array_equal(gotp, up)


def test_reverse_injection_and_linearity():
    shape, R = (12, 10, 9), 4
    v, dt = model(shape, R)
    nx, ny, nz = shape
    data = np.random.default_rng(9).standard_normal((6, ny, nx))
    a, _, _ = oracle.run_ext(v, DX, dt, R, 6, amp=0.0, inject=(4, -1, data, True, 1.0))
    b, _, _ = oracle.run_ext(v, DX, dt, R, 6, amp=0.0, inject=(4, -1, data[::-1].copy(), False, 1.0))
    c, _, _ = oracle.run_ext(v, DX, dt, R, 6, amp=0.0, inject=(4, -1, data, True, 2.0))
    assert np.array_equal(a, b)
    assert np.array_equal(2.0 * a, c)                    # power-of-two scaling is exact
    # steps beyond the data inject nothing
    d, dp, _ = oracle.run_ext(v, DX, dt, R, 9, amp=0.0, inject=(4, -1, data, False, 1.0))
    e, ep = oracle.run(v, DX, dt, R, 3, amp=0.0, u0=oracle.run_ext(v, DX, dt, R, 6, amp=0.0,
                                                                     inject=(4, -1, data, False, 1.0))[0],
                       um1=oracle.run_ext(v, DX, dt, R, 6, amp=0.0, inject=(4, -1, data, False, 1.0))[1])
    assert np.array_equal(d, e) and np.array_equal(dp, ep)


def test_record_is_the_plane_after_each_step():
    shape, R = (13, 12, 11), 5
    v, dt = model(shape, R)
    _, _, tr = oracle.run_ext(v, DX, dt, R, 6, src=(6, 6, 5), record=(2, -1), absorb=(3, 0.2))
    _, _, row = oracle.run_ext(v, DX, dt, R, 6, src=(6, 6, 5), record=(2, 4), absorb=(3, 0.2))
    u = up = None
    for m in range(6):
        u, up, _ = oracle.run_ext(v, DX, dt, R, 1, src=(6, 6, 5), u0=u, um1=up, n0=m, absorb=(3, 0.2))
        assert np.array_equal(tr[m], u[2])
        assert np.array_equal(row[m, 0], u[2, 4])


def test_migration_pairs_source_and_receiver_fields_in_time():
    """The chunked migration equals a step-by-step one that keeps every
    forward field and every backward field and sums S(t) r^{T+1-t}."""
    shape, R = (16, 14, 18), 4
    v, dt = model(shape, R, layers=2)
    T, k, zr, src, absorb = 12, 3, 2, (8, 7, 3), (3, 0.2)
    image, d, snaps = rtm.migrate(v, DX, dt, R, T, src, zr, k, absorb=absorb)
    fwd = {}
    u = up = None
    traces = []
    for n in range(T):
        u, up, tr = oracle.run_ext(v, DX, dt, R, 1, src=src, u0=u, um1=up, n0=n, absorb=absorb, record=(zr, -1))
        fwd[n + 1] = u
        traces.append(tr[0])
    traces = np.array(traces)
    assert np.array_equal(traces, d)
    bwd = {}
    r = rp = None
    for m in range(T):
        r, rp, _ = oracle.run_ext(v, DX, dt, R, 1, amp=0.0, u0=r, um1=rp, absorb=absorb,
                                  inject=(zr, -1, traces[T - 1 - m][None], False, 1.0))
        bwd[m + 1] = r
    want = sum(fwd[t] * bwd[T + 1 - t] for t in range(k, T + 1, k))
    assert np.allclose(image, want, rtol=1e-14, atol=0)
    for t, s in snaps.items():
        assert np.array_equal(s, fwd[t])


def test_migration_images_the_reflector():
    """Two half-spaces (2000 / 3000 m/s, interface at z = 32), source and
    receivers near the top, absorbing layer: the Laplacian-filtered image
    has its deep maximum at the interface, far above the background between
    the acquisition and the interface."""
    n, R = 64, 4
    v = np.full((n, n, n), 2000.0)
    v[n // 2:] = 3000.0
    dt = workloads.time_step(oracle.cfl_limit(R), DX, 3000.0)
    image, _, _ = rtm.migrate(v, DX, dt, R, 480, (n // 2, n // 2, 8), 6, 4, absorb=(12, 0.2), f=25.0)
    prof = np.abs(oracle.laplacian(image, R)[:, 16:48, 16:48]).mean(axis=(1, 2))
    deep = 26 + int(np.argmax(prof[26:40]))
    assert abs(deep - 32) <= 2
    assert prof[deep] > 10 * np.median(prof[16:25])
