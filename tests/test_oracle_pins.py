"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: a Taylor
solve in exact rationals, a textbook table, closed forms, a library
convolution, a dense-matrix brute force on a tiny grid, conservation laws and
symmetries of the scheme.  A dropped term, a wrong sign, a swapped index or a
wrong coefficient in the oracle fails at least one of them.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1310_8232_gb300 import workloads


def taylor_weights(R: int) -> list[Fraction]:
    """Symmetric weights w_0..w_R of the second difference by Taylor matching:
    sum over offsets s = -R..R of w_|s| s^(2m) / (2m)! = [m == 1], m = 0..R,
    solved in exact rationals by Gauss-Jordan elimination."""
    n = R + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for m in range(n):
        for r in range(n):
            if r == 0:
                A[m][r] = Fraction(1 if m == 0 else 0)
            else:
                A[m][r] = Fraction(2 * r ** (2 * m), math.factorial(2 * m))
        b[m] = Fraction(1 if m == 1 else 0)
    # Gauss-Jordan
    for col in range(n):
        piv = next(i for i in range(col, n) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        inv = 1 / A[col][col]
        A[col] = [a * inv for a in A[col]]
        b[col] *= inv
        for i in range(n):
            if i != col and A[i][col] != 0:
                f = A[i][col]
                A[i] = [a - f * c for a, c in zip(A[i], A[col])]
                b[i] -= f * b[col]
    return b


@pytest.mark.parametrize("R", [1, 2, 3, 4, 5, 6])
def test_coeffs_equal_exact_taylor_solve(R):
    got = [Fraction(n, d) for n, d in oracle.fd_coeffs_rational(R)]
    assert got == taylor_weights(R)
    # doubles are the correctly rounded rationals
    c = oracle.fd_coeffs(R)
    for r in range(R + 1):
        assert c[r] == float(got[r])


def test_coeffs_textbook_table():
    for row in read_golden("fd_weights_textbook.txt"):
        R = int(row[0])
        want = [Fraction(x) for x in row[1:]]
        got = [Fraction(n, d) for n, d in oracle.fd_coeffs_rational(R)]
        assert got == want, R


@pytest.mark.parametrize("R", [4, 5])
def test_coeffs_sum_to_zero_and_alternate(R):
    q = [Fraction(n, d) for n, d in oracle.fd_coeffs_rational(R)]
    assert q[0] + 2 * sum(q[1:]) == 0
    for r in range(1, R + 1):
        assert (q[r] > 0) == (r % 2 == 1)


def test_coeffs_r5_values():
    # The paper's order (10th in space, Sec. 2): c_0..c_5 of the order-10 weights.
    got = [Fraction(n, d) for n, d in oracle.fd_coeffs_rational(5)]
    assert got == [Fraction(-5269, 1800), Fraction(5, 3), Fraction(-5, 21),
                   Fraction(5, 126), Fraction(-5, 1008), Fraction(1, 3150)]


@pytest.mark.parametrize("R", [4, 5])
def test_constant_field(R):
    n = 2 * R + 5
    u = np.full((n, n + 1, n + 2), 3.0)
    L = oracle.laplacian(u, R)
    inner = L[R:-R, R:-R, R:-R]
    assert np.all(inner == 0.0) or np.max(np.abs(inner)) < 1e-13
    # corner (0,0,0): on every axis the R lower neighbours are ghosts, so
    # Lambda = 3 * (c_0 + sum c_r) * const = 3 * (c_0 / 2) * const.
    c = oracle.fd_coeffs(R)
    assert L[0, 0, 0] == pytest.approx(3.0 * 1.5 * c[0], rel=1e-14)


@pytest.mark.parametrize("R", [4, 5])
def test_polynomials_exact_to_degree_2R_plus_1(R):
    n = 4 * R + 3
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = x.astype(np.float64) / n
    y = y.astype(np.float64) / n
    z = z.astype(np.float64) / n
    s = slice(R, n - R)
    # x^2 + y^2 + z^2 on unit grid spacing -> Lambda = 6 (in grid units)
    X, Y, Z = x * n, y * n, z * n
    L = oracle.laplacian(X**2 + Y**2 + Z**2, R)
    np.testing.assert_allclose(L[s, s, s], 6.0, rtol=0, atol=1e-9)
    for k in range(2, 2 * R + 2):
        u = (x + 0.5 * y - 0.25 * z + 0.3) ** k
        L = oracle.laplacian(u, R)
        # d2/di2 with x = i/n: chain rule gives factor 1/n^2 per axis
        exact = k * (k - 1) * (x + 0.5 * y - 0.25 * z + 0.3) ** (k - 2) * (1 + 0.25 + 0.0625) / n**2
        err = np.max(np.abs(L[s, s, s] - exact[s, s, s])) / np.max(np.abs(exact[s, s, s]))
        assert err < 1e-9, (k, err)
    # one degree higher is NOT exact: the order is exactly 2R.  On integer
    # coordinates centred in the box, X^(2R+2) has exact Laplacian 0 at the
    # centre, while the 2R-order difference leaves a residual of order 10^3.
    X = np.arange(n, dtype=np.float64) - n // 2
    u = np.broadcast_to(X ** (2 * R + 2), (n, n, n)).copy()
    L = oracle.laplacian(u, R)
    assert abs(L[n // 2, n // 2, n // 2]) > 10.0


@pytest.mark.parametrize("R", [4, 5])
def test_laplacian_matches_library_correlate(R):
    ndimage = pytest.importorskip("scipy.ndimage")
    u = np.random.default_rng(3).standard_normal((13, 17, 19))
    c = [float(Fraction(a, b)) for a, b in taylor_weights_pairs(R)]
    k = np.zeros((2 * R + 1,) * 3)
    k[R, R, R] = 3 * c[0]
    for r in range(1, R + 1):
        for sgn in (-1, 1):
            k[R + sgn * r, R, R] = c[r]
            k[R, R + sgn * r, R] = c[r]
            k[R, R, R + sgn * r] = c[r]
    ref = ndimage.correlate(u, k, mode="constant", cval=0.0)
    L = oracle.laplacian(u, R)
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def taylor_weights_pairs(R):
    return [(f.numerator, f.denominator) for f in taylor_weights(R)]


def dense_laplacian_matrix(nx, ny, nz, R):
    """Lambda as an explicit N x N matrix, entry by entry (offset lookup)."""
    c = [float(f) for f in taylor_weights(R)]
    N = nx * ny * nz
    A = np.zeros((N, N))

    def idx(i, j, k):
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                A[p, p] += 3 * c[0]
                for r in range(1, R + 1):
                    for (di, dj, dk) in ((r, 0, 0), (-r, 0, 0), (0, r, 0), (0, -r, 0),
                                         (0, 0, r), (0, 0, -r)):
                        ii, jj, kk = i + di, j + dj, k + dk
                        if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                            A[p, idx(ii, jj, kk)] += c[r]
    return A


@pytest.mark.parametrize("steps", [12, 13, 14])
@pytest.mark.parametrize("R,shape", [(4, (5, 5, 5)), (5, (6, 4, 7))])
def test_bruteforce_dense_matrix(R, shape, steps):
    nx, ny, nz = shape
    A = dense_laplacian_matrix(nx, ny, nz, R)
    assert np.array_equal(A, A.T)           # symmetric with ghost zeros
    rng = np.random.default_rng(11)
    v = rng.uniform(1500, 4500, (nz, ny, nx))
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / v.max()
    f = 15.0
    src = (nx // 2, ny // 2, nz // 2)
    u0 = rng.standard_normal((nz, ny, nx))
    um1 = rng.standard_normal((nz, ny, nx))
    got, got_prev = oracle.run(v, dx, dt, R, steps, src=src, f=f, u0=u0, um1=um1, n0=3)
    K = (v * v * dt * dt / (dx * dx)).ravel()
    a, b = u0.ravel().copy(), um1.ravel().copy()
    s = (src[2] * ny + src[1]) * nx + src[0]
    for n in range(3, 3 + steps):
        nxt = 2 * a - b + K * (A @ a)
        tau = n * dt - 1.0 / f
        w = (1 - 2 * (math.pi * f * tau) ** 2) * math.exp(-((math.pi * f * tau) ** 2))
        nxt[s] += v.ravel()[s] ** 2 * dt * dt * w
        a, b = nxt, a
    scale = np.max(np.abs(a))
    np.testing.assert_allclose(got.ravel(), a, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(got_prev.ravel(), b, rtol=0, atol=1e-12 * scale)


def test_energy_matches_dense_definition():
    R, (nx, ny, nz) = 4, (5, 6, 5)
    A = dense_laplacian_matrix(nx, ny, nz, R)
    rng = np.random.default_rng(5)
    v = rng.uniform(1500, 4500, (nz, ny, nx))
    u1, u0 = rng.standard_normal((2, nz, ny, nx))
    dx, dt = 10.0, 1e-3
    K = (v * v * dt * dt / (dx * dx)).ravel()
    want = np.sum((u1 - u0).ravel() ** 2 / K) - u1.ravel() @ (A @ u0.ravel())
    got = oracle.energy(v, dx, dt, R, u1, u0)
    assert got == pytest.approx(want, rel=1e-12)


def test_one_dimensional_reduction():
    # ny = nz = 1: the y and z neighbours are all ghosts, so the scheme is the
    # 1D recursion with Lambda_1D = correlate(u, stencil) + 2 c_0 u.
    R, nx = 4, 101
    c = [float(f) for f in taylor_weights(R)]
    w = np.array([c[abs(r)] for r in range(-R, R + 1)])
    v = np.full((1, 1, nx), 2000.0)
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / 2000.0
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal(nx)
    um1 = rng.standard_normal(nx)
    steps = 40
    got, _ = oracle.run(v, dx, dt, R, steps, amp=0.0, u0=u0.reshape(1, 1, nx),
                        um1=um1.reshape(1, 1, nx))
    k = (2000.0 * dt / dx) ** 2
    a, b = u0.copy(), um1.copy()
    for _ in range(steps):
        lap = np.convolve(a, w[::-1], mode="same") + 2 * c[0] * a
        a, b = 2 * a - b + k * lap, a
    np.testing.assert_allclose(got.ravel(), a, rtol=0, atol=1e-11 * np.max(np.abs(a)))


def test_axis_permutation_symmetry():
    R, n = 4, 21
    v = np.full((n, n, n), 2000.0)
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / 2000.0
    u, _ = oracle.run(v, dx, dt, R, 30)
    scale = np.max(np.abs(u))
    assert scale > 0
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        np.testing.assert_allclose(u, np.transpose(u, perm), rtol=0, atol=1e-13 * scale)


def test_blocked_equals_unblocked_bit_for_bit():
    # The paper's Efficient and Wrong blocksizes (Sec. 3.1) on a 200x200x80 slab
    nx, ny, nz, R = 200, 200, 80, 5
    v = workloads.layered_velocity(nx, ny, nz, seed=1310).astype(np.float64)
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / v.max()
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal((nz, ny, nx))
    ref, ref_prev = oracle.run(v, dx, dt, R, 2, u0=u0)
    for block in ((15, 15, 143), (159, 209, 175), (7, 33, 5), (1, 1, 1)):
        got, got_prev = oracle.run(v, dx, dt, R, 2, u0=u0, block=block)
        assert np.array_equal(got, ref), block
        assert np.array_equal(got_prev, ref_prev), block


def test_thread_count_does_not_change_bits():
    nx, ny, nz, R = 30, 20, 25, 4
    v = workloads.layered_velocity(nx, ny, nz).astype(np.float64)
    dt = 0.5 * oracle.cfl_limit(R) * 10.0 / v.max()
    a, _ = oracle.run(v, 10.0, dt, R, 20, nthreads=1)
    b, _ = oracle.run(v, 10.0, dt, R, 20, nthreads=max(2, oracle.max_threads()))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("R", [4, 5])
def test_energy_conserved_without_source(R):
    n = 24
    v = workloads.layered_velocity(n, n, n, n_layers=3, seed=4).astype(np.float64)
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / v.max()
    u0 = workloads.gaussian_bump(n, n, n, width=3.0).astype(np.float64)
    u, up = u0.copy(), u0.copy()
    e0 = oracle.energy(v, dx, dt, R, u, up)
    assert e0 > 0
    for _ in range(10):
        u, up = oracle.run(v, dx, dt, R, 100, amp=0.0, u0=u, um1=up)
        e = oracle.energy(v, dx, dt, R, u, up)
        assert abs(e - e0) / e0 < 1e-12


def test_time_reversal():
    R, n, N = 5, 20, 60
    v = workloads.layered_velocity(n, n, n, n_layers=4, seed=8).astype(np.float64)
    dx = 10.0
    dt = 0.5 * oracle.cfl_limit(R) * dx / v.max()
    u0 = workloads.gaussian_bump(n, n, n).astype(np.float64)
    um1 = u0 * 0.9
    u, up = oracle.run(v, dx, dt, R, N, amp=0.0, u0=u0, um1=um1)
    back, back_prev = oracle.run(v, dx, dt, R, N, amp=0.0, u0=up, um1=u)
    # after N reversed steps: back = u^{-1}... the pair (u^{0}, u^{-1}) swapped
    np.testing.assert_allclose(back, um1, rtol=0, atol=1e-12 * np.max(np.abs(u0)))
    np.testing.assert_allclose(back_prev, u0, rtol=0, atol=1e-12 * np.max(np.abs(u0)))


def test_source_linearity_power_of_two_is_exact():
    R, n = 4, 16
    v = workloads.layered_velocity(n, n, n, seed=2).astype(np.float64)
    dt = 0.5 * oracle.cfl_limit(R) * 10.0 / v.max()
    a, _ = oracle.run(v, 10.0, dt, R, 25)
    b, _ = oracle.run(v, 10.0, dt, R, 25, amp=4.0)
    assert np.array_equal(b, 4.0 * a)


def test_superposition_of_initial_states():
    R, n = 5, 18
    v = workloads.layered_velocity(n, n, n, seed=6).astype(np.float64)
    dt = 0.5 * oracle.cfl_limit(R) * 10.0 / v.max()
    rng = np.random.default_rng(1)
    p, q = rng.standard_normal((2, n, n, n))
    a, _ = oracle.run(v, 10.0, dt, R, 15, amp=0.0, u0=p)
    b, _ = oracle.run(v, 10.0, dt, R, 15, amp=0.0, u0=q)
    c, _ = oracle.run(v, 10.0, dt, R, 15, amp=0.0, u0=p + q)
    np.testing.assert_allclose(c, a + b, rtol=0, atol=1e-12 * np.max(np.abs(c)))


@pytest.mark.parametrize("R", [4, 5])
def test_cfl_limit_matches_symbol_and_dynamics(R):
    c = [float(f) for f in taylor_weights(R)]
    theta = np.linspace(0, np.pi, 20001)
    sym = c[0] + 2 * sum(c[r] * np.cos(r * theta) for r in range(1, R + 1))
    W = np.max(np.abs(sym))
    assert oracle.cfl_limit(R) == pytest.approx(2 / np.sqrt(3 * W), rel=1e-12)
    # values quoted for the two orders (stability bounds of the 3D scheme)
    assert oracle.cfl_limit(R) == pytest.approx({4: 0.452856, 5: 0.441942}[R], abs=2e-6)
    # dynamics: just below the bound stays bounded, just above blows up
    n, vel, dx = 12, 2000.0, 10.0
    v = np.full((n, n, n), vel)
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal((n, n, n))
    for frac, grows in ((0.97, False), (1.05, True)):
        dt = frac * oracle.cfl_limit(R) * dx / vel
        u, _ = oracle.run(v, dx, dt, R, 400, amp=0.0, u0=u0, um1=u0)
        assert (np.max(np.abs(u)) > 1e6) == grows, frac


def test_ricker_closed_form():
    f, t0 = 15.0, 1.0 / 15.0
    assert oracle.ricker(f, t0, t0) == 1.0
    tz = 1.0 / (math.sqrt(2.0) * math.pi * f)
    assert abs(oracle.ricker(f, t0, t0 + tz)) < 1e-15
    assert abs(oracle.ricker(f, t0, t0 - tz)) < 1e-15
    tm = math.sqrt(1.5) / (math.pi * f)
    assert oracle.ricker(f, t0, t0 + tm) == pytest.approx(-2 * math.exp(-1.5), rel=1e-14)


def test_rel_l2_matches_numpy():
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((2, 7, 8, 9))
    assert oracle.rel_l2(a, b) == pytest.approx(np.linalg.norm(a - b) / np.linalg.norm(b),
                                                rel=1e-13)
