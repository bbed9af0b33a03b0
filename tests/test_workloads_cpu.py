"""CPU checks of the seeded input generators (`workloads/`), against what the
flows they stand for must satisfy rather than against their own formulas:
the Taylor-Green fields are divergence-free and their pressure solves the
pressure Poisson equation (the 2-D one also the steady Euler balance), the
2-D decay law solves the unsteady Stokes equation, the double shear layer is
divergence-free and mirror-symmetric, the Poiseuille profile has a constant
second difference and vanishes at the halfway walls, and the random and
batch draws are reproducible and stay in their stated ranges.  Derivatives
are spectral (exact for these band-limited periodic fields)."""
import math

import numpy as np
import pytest

import workloads as W

CS2 = 1.0 / 3.0


def _d(f, axis, order=1):
    """Spectral derivative of a periodic field along `axis` (unit spacing)."""
    n = f.shape[axis]
    k = 2.0 * math.pi * np.fft.fftfreq(n)
    shape = [1] * f.ndim
    shape[axis] = n
    F = np.fft.fft(f, axis=axis) * (1j * k.reshape(shape)) ** order
    return np.real(np.fft.ifft(F, axis=axis))


@pytest.mark.parametrize("n", [16, 48])
def test_taylor_green_2d_is_a_steady_euler_state(n):
    u0, rho0 = 0.05, 1.0
    rho, u = W.taylor_green_2d(n, u0, rho0)
    rho, ux, uy = rho[0], u[0, 0], u[1, 0]  # (ny, nx): axis 1 is x, axis 0 is y
    assert abs(np.max(np.abs(ux)) - u0) < 1e-12 * u0 * n
    assert np.max(np.abs(_d(ux, 1) + _d(uy, 0))) < 1e-12 * u0
    # grad p = -rho0 (u . grad) u with p = cs^2 rho (the vortex's initial balance)
    p = CS2 * rho
    for comp, a in ((ux, 1), (uy, 0)):
        adv = ux * _d(comp, 1) + uy * _d(comp, 0)
        assert np.max(np.abs(_d(p, a) + rho0 * adv)) < 1e-9 * np.max(np.abs(adv))
    assert abs(np.mean(rho) - rho0) < 1e-15


def test_taylor_green_2d_decay_solves_unsteady_stokes():
    n, u0, nu, t, dt = 32, 0.05, 0.02, 40.0, 1e-3
    u = W.taylor_green_2d_exact(n, u0, nu, t)[:, 0]
    dudt = (W.taylor_green_2d_exact(n, u0, nu, t + dt)[:, 0] -
            W.taylor_green_2d_exact(n, u0, nu, t - dt)[:, 0]) / (2 * dt)
    lap = np.stack([_d(c, 0, 2) + _d(c, 1, 2) for c in u])
    assert np.max(np.abs(dudt - nu * lap)) < 1e-9 * np.max(np.abs(nu * lap))
    assert np.array_equal(W.taylor_green_2d_exact(n, u0, nu, 0.0), W.taylor_green_2d(n, u0)[1])


@pytest.mark.parametrize("n", [12, 24])
def test_taylor_green_3d_divergence_free_with_poisson_pressure(n):
    u0, rho0 = 0.05, 1.0
    rho, u = W.taylor_green_3d(n, u0, rho0)  # (nz, ny, nx): axis 2 is x
    axis = {0: 2, 1: 1, 2: 0}
    div = sum(_d(u[a], axis[a]) for a in range(3))
    assert np.max(np.abs(div)) < 1e-12 * u0
    # lap p = -rho0 d_a d_b (u_a u_b)
    p = CS2 * rho
    lap_p = sum(_d(p, ax, 2) for ax in range(3))
    rhs = np.zeros_like(p)
    for a in range(3):
        for b in range(3):
            rhs -= rho0 * _d(_d(u[a] * u[b], axis[a]), axis[b])
    assert np.max(np.abs(lap_p - rhs)) < 1e-9 * np.max(np.abs(rhs))
    assert np.all(u[2] == 0.0)


@pytest.mark.parametrize("n", [64, 256])
def test_double_shear_layer_structure(n):
    U0, delta = 0.1, 0.05
    rho, u = W.double_shear(n, U0=U0, delta=delta)
    ux, uy = u[0, 0], u[1, 0]
    assert np.array_equal(rho, np.ones_like(rho))
    # u_x depends on y only, u_y on x only: divergence-free on any stencil
    assert np.all(ux == ux[:, :1]) and np.all(uy == uy[:1, :])
    # mirror symmetry of the two layers about y = 1/2, zero crossings at 1/4, 3/4
    col = ux[:, 0]
    assert np.allclose(col[1:], col[1:][::-1], rtol=0, atol=1e-15)
    assert abs(col[n // 4]) < 1e-15 and abs(col[3 * n // 4]) < 1e-15
    assert np.max(np.abs(ux)) <= U0 and abs(np.max(np.abs(uy)) - delta * U0) < 1e-15
    assert abs(np.mean(uy)) < 1e-15
    # the square lattice is the rectangular one with nx = ny
    r2, u2 = W.double_shear_rect(n, n, U0=U0, delta=delta)
    assert np.array_equal(u2, u) and np.array_equal(r2, rho)


def test_poiseuille_profile_is_the_discrete_parabola():
    N, uc = 31, 0.02
    u = W.poiseuille_profile(N, uc)
    second = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.allclose(second, -8.0 * uc / N ** 2, rtol=1e-12, atol=0)
    assert np.allclose(u, u[::-1], rtol=0, atol=1e-17)
    # extrapolated to the halfway walls (y = 0 and y = N) it vanishes
    for a, b, c in ((u[0], u[1], u[2]), (u[-1], u[-2], u[-3])):
        wall = (15 * a - 10 * b + 3 * c) / 8  # quadratic extrapolation half a node out
        assert abs(wall) < 1e-17
    assert abs(u[N // 2] - uc) < 1e-15  # N odd: the middle node sits on the centre line


def test_square_cylinder_mask_is_centred():
    m = W.square_cylinder_mask(200, 81, 21)
    assert m.dtype == np.uint8 and m.shape == (1, 81, 200)
    assert int(m.sum()) == 21 * 21
    ys, xs = np.nonzero(m[0])
    assert xs.max() - xs.min() == 20 and ys.max() - ys.min() == 20
    assert abs((xs.min() + xs.max()) / 2 - (200 - 1) / 2) <= 0.5
    assert abs((ys.min() + ys.max()) / 2 - (81 - 1) / 2) <= 0.5


def test_random_draws_reproducible_and_bounded():
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    a = W.random_populations(w, (3, 5, 7), np.random.default_rng(1), amp=0.05)
    b = W.random_populations(w, (3, 5, 7), np.random.default_rng(1), amp=0.05)
    assert np.array_equal(a, b) and a.shape == (9, 3, 5, 7)
    rel = a / w[:, None, None, None] - 1.0
    assert np.all(np.abs(rel) <= 0.05) and np.all(a > 0)
    rho, u = W.random_macros((4, 6, 8), 3, np.random.default_rng(2), umax=0.08, drho=0.02)
    assert u.shape == (3, 4, 6, 8) and np.all(np.abs(u) <= 0.08)
    assert np.all(np.abs(rho - 1.0) <= 0.02)


def test_batch_lattice_draw():
    a = W.batch_lattices()
    assert a == W.batch_lattices() and len(a) == 256
    assert a != W.batch_lattices(seed=W.BATCH_SEED + 1)
    for d in a:
        assert 64 <= d["nx"] <= 1024 and 64 <= d["ny"] <= 1024
        assert 1e3 <= d["Re"] <= 1e7
        assert d["Lambda"] in (1.0 / 12.0, 3.0 / 16.0, 0.25)
    # the draw spans its ranges
    assert len({d["Lambda"] for d in a}) == 3
    assert min(d["Re"] for d in a) < 1e4 and max(d["Re"] for d in a) > 1e6
