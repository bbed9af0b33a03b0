"""Seeded, synthetic inputs shaped like the paper's benchmarks.

This module serves both the CUDA path and the FP64 oracle and holds none of the
method's arithmetic: it produces initial macroscopic fields (density, velocity),
solid masks, random population states and parameter draws.  Equilibrium
populations, relaxation rates and everything else of the scheme are computed by
each side on its own.

Conventions: scalar fields have shape ``(nz, ny, nx)`` (nz = 1 in 2-D), vector
fields ``(D, nz, ny, nx)``; node (i, j, k) sits at x = i, y = j, z = k (lattice
units, 0-based).
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared, used only to express pressure as density

BATCH_SEED = 2602066


def taylor_green_2d(n: int, u0: float = 0.05, rho0: float = 1.0):
    """Decaying Taylor-Green vortex on an n x n periodic lattice (Sec. 3.2):
    u = u0 sin(kx) cos(ky), v = -u0 cos(kx) sin(ky), k = 2 pi / n, with the
    matching pressure p = p0 + rho0 u0^2 / 4 (cos 2kx + cos 2ky) carried by the
    density rho = p / cs^2."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[j, i] = i
    ux = u0 * np.sin(k * X) * np.cos(k * Y)
    uy = -u0 * np.cos(k * X) * np.sin(k * Y)
    rho = rho0 + rho0 * u0 * u0 / (4.0 * CS2) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return rho[None], np.stack([ux, uy])[:, None]


def taylor_green_2d_exact(n: int, u0: float, nu: float, t: float):
    """Velocity of the 2-D vortex above at time t: amplitude decays as exp(-2 nu k^2 t)."""
    k = 2.0 * math.pi / n
    _, u = taylor_green_2d(n, u0)
    return u * math.exp(-2.0 * nu * k * k * t)


def double_shear(n: int, U0: float = 0.1, kappa: float = 80.0, delta: float = 0.05,
                 rho0: float = 1.0):
    """Double shear layer on an n x n periodic lattice (Sec. 3.1), y = j/n, x = i/n."""
    s = np.arange(n, dtype=np.float64) / n
    X, Y = np.meshgrid(s, s, indexing="xy")
    ux = np.where(Y <= 0.5, U0 * np.tanh(kappa * (Y - 0.25)), U0 * np.tanh(kappa * (0.75 - Y)))
    uy = delta * U0 * np.sin(2.0 * math.pi * (X + 0.25))
    rho = np.full_like(ux, rho0)
    return rho[None], np.stack([ux, uy])[:, None]


def taylor_green_3d(n: int, u0: float = 0.05, rho0: float = 1.0):
    """3-D Taylor-Green vortex on an n^3 periodic lattice, k = 2 pi / n:
    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0,
    p = p0 + rho0 u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2)."""
    k = 2.0 * math.pi / n
    c = np.arange(n, dtype=np.float64)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    ux = u0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z)
    uy = -u0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z)
    uz = np.zeros_like(ux)
    rho = rho0 + rho0 * u0 * u0 / (16.0 * CS2) * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * (
        np.cos(2 * k * Z) + 2.0)
    return rho, np.stack([ux, uy, uz])


def channel_at_rest(shape, D: int, rho0: float = 1.0):
    """Uniform density, zero velocity (start of a force-driven channel run)."""
    rho = np.full(shape, rho0)
    return rho, np.zeros((D,) + tuple(shape))


def poiseuille_profile(n_wall: int, u_c: float) -> np.ndarray:
    """Discrete analytic profile of force-driven flow between halfway bounce-back
    walls (Sec. 3.3): u = 4 u_c y (N - y) / N^2 at y = j + 1/2, j = 0..N-1."""
    y = np.arange(n_wall, dtype=np.float64) + 0.5
    return 4.0 * u_c * y * (n_wall - y) / (n_wall * n_wall)


def square_cylinder_mask(nx: int, ny: int, side: int) -> np.ndarray:
    """uint8 (1, ny, nx) mask with a centred side x side solid square."""
    m = np.zeros((1, ny, nx), dtype=np.uint8)
    x0 = (nx - side) // 2
    y0 = (ny - side) // 2
    m[0, y0:y0 + side, x0:x0 + side] = 1
    return m


def random_populations(w: np.ndarray, shape, rng: np.random.Generator, amp: float = 0.05,
                       rho0: float = 1.0) -> np.ndarray:
    """Random positive population states w_i rho0 (1 + amp * xi), xi ~ U(-1, 1):
    near-equilibrium but with every moment (including ghosts) excited."""
    w = np.asarray(w, dtype=np.float64)
    xi = rng.uniform(-1.0, 1.0, size=(len(w),) + tuple(shape))
    wb = w.reshape((len(w),) + (1,) * len(tuple(shape)))
    return wb * rho0 * (1.0 + amp * xi)


def random_macros(shape, D: int, rng: np.random.Generator, umax: float = 0.08,
                  drho: float = 0.02, rho0: float = 1.0):
    rho = rho0 * (1.0 + drho * rng.uniform(-1, 1, size=shape))
    u = umax * rng.uniform(-1, 1, size=(D,) + tuple(shape))
    return rho, u


def batch_lattices(count: int = 256, seed: int = BATCH_SEED, side_min: int = 64,
                   side_max: int = 1024):
    """Uneven double-shear lattices for the batched driver: nx, ny ~ U{side_min..side_max}
    independently, Re ~ log-uniform [1e3, 1e7], Lambda ~ U{1/12, 3/16, 1/4}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.integers(side_min, side_max + 1))
        ny = int(rng.integers(side_min, side_max + 1))
        Re = float(10.0 ** rng.uniform(3.0, 7.0))
        Lam = float(rng.choice([1.0 / 12.0, 3.0 / 16.0, 0.25]))
        out.append({"nx": nx, "ny": ny, "Re": Re, "Lambda": Lam})
    return out


def double_shear_rect(nx: int, ny: int, U0: float = 0.1, kappa: float = 80.0,
                      delta: float = 0.05, rho0: float = 1.0):
    """Double shear layer on an nx x ny periodic lattice (x = i/nx, y = j/ny)."""
    sx = np.arange(nx, dtype=np.float64) / nx
    sy = np.arange(ny, dtype=np.float64) / ny
    X, Y = np.meshgrid(sx, sy, indexing="xy")
    ux = np.where(Y <= 0.5, U0 * np.tanh(kappa * (Y - 0.25)), U0 * np.tanh(kappa * (0.75 - Y)))
    uy = delta * U0 * np.sin(2.0 * math.pi * (X + 0.25))
    rho = np.full_like(ux, rho0)
    return rho[None], np.stack([ux, uy])[:, None]
