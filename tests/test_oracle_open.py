"""Pins of the oracle's open boundaries and momentum exchange (Sec. 3.4):
the Zou-He outlet gives its nodes exactly the prescribed density and zero
transverse velocity; the uniform stream that the moving-wall inlet imposes
is an exact fixed point of both boundaries; and the momentum-exchange force
on a solid body balances, at steady state, the body force on the fluid
around it."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _params(shape, periodic, solid=None, F=(0.0, 0.0, 0.0), nu=0.1):
    nz, ny, nx = shape
    wp, wm = O.rates(nu=nu, Lambda=3 / 16)
    return O.Params(O.D2Q9, nx, ny, nz, collision=O.P_TRT, omega_plus=wp, omega_minus=wm,
                    force=F, periodic=periodic, solid=solid)


def test_zou_he_outlet_sets_density_and_zero_transverse_velocity():
    shape = (1, 9, 12)
    p = _params(shape, (0, 1, 1))
    rng = np.random.default_rng(71)
    info = O.lattice_info(O.D2Q9)
    f = W.random_populations(info["w"], shape, rng, amp=0.2)
    for rho_out in (1.0, 0.97):
        g = O.step_open(p, f, 1, u_in=0.03, rho_out=rho_out)
        rho, u = O.macros(p, g)
        assert np.max(np.abs(rho[0, :, -1] - rho_out)) < 1e-14
        assert np.max(np.abs(u[1, 0, :, -1])) < 1e-14
        # negative control: the other columns carry the random state's density
        assert np.max(np.abs(rho[0, :, -2] - rho_out)) > 1e-3


def test_uniform_stream_is_a_fixed_point_of_the_open_boundaries():
    """No obstacle, y periodic: the uniform stream at rho = rho_out, u = (u_in, 0)
    is reproduced exactly (to rounding) by the moving-wall inlet and the Zou-He
    outlet -- the odd part of the third-order equilibrium of a D2Q9 pair is
    exactly 6 w rho (e.u) for a stream along x, which both rules supply.
    Negative controls: an inlet speed different from the stream's, or a
    reversed wall term, changes the state in one step."""
    shape = (1, 6, 16)
    p = _params(shape, (0, 1, 1), nu=0.05)
    rho = np.ones(shape)
    u = np.zeros((2,) + shape)
    u_in = 0.04
    u[0] = u_in
    f = O.init_equilibrium(p, rho, u)
    g = O.step_open(p, f, 200, u_in=u_in, rho_out=1.0)
    assert np.max(np.abs(g - f)) < 1e-13
    g1 = O.step_open(p, f, 1, u_in=1.1 * u_in, rho_out=1.0)
    assert np.max(np.abs(g1 - f)) > 1e-4 * u_in
    g2 = O.step_open(p, f, 1, u_in=-u_in, rho_out=1.0)
    assert np.max(np.abs(g2 - f)) > 1e-3 * u_in


def test_momentum_exchange_balances_the_body_force():
    """Periodic box, resting square obstacle, uniform body force F on the fluid:
    at steady state the force on the solid equals N_fluid F (and no y force)."""
    shape = (1, 20, 20)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[0, 8:12, 8:12] = 1
    F = (1e-5, 0.0, 0.0)
    p = _params(shape, (1, 1, 1), solid=solid, F=F)
    rho0, u0 = W.channel_at_rest(shape, 2)
    f = O.init_equilibrium(p, rho0, u0)
    g = O.step(p, f, 8000, nthreads=4)
    force = O.momentum_exchange(p, g)
    nfluid = int((solid == 0).sum())
    assert force[0] == pytest.approx(nfluid * F[0], rel=1e-6)
    assert abs(force[1]) < 1e-9 * nfluid * F[0]
    # negative control: the state at rest (before the flow develops) is not balanced
    assert abs(O.momentum_exchange(p, f)[0] - nfluid * F[0]) > 0.5 * nfluid * F[0]
