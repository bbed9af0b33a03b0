"""Pins of the oracle's Scheme II forcing (Eq. source_simple, Eq. Gi): the
simplified projection source (1 - w+/2) F_i plus the cubic-velocity correction
G_i built from d_g Phi_abg, Phi_aaa = rho u_a^3.

What fixes each check independently of the oracle's own formulas:
  - the moments of G_i and of F_i printed with the Chapman-Enskog analysis
    (Eq. source_moments) and the second moment of the Guo source;
  - exact differences of a field that is linear in x (central and one-sided
    differences are both exact), and the second-order convergence of the
    central difference on a sine;
  - the physics the correction exists for: without G_i the damping of a sound
    wave carried by a uniform stream U falls by the cubic defect of the
    equilibrium's third moment, by 1.5 (3 U^2 +- sqrt(3) U^3) relative to the
    resting wave; with G_i the damping is Galilean invariant.
"""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def _vel(lat):
    return np.array(O.lattice_info(lat)["e"], dtype=float)


def _params(lat, nx=8, ny=6, nz=1, force=(0.0, 0.0, 0.0), coll=O.P_TRT, periodic=(1, 1, 1),
            solid=None):
    return O.Params(lat, nx, ny, nz if lat == O.D3Q19 else 1, collision=coll, omega_plus=1.3,
                    omega_minus=1.7, force=force, periodic=periodic, solid=solid)


def _node_state(lat, rng):
    D = 2 if lat == O.D2Q9 else 3
    u = np.zeros(3)
    u[:D] = 0.08 * rng.standard_normal(D)
    f = O.equilibrium(lat, 1.0 + 0.02 * rng.standard_normal(), u)
    return f * (1.0 + 0.01 * rng.standard_normal(f.size))


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT, O.TRT_RLB, O.BGK])
def test_g_has_the_printed_moments(lat, coll):
    """Eq. source_moments: sum G = 0, sum e G = 0, sum e_a e_b G = -(1 - w+/2) d_g Phi_abg.
    G is isolated as the difference of two Scheme II collisions of the same
    node that differ only in d_g Phi."""
    rng = np.random.default_rng(11 + lat + 7 * coll)
    D = 2 if lat == O.D2Q9 else 3
    p = _params(lat, force=(2e-5, -1e-5, 3e-5 if D == 3 else 0.0), coll=coll)
    e = _vel(lat)
    for _ in range(5):
        f = _node_state(lat, rng)
        d = np.zeros((3, 3))
        a = rng.standard_normal((D, D)) * 1e-3
        d[:D, :D] = a + a.T  # any symmetric tensor; Phi of the paper gives a diagonal one
        G = O.collide_s2(p, f, d) - O.collide_s2(p, f, np.zeros((3, 3)))
        hg = 1.0 - 0.5 * p.omega_plus
        assert abs(G.sum()) < 1e-15
        np.testing.assert_allclose(e.T @ G, 0.0, atol=1e-15)
        m2 = np.einsum("ia,ib,i->ab", e, e, G)[:D, :D]
        np.testing.assert_allclose(m2, -hg * d[:D, :D], rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT, O.TRT_RLB])
def test_scheme2_force_projection_against_guo(lat, coll):
    """With d_g Phi = 0 the two schemes differ only in the symmetric part of the
    source: Scheme II's F_i has no second moment (Eq. source_moments), the Guo
    source has (1 - w+/2)(u_a F_b + u_b F_a) (Eq. source_guo), with u the
    half-force velocity.  Both add F to the momentum and conserve mass, and
    without a force the two collisions coincide."""
    rng = np.random.default_rng(5 + lat + 3 * coll)
    D = 2 if lat == O.D2Q9 else 3
    F = np.array([3e-5, -2e-5, 1e-5 if D == 3 else 0.0])
    p = _params(lat, force=tuple(F), coll=coll)
    e = _vel(lat)
    zero = np.zeros((3, 3))
    for _ in range(5):
        f = _node_state(lat, rng)
        s1 = O.collide(p, f)
        s2 = O.collide_s2(p, f, zero)
        rho = f.sum()
        u = (e.T @ f + 0.5 * F) / rho
        hg = 1.0 - 0.5 * p.omega_plus
        assert abs(s2.sum() - f.sum()) < 1e-14
        np.testing.assert_allclose(e.T @ s2, e.T @ f + F, atol=1e-15)
        diff = np.einsum("ia,ib,i->ab", e, e, s1 - s2)[:D, :D]
        want = hg * (np.outer(u, F) + np.outer(F, u))[:D, :D]
        # Both collisions round each population to about eps |f|, so an entry of
        # `diff` carries that much absolute error whatever its size.  On D2Q9 and
        # D3Q19 every entry of `want` is large enough for rtol alone; on D3Q27 the
        # random states give an entry near 1e-9 (rtol: 1e-18), so the bound there
        # is one population's rounding, eps max|f| (about 6e-17).
        atol = 1e-18 if lat != O.D3Q27 else np.finfo(float).eps * np.max(np.abs(f))
        np.testing.assert_allclose(diff, want, rtol=1e-9, atol=atol)
    p0 = _params(lat, coll=coll)
    f = _node_state(lat, rng)
    np.testing.assert_array_equal(O.collide_s2(p0, f, zero), O.collide(p0, f))


def _eq_state(p, rho, u):
    return O.init_equilibrium(p, rho, u)


def test_gradient_exact_for_linear_flux_with_walls_and_solids():
    """rho = 1, u_x = (c0 + c1 x)^(1/3): Phi_xxx = c0 + c1 x is linear, so the
    central difference inside and the one-sided differences at the walls and
    next to a solid column all equal c1; a node between two solid columns has
    no neighbour along x and gets 0; d_y Phi_yyy = 0 with u_y = 0."""
    nx, ny = 12, 5
    solid = np.zeros((1, ny, nx), np.uint8)
    solid[0, :, 5] = 1
    solid[0, :, 7] = 1
    p = _params(O.D2Q9, nx, ny, periodic=(0, 1, 1), solid=solid)
    c0, c1 = 1e-4, 3e-5
    x = np.arange(nx, dtype=float)
    u = np.zeros((2, 1, ny, nx))
    u[0] = np.cbrt(c0 + c1 * x)[None, None, :]
    f = _eq_state(p, np.ones((1, ny, nx)), u)
    d = O.cubic_flux_gradient(p, f)
    fluid = solid[0] == 0
    want = np.where(fluid, c1, 0.0)
    want[:, 6] = 0.0  # both x-neighbours solid
    np.testing.assert_allclose(d[0, 0], want, rtol=1e-9, atol=1e-18)
    np.testing.assert_allclose(d[1, 0], 0.0, atol=1e-18)


def test_gradient_exact_for_linear_flux_along_z_d3q19():
    nx, ny, nz = 4, 3, 7
    p = _params(O.D3Q19, nx, ny, nz, periodic=(1, 1, 0))
    c0, c1 = 2e-4, -2e-5
    z = np.arange(nz, dtype=float)
    u = np.zeros((3, nz, ny, nx))
    u[2] = np.cbrt(c0 + c1 * z)[:, None, None]
    f = _eq_state(p, np.ones((nz, ny, nx)), u)
    d = O.cubic_flux_gradient(p, f)
    np.testing.assert_allclose(d[2], c1, rtol=1e-9, atol=1e-18)
    np.testing.assert_allclose(d[:2], 0.0, atol=1e-18)


def test_gradient_second_order_on_periodic_sine():
    """u_x = U sin(kx), rho = 1: d_x (u_x^3) = 3 U^3 k sin^2 cos.  The central
    difference error falls by 4 when the resolution doubles."""
    errs = []
    for nx in (16, 32, 64):
        p = _params(O.D2Q9, nx, 1)
        k = 2 * np.pi / nx
        x = np.arange(nx)
        U = 0.1
        u = np.zeros((2, 1, 1, nx))
        u[0, 0, 0] = U * np.sin(k * x)
        f = _eq_state(p, np.ones((1, 1, nx)), u)
        d = O.cubic_flux_gradient(p, f)[0, 0, 0]
        exact = 3 * U**3 * k * np.sin(k * x) ** 2 * np.cos(k * x)
        errs.append(np.abs(d - exact).max() / np.abs(exact).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def _sound_damping(U, scheme2, sign=1, coll=O.P_TRT, nx=64, nu=0.05, T=1000):
    """Damping rate of a travelling sound wave (direction sign) carried by a
    uniform stream U along x: rho = 1 + d cos(kx), u_x = U + sign cs d cos(kx)."""
    tp = 3 * nu + 0.5
    tm = 0.25 / (tp - 0.5) + 0.5
    p = O.Params(O.D2Q9, nx, 1, 1, collision=coll, omega_plus=1 / tp, omega_minus=1 / tm)
    x = np.arange(nx)
    k = 2 * np.pi / nx
    d = 1e-4
    rho = (1 + d * np.cos(k * x)).reshape(1, 1, nx)
    u = np.zeros((2, 1, 1, nx))
    u[0, 0, 0] = U + sign * np.sqrt(CS2) * d * np.cos(k * x)
    f = _eq_state(p, rho, u)
    g = O.step_s2(p, f, T) if scheme2 else O.step(p, f, T)
    r, _ = O.macros(p, g)
    amp = np.abs(np.fft.rfft(r.reshape(-1))[1]) / (nx / 2)
    return -np.log(amp / d) / T


@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT])
@pytest.mark.parametrize("sign", [1, -1])
def test_g_makes_sound_damping_galilean_invariant(coll, sign):
    """Without G_i the equilibrium's third moment misses rho u_x^3, so the
    normal viscous stress loses (tau+ - 1/2) d_x (rho u_x^3).  Linearised on a
    wave travelling with u' = sign cs rho' in a stream U, that is a fraction
    1.5 (3 U^2 + sign sqrt(3) U^3) of the longitudinal coefficient 2 cs^2 (tau+ - 1/2),
    and the damping rate drops by that fraction.  With G_i (Scheme II) the
    rate is that of the resting wave."""
    U = 0.1
    g0 = _sound_damping(0.0, False, sign, coll)
    g1 = _sound_damping(U, False, sign, coll)
    g2 = _sound_damping(U, True, sign, coll)
    defect = 1.5 * (3 * U * U + sign * np.sqrt(3.0) * U**3)
    assert g1 / g0 == pytest.approx(1.0 - defect, abs=2e-3)
    assert g2 / g0 == pytest.approx(1.0, abs=1e-3)
    assert _sound_damping(0.0, True, sign, coll) == pytest.approx(g0, rel=1e-6)
