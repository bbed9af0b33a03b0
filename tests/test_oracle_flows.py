"""Flow-level pins of the oracle (collision + streaming + bounce-back +
diagnostics) against the paper's analytic benchmarks and printed numbers:
force-driven Poiseuille flow exact at Lambda = 3/16 (Sec. 3.3, Tab. p_l2),
Taylor-Green decay (Sec. 3.2, Eq. TG), closed forms of the diagnostics, and
brute-force streaming."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _poiseuille(lat, nx, N, nz, uc, nu, Lam, coll, n_diff=40.0):
    wp, wm = O.rates(nu=nu, Lambda=Lam)
    g = 8.0 * nu * uc / N ** 2
    p = O.Params(lat, nx, N, nz, collision=coll, omega_plus=wp, omega_minus=wm,
                 force=(g, 0.0, 0.0), periodic=(1, 0, 1))
    rho, u = W.channel_at_rest(p.shape, p.D)
    f = O.init_equilibrium(p, rho, u)
    nst = int(n_diff / (math.pi ** 2 * nu / N ** 2))
    f = O.step(p, f, nst)
    _, uu = O.macros(p, f)
    prof = W.poiseuille_profile(N, uc)
    ux = np.moveaxis(uu[0], 1, -1).reshape(-1, N)  # every column across the channel
    return O.l2(ux, np.broadcast_to(prof, ux.shape)), uu


@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT_RLB])
def test_poiseuille_d2q9_table(coll, golden):
    """Tab. p_l2: D2Q9 4 x 32, u_c = 0.1, Re = 1, 5, 10 at Lambda = 3/16 gives the
    discrete parabola u = 4 u_c y (N - y)/N^2, y = j + 1/2, to roundoff (the paper
    prints 4e-13 .. 1.2e-12); Lambda = 1/4 leaves the O(1e-4) bounce-back slip."""
    for r in golden("poiseuille_l2.txt"):
        Re, printed = float(r[0]), max(float(r[2]), float(r[3]))
        nu = 0.1 * 32 / Re
        l2, uu = _poiseuille(O.D2Q9, 4, 32, 1, 0.1, nu, 3.0 / 16.0, coll)
        assert l2 < 5.0 * printed, (Re, l2)
        assert np.max(np.abs(uu[1])) < 1e-13
    l2_bad, _ = _poiseuille(O.D2Q9, 4, 32, 1, 0.1, 3.2, 0.25, coll)
    assert 1e-5 < l2_bad < 1e-2


def test_poiseuille_d3q19_channel():
    """The D3Q19 channel (walls normal to y, periodic x and z) reaches the same
    discrete parabola to roundoff at Lambda = 3/16, not at Lambda = 1/4."""
    l2, uu = _poiseuille(O.D3Q19, 3, 12, 3, 0.05, 0.4, 3.0 / 16.0, O.P_TRT, n_diff=34.0)
    assert l2 < 1e-12
    assert np.max(np.abs(uu[1:])) < 1e-13
    l2_bad, _ = _poiseuille(O.D3Q19, 3, 12, 3, 0.05, 0.4, 0.25, O.P_TRT, n_diff=34.0)
    assert l2_bad > 1e-4


@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT, O.TRT_RLB])
def test_taylor_green_2d_decay(coll):
    """Sec. 3.2 (Eq. TG) on 64^2, u0 = 0.05, nu = 0.01, Lambda = 1/4, 1000 steps:
    kinetic energy and enstrophy decay as exp(-4 nu k^2 t) within 1% (lattice and
    Mach errors of a second-order scheme at N = 64), velocity within 0.5% L2 of the
    analytic field; mass conserved to roundoff, momentum stays zero."""
    n, u0, nu, t = 64, 0.05, 0.01, 1000
    wp, wm = O.rates(nu=nu, Lambda=0.25)
    p = O.Params(O.D2Q9, n, n, 1, collision=coll, omega_plus=wp, omega_minus=wm)
    rho, u = W.taylor_green_2d(n, u0)
    f0 = O.init_equilibrium(p, rho, u)
    d0 = O.diagnostics(p, f0)
    f1 = O.step(p, f0, t)
    d1 = O.diagnostics(p, f1)
    k = 2 * math.pi / n
    decay = math.exp(-4 * nu * k * k * t)
    assert d1["kinetic_energy"] / d0["kinetic_energy"] == pytest.approx(decay, rel=0.01)
    assert d1["enstrophy"] / d0["enstrophy"] == pytest.approx(decay, rel=0.01)
    _, uu = O.macros(p, f1)
    assert O.l2(uu, W.taylor_green_2d_exact(n, u0, nu, t)) < 5e-3
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < 1e-12
    assert np.max(np.abs(d1["momentum"])) < 1e-11
    assert d1["nan_flag"] == 0


def test_taylor_green_3d_linear_decay():
    """3-D vortex at small amplitude (Stokes regime) on 24^3: u has |k|^2 = 3 k^2,
    so kinetic energy decays as exp(-6 nu k^2 t); within 2% at N = 24."""
    n, u0, nu, t = 24, 1e-3, 0.02, 120
    wp, wm = O.rates(nu=nu, Lambda=0.25)
    p = O.Params(O.D3Q19, n, n, n, collision=O.P_TRT, omega_plus=wp, omega_minus=wm)
    rho, u = W.taylor_green_3d(n, u0)
    f0 = O.init_equilibrium(p, rho, u)
    d0 = O.diagnostics(p, f0)
    f1 = O.step(p, f0, t, nthreads=4)
    d1 = O.diagnostics(p, f1)
    k = 2 * math.pi / n
    assert d1["kinetic_energy"] / d0["kinetic_energy"] == pytest.approx(
        math.exp(-6 * nu * k * k * t), rel=0.02)


def test_diagnostics_closed_forms():
    """For the 2-D vortex field sampled on the nodes, the second-order central
    difference vorticity is 2 u0 sin(k) sin(kx) sin(ky), so the enstrophy
    1/2 sum |w|^2 is u0^2 sin^2(k) n^2 / 2; kinetic energy 1/2 sum rho |u|^2 and
    mass sum rho follow from the input fields (equilibrium state, F = 0)."""
    n, u0 = 32, 0.04
    p = O.Params(O.D2Q9, n, n, 1, collision=O.P_TRT)
    rho, u = W.taylor_green_2d(n, u0)
    f = O.init_equilibrium(p, rho, u)
    d = O.diagnostics(p, f)
    k = 2 * math.pi / n
    assert d["enstrophy"] == pytest.approx(0.5 * u0 ** 2 * math.sin(k) ** 2 * n * n, rel=1e-12)
    assert d["kinetic_energy"] == pytest.approx(0.5 * np.sum(rho * (u ** 2).sum(0)), rel=1e-12)
    assert d["mass"] == pytest.approx(rho.sum(), rel=1e-14)
    assert np.allclose(d["momentum"][:2], (rho * u).reshape(2, -1).sum(1), atol=1e-13)
    bad = f.copy()
    bad[3, 0, 5, 7] = np.nan
    assert O.diagnostics(p, bad)["nan_flag"] == 1


def test_l2_norm_definition():
    """Sec. 3: L2 = sqrt(sum (qn - qa)^2 / sum qa^2)."""
    qa = np.array([3.0, 4.0])
    assert O.l2(qa, qa) == 0.0
    assert O.l2(2 * qa, qa) == pytest.approx(1.0)
    assert O.l2(np.array([3.0, 0.0]), qa) == pytest.approx(4.0 / 5.0)


def _brute_stream(p, fstar, solid):
    """Independent pull-form streaming in numpy: f_i(x) = f*_i(x - e_i), or
    f*_ibar(x) when x - e_i is solid or beyond a non-periodic edge."""
    info = O.lattice_info(p.lattice)
    e, opp = info["e"], info["opp"]
    nz, ny, nx = p.shape
    out = fstar.copy()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid is not None and solid[z, y, x]:
                    continue
                for i in range(info["Q"]):
                    s = [x - e[i, 0], y - e[i, 1], z - e[i, 2]]
                    ext = [nx, ny, nz]
                    wall = False
                    for a in range(3):
                        if not 0 <= s[a] < ext[a]:
                            if p.periodic[a]:
                                s[a] %= ext[a]
                            else:
                                wall = True
                    if not wall and solid is not None and solid[s[2], s[1], s[0]]:
                        wall = True
                    out[i, z, y, x] = (fstar[opp[i], z, y, x] if wall
                                       else fstar[i, s[2], s[1], s[0]])
    return out


@pytest.mark.parametrize("lat,shape,periodic", [
    (O.D2Q9, (1, 7, 9), (1, 1, 1)),
    (O.D2Q9, (1, 6, 5), (0, 1, 1)),
    (O.D3Q19, (4, 5, 6), (1, 0, 1)),
    (O.D3Q19, (3, 4, 5), (0, 0, 0)),
    (O.D3Q27, (3, 4, 5), (1, 0, 1)),
    (O.D3Q27, (3, 3, 4), (0, 0, 0)),
])
def test_streaming_matches_brute_force(lat, shape, periodic):
    """One oracle step equals node-wise collision (oracle_collide) followed by an
    independent pull-form streaming with walls and an interior solid block."""
    nz, ny, nx = shape
    rng = np.random.default_rng(13)
    info = O.lattice_info(lat)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[nz // 2, ny // 2, nx // 2] = 1
    solid[0, 0, nx - 1] = 1
    p = O.Params(lat, nx, ny, nz, collision=O.P_TRT, omega_plus=1.6, omega_minus=1.1,
                 force=(1e-3, -1e-3, 2e-3), periodic=periodic, solid=solid)
    f = W.random_populations(info["w"], shape, rng, amp=0.2)
    got = O.step(p, f, 1)
    Q = info["Q"]
    fstar = O.collide(p, f.reshape(Q, -1).T.copy()).T.reshape(f.shape)
    fstar = np.where(solid[None] != 0, f, fstar)
    ref = _brute_stream(p, fstar, solid)
    fl = solid[None].repeat(Q, 0) == 0
    assert np.array_equal(got[fl], ref[fl])


def test_pull_sample_matches_step():
    """The sampled-node helper used for full-size parity (oracle.pull_sample)
    agrees bitwise with a whole-lattice oracle step, walls and solids included."""
    nz, ny, nx = 5, 6, 7
    rng = np.random.default_rng(14)
    info = O.lattice_info(O.D3Q19)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[2, 3, 3] = 1
    p = O.Params(O.D3Q19, nx, ny, nz, collision=O.TRT_RLB, omega_plus=1.2, omega_minus=1.7,
                 force=(1e-3, 0, 0), periodic=(1, 0, 1), solid=solid)
    f = W.random_populations(info["w"], (nz, ny, nx), rng, amp=0.2)
    ref = O.step(p, f, 1)
    nodes = [(0, 0, 0), (6, 5, 4), (3, 2, 2), (2, 3, 3 - 1), (4, 3, 2)]
    fs = lambda pts: np.array([f[:, z, y, x] for x, y, z in pts])
    got = O.pull_sample(p, fs, nodes)
    for k, (x, y, z) in enumerate(nodes):
        assert np.array_equal(got[k], ref[:, z, y, x])


def test_rest_state_is_a_fixed_point_with_solids():
    """A fluid at rest (f = w rho0) stays at rest exactly under halfway bounce-back
    at walls and around a solid block, for every collision."""
    nz, ny, nx = 1, 10, 12
    solid = W.square_cylinder_mask(nx, ny, 4)
    for coll in (O.P_TRT, O.TRT, O.TRT_RLB):
        p = O.Params(O.D2Q9, nx, ny, nz, collision=coll, omega_plus=1.3, omega_minus=0.7,
                     periodic=(1, 0, 1), solid=solid)
        rho, u = W.channel_at_rest(p.shape, 2)
        f0 = O.init_equilibrium(p, rho, u)
        f1 = O.step(p, f0, 20)
        assert np.max(np.abs(f1 - f0)) < 1e-15


def test_threads_do_not_change_results():
    n = 24
    wp, wm = O.rates(nu=0.02, Lambda=0.25)
    p = O.Params(O.D2Q9, n, n, 1, collision=O.P_TRT, omega_plus=wp, omega_minus=wm,
                 force=(1e-5, 0, 0))
    rho, u = W.double_shear(n)
    f0 = O.init_equilibrium(p, rho, u)
    assert np.array_equal(O.step(p, f0, 10, nthreads=1), O.step(p, f0, 10, nthreads=4))


def test_mass_conserved_with_walls_solid_and_force():
    nz, ny, nx = 1, 16, 20
    solid = W.square_cylinder_mask(nx, ny, 4)
    wp, wm = O.rates(nu=0.05, Lambda=3 / 16)
    p = O.Params(O.D2Q9, nx, ny, nz, collision=O.P_TRT, omega_plus=wp, omega_minus=wm,
                 force=(1e-4, 0, 0), periodic=(1, 0, 1), solid=solid)
    rho, u = W.channel_at_rest(p.shape, 2)
    f0 = O.init_equilibrium(p, rho, u)
    f1 = O.step(p, f0, 200)
    fl = solid[None].repeat(9, 0) == 0
    assert abs(f1[fl].sum() - f0[fl].sum()) < 1e-11
