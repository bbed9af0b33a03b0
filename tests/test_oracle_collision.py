"""Pins of the oracle's per-node collision against what the paper's theorems and
the mathematics fix: conservation (Eq. macro), ghost annihilation (Eq.
collision_PTRT), the equivalence P-TRT = TRT-RLB (Thm 2nd, Thm 3rd, Rmk exact),
the textbook TRT-Guo and BGK special cases, the rest-state spectrum (Eq.
collision_PTRT / collision_TRT) and the zero ghost eigenvalue of the evolution
operator (Thm stability)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

CS2 = 1.0 / 3.0
LATTICES = [O.D2Q9, O.D3Q19]
ALL = [O.TRT, O.TRT_RLB, O.P_TRT, O.BGK, O.RLB]
RATES = [(1.9, 1.2), (1.0, 1.6), (0.05, 1.99), (1.999, 0.3)]


def _states(lat, n, seed, amp=0.1):
    info = O.lattice_info(lat)
    rng = np.random.default_rng(seed)
    return info, W.random_populations(info["w"], (n,), rng, amp=amp).T.copy()


def _params(lat, coll, wp, wm, F=(0.0, 0.0, 0.0)):
    return O.Params(lat, 1, 1, 1, collision=coll, omega_plus=wp, omega_minus=wm, force=F)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("coll", ALL)
def test_mass_and_momentum_conservation(lat, coll):
    """sum f* = sum f and sum e f* = sum e f + F per node (Eq. macro with the force
    impulse), for every collision, rate pair and a non-zero force."""
    info, f = _states(lat, 40, 1 + lat)
    D = info["D"]
    e = info["e"][:, :D].astype(float)
    F = np.array([2e-3, -1e-3, 5e-4])
    for wp, wm in RATES:
        fs = O.collide(_params(lat, coll, wp, wm, F), f)
        assert np.max(np.abs(fs.sum(1) - f.sum(1))) < 2e-15
        assert np.max(np.abs(fs @ e - f @ e - F[:D])) < 2e-16 * 40


@pytest.mark.parametrize("lat", LATTICES)
def test_ghost_moments_vanish_after_ptrt(lat):
    """P-TRT annihilates the ghost moments of the post-collision state (ghost
    relaxation factor 0, Eq. collision_PTRT); TRT does not (negative control)."""
    info, f = _states(lat, 40, 3)
    F = (1e-3, 2e-3, -1e-3)
    phi = info["phi"]
    fs_p = O.collide(_params(lat, O.P_TRT, 1.7, 1.1, F), f)
    fs_t = O.collide(_params(lat, O.TRT, 1.7, 1.1, F), f)
    g_pre = f @ phi.T
    g_p = fs_p @ phi.T
    g_t = fs_t @ phi.T
    assert np.max(np.abs(g_p)) < 1e-16
    assert np.max(np.abs(g_t)) > 1e-4 * np.max(np.abs(g_pre))


@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_and_rest_weights_have_no_ghost_content(lat):
    """The ghost vectors are w-orthogonal to span{1, H2} (Eq. S_decomp), which
    holds the rest weights and the symmetric part of the third-order f_eq (Eq.
    feq), so the ghost moments of f_eq(rho, u) vanish for any rho, u and those of
    f_neq equal those of f (up to rounding).  Negative control: the ghost moments
    of a random state do not vanish."""
    info = O.lattice_info(lat)
    phi, w = info["phi"], info["w"]
    assert np.max(np.abs(phi @ w)) < 1e-15
    rng = np.random.default_rng(31)
    for _ in range(20):
        rho = 1.0 + 0.2 * rng.uniform(-1, 1)
        u = 0.15 * rng.uniform(-1, 1, size=info["D"])
        feq = O.equilibrium(lat, rho, u)
        assert np.max(np.abs(phi @ feq)) < 1e-15
    _, f = _states(lat, 5, 32)
    assert np.min(np.max(np.abs(f @ phi.T), axis=1)) > 1e-6


def test_d2q9_ghost_vanishes_with_printed_mode(golden):
    """Same as above with the printed D2Q9 mode values (App. A.1), not the oracle's."""
    rows = golden("d2q9_ghost.txt")
    phi = np.array([float(r[1]) for r in rows if r[0].isdigit()]) * CS2 ** 2
    _, f = _states(O.D2Q9, 30, 4)
    fs = O.collide(_params(O.D2Q9, O.P_TRT, 1.8, 1.3, (1e-3, -1e-3, 0)), f)
    assert np.max(np.abs(fs @ phi)) < 1e-16


@pytest.mark.parametrize("lat", LATTICES)
def test_ptrt_equals_trt_rlb(lat):
    """Rmk exact: P-TRT and TRT-RLB give the same post-collision state, per node,
    to 1e-13 relative, including with a body force (Eq. R3_force) and at extreme
    rates (tau+ close to 1/2 and large tau+)."""
    info, f = _states(lat, 200, 5, amp=0.3)
    F = (3e-3, -2e-3, 1e-3)
    for wp, wm in RATES + [(1.0 / 11503.0, 1.6)]:
        a = O.collide(_params(lat, O.P_TRT, wp, wm, F), f)
        b = O.collide(_params(lat, O.TRT_RLB, wp, wm, F), f)
        rel = np.max(np.abs(a - b)) / np.max(np.abs(a))
        assert rel < 1e-13, (wp, wm, rel)


def _moments(info, f, F):
    D = info["D"]
    e = info["e"][:, :D].astype(float)
    rho = f.sum()
    u = (f @ e + 0.5 * np.asarray(F[:D])) / rho
    return e, rho, u


@pytest.mark.parametrize("lat", LATTICES)
def test_trt_is_textbook_trt_guo(lat):
    """With the force reading (first-order term kept, whole Guo source at
    (1 - w+/2)), TRT is the textbook parity-split TRT with Guo forcing:
    f* = f - w+ (f+ - feq+) - w- (f- - feq-) + (1 - w+/2) S+ + (1 - w-/2) S-,
    S = w [(e - u).F/cs^2 + (e.u)(e.F)/cs^4] (Eq. source_guo)."""
    info, f = _states(lat, 30, 6)
    opp = info["opp"]
    F = np.array([2e-3, 1e-3, -1e-3])
    for wp, wm in RATES:
        fs = O.collide(_params(lat, O.TRT, wp, wm, F), f)
        for n in range(f.shape[0]):
            e, rho, u = _moments(info, f[n], F)
            feq = O.equilibrium(lat, rho, u)
            D = info["D"]
            eu, eF, uF = e @ u, e @ F[:D], u @ F[:D]
            S = info["w"] * ((eF - uF) / CS2 + eu * eF / CS2 ** 2)
            plus = lambda v: 0.5 * (v + v[opp])
            minus = lambda v: 0.5 * (v - v[opp])
            ref = (f[n] - wp * (plus(f[n]) - plus(feq)) - wm * (minus(f[n]) - minus(feq))
                   + (1 - wp / 2) * plus(S) + (1 - wm / 2) * minus(S))
            assert np.allclose(fs[n], ref, rtol=0, atol=2e-15)


@pytest.mark.parametrize("lat", LATTICES)
def test_bgk_special_cases(lat):
    """Equal rates: TRT reduces to BGK, f* = f - w (f - feq) without force; the BGK
    comparator equals TRT with w- = w+ with force."""
    info, f = _states(lat, 30, 8)
    for w in (0.6, 1.0, 1.9):
        fs = O.collide(_params(lat, O.TRT, w, w), f)
        for n in range(f.shape[0]):
            e, rho, u = _moments(info, f[n], (0, 0, 0))
            feq = O.equilibrium(lat, rho, u)
            assert np.allclose(fs[n], f[n] - w * (f[n] - feq), rtol=0, atol=2e-15)
        F = (1e-3, -2e-3, 3e-3)
        a = O.collide(_params(lat, O.BGK, w, 0.3, F), f)
        b = O.collide(_params(lat, O.TRT, w, w, F), f)
        assert np.allclose(a, b, rtol=0, atol=2e-15)


@pytest.mark.parametrize("lat", LATTICES)
def test_rlb_is_ptrt_with_unit_minus_rate(lat):
    """Second-order RLB (single rate, third order dropped) equals P-TRT with
    w- = 1 (the equivalence theorems applied to R3 relaxed fully)."""
    _, f = _states(lat, 50, 9, amp=0.2)
    F = (1e-3, 1e-3, -2e-3)
    for w in (0.7, 1.5, 1.98):
        a = O.collide(_params(lat, O.RLB, w, 0.123, F), f)
        b = O.collide(_params(lat, O.P_TRT, w, 1.0, F), f)
        assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 1e-14


def test_printed_forcing_breaks_conservation():
    """Why the force reading: Eq. PTRT taken literally with Scheme I as printed
    (no first-order term, -u.F/cs^2 attached to 1 - 1/(2 tau_s2)) changes the mass
    by (w- - w+)/2 u.F/cs^2 and gives the momentum impulse (3/2 - w-/2) F instead
    of F, while the oracle's reading conserves both exactly."""
    lat = O.D2Q9
    info, f = _states(lat, 10, 10)
    opp, w = info["opp"], info["w"]
    F = np.array([2e-3, -1e-3, 0.0])
    wp, wm = 1.6, 0.8
    ref = O.collide(_params(lat, O.P_TRT, wp, wm, F), f)
    for n in range(f.shape[0]):
        e, rho, u = _moments(info, f[n], F)
        feq = O.equilibrium(lat, rho, u)
        fneq = f[n] - feq
        fp, fm = 0.5 * (fneq + fneq[opp]), 0.5 * (fneq - fneq[opp])
        Fi = w * (e @ F[:2]) / CS2
        pg = ref[n] - feq - (1 - wp) * fp - (1 - wm) * (fm + 0.5 * Fi) - 0.5 * Fi - (
            1 - wp / 2) * w * ((e @ u) * (e @ F[:2]) / CS2 ** 2 - u @ F[:2] / CS2)
        # pg = -(1-w+) P_G fneq: recover the literal printed form with the same ghost part
        s1 = w * ((1 - wp / 2) * (e @ u) * (e @ F[:2]) / CS2 ** 2
                  + (1 - wm / 2) * ((e @ F[:2]) - u @ F[:2]) / CS2)
        lit = feq + (1 - wp) * fp + pg + (1 - wm) * (fm + 0.5 * Fi) + s1
        dm = lit.sum() - f[n].sum()
        assert dm == pytest.approx((wm - wp) / 2 * (u @ F[:2]) / CS2, abs=1e-14)
        dj = lit @ e - f[n] @ e
        assert np.allclose(dj, (1.5 - wm / 2) * F[:2], atol=1e-15)
        assert abs(ref[n].sum() - f[n].sum()) < 1e-15


def _jacobian(lat, coll, wp, wm, h=1e-6):
    info = O.lattice_info(lat)
    f0 = info["w"].copy()
    Q = info["Q"]
    p = _params(lat, coll, wp, wm)
    J = np.zeros((Q, Q))
    for j in range(Q):
        d = np.zeros(Q)
        d[j] = h
        J[:, j] = (O.collide(p, f0 + d) - O.collide(p, f0 - d)) / (2 * h)
    return info, J


@pytest.mark.parametrize("lat", LATTICES)
def test_rest_state_spectrum(lat, golden):
    """Linearised collision at rest (Eq. collision_PTRT / collision_TRT): eigenvalues
    1 (D+1 times), 1-w+ (M2 times), 1-w- (N3 times) and, for the N_G ghosts, 0 for
    P-TRT and TRT-RLB but 1-w+ for TRT."""
    name = "D2Q9" if lat == O.D2Q9 else "D3Q19"
    row = [r for r in golden("lattice_summary.txt") if r[0] == name][0]
    Q, D, NG, N3, M2 = int(row[1]), int(row[2]), int(row[7]), int(row[8]), int(row[9])
    wp, wm = 1.7, 1.15
    for coll, ghost in [(O.P_TRT, 0.0), (O.TRT_RLB, 0.0), (O.TRT, 1 - wp)]:
        _, J = _jacobian(lat, coll, wp, wm)
        ev = np.sort(np.linalg.eigvals(J).real)
        want = np.sort([1.0] * (D + 1) + [1 - wp] * M2 + [1 - wm] * N3 + [ghost] * NG)
        assert len(ev) == Q
        assert np.allclose(ev, want, atol=1e-8), (coll, ev, want)


@pytest.mark.parametrize("lat", LATTICES)
def test_evolution_operator_has_zero_ghost_eigenvalue(lat):
    """Thm stability: L = A(k) C with A = diag(exp(-i k.e_i)) has the eigenvalue 0
    (with multiplicity N_G) for P-TRT at every wave vector; TRT has none."""
    info = O.lattice_info(lat)
    D = info["D"]
    e = info["e"][:, :D].astype(float)
    rng = np.random.default_rng(12)
    for coll, zero in [(O.P_TRT, True), (O.TRT, False)]:
        _, C = _jacobian(lat, coll, 1.9, 1.6)
        for _ in range(5):
            k = rng.uniform(-math.pi, math.pi, size=D)
            A = np.diag(np.exp(-1j * (e @ k)))
            sv = np.linalg.svd(A @ C, compute_uv=False)
            if zero:
                assert np.sum(sv < 1e-7) == info["NG"]
            else:
                assert np.min(sv) > 1e-3


def test_rates_from_physical_parameters(golden):
    """tau+ = 1/2 + nu/cs^2 (Eq. viscosity) and Lambda = (tau+ - 1/2)(tau- - 1/2)
    (Sec. 3.2); the Poiseuille table's tau_s1 for Re = u_c N/nu (Tab. p_l2) and the
    Taylor-Green case nu = 0.01, Lambda = 1/4 (tau+ = 0.53)."""
    wp, wm = O.rates(nu=0.01, Lambda=0.25)
    assert 1 / wp == pytest.approx(0.53, abs=1e-14)
    assert (1 / wp - 0.5) * (1 / wm - 0.5) == pytest.approx(0.25, abs=1e-14)
    for r in golden("poiseuille_l2.txt"):
        Re, tau = float(r[0]), float(r[1])
        wp, _ = O.rates(nu=0.1 * 32 / Re, Lambda=3 / 16)
        assert 1 / wp == pytest.approx(tau, abs=1e-12)
    wp, wm = O.rates(tau_plus=0.8, tau_minus=1 / 1.6)
    assert (wp, wm) == (pytest.approx(1.25), pytest.approx(1.6))
    with pytest.raises(ValueError):
        O.rates(nu=0.01, tau_plus=0.6, Lambda=0.25)
    with pytest.raises(ValueError):
        O.rates(nu=0.01)
