"""Pins of the oracle's lattice tables, Hermite algebra and subspace structure
(Sec. 2.1, Sec. 2.3, App. A) against printed tables, moment identities and
brute-force linear algebra in numpy."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0
LATTICES = [O.D2Q9, O.D3Q19]


def _w_inner(w, a, b):
    return float(np.sum(w * a * b))


@pytest.mark.parametrize("lat", LATTICES)
def test_moment_isotropy(lat):
    """sum w = 1, sum w e = 0, sum w e e = cs^2 I, fourth-order isotropy, odd moments
    vanish: the conditions that fix the weights (and the D3Q19 weights that the
    paper does not print)."""
    info = O.lattice_info(lat)
    e, w, D = info["e"][:, :info["D"]].astype(float), info["w"], info["D"]
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ e, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(M2, CS2 * np.eye(D), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(D)
    iso = CS2 * CS2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)


@pytest.mark.parametrize("lat", LATTICES)
def test_opposites_and_parity(lat):
    """e_ibar = -e_i, w_ibar = w_i, and H^(n)_ibar = (-1)^n H^(n)_i (Sec. 2.1)."""
    info = O.lattice_info(lat)
    e, w, opp = info["e"], info["w"], info["opp"]
    assert np.array_equal(e[opp], -e)
    assert np.array_equal(w[opp], w)
    H2, H3 = O.hermite(lat)
    assert np.array_equal(H2[opp], H2)
    assert np.array_equal(H3[opp], -H3)


def test_d2q9_matches_printed_table(golden):
    """Velocity order and weights of Eq. (D2Q9)."""
    info = O.lattice_info(O.D2Q9)
    for row in golden("d2q9_lattice.txt"):
        i, ex, ey, w = int(row[0]), int(row[1]), int(row[2]), float(Fraction(row[3]))
        assert info["e"][i, 0] == ex and info["e"][i, 1] == ey
        assert info["w"][i] == pytest.approx(w, abs=1e-16)


def test_d2q9_ghost_matches_printed_values(golden):
    """App. A.1: phi_i in units of cs^4 and the norm 4 cs^8 (after the oracle's
    orthogonalisation, which must leave the D2Q9 mode unchanged)."""
    info = O.lattice_info(O.D2Q9)
    assert info["NG"] == 1
    rows = golden("d2q9_ghost.txt")
    vals = {int(r[0]): float(r[1]) for r in rows if r[0].isdigit()}
    norm = float([r[1] for r in rows if r[0] == "norm_over_cs8"][0])
    cs4 = CS2 ** 2
    for i, v in vals.items():
        assert info["phi"][0, i] == pytest.approx(v * cs4, abs=1e-15)
    assert info["phinorm"][0] == pytest.approx(norm * cs4 * cs4, rel=1e-14)


def _sym_antisym_bases(info):
    """Unit bases of the symmetric / antisymmetric subspaces (Eq. parity)."""
    Q, opp = info["Q"], info["opp"]
    S, A = [], []
    seen = set()
    for i in range(Q):
        if i in seen:
            continue
        j = opp[i]
        seen.update((i, j))
        v = np.zeros(Q)
        v[i] += 1
        v[j] += 1
        S.append(v)
        if j != i:
            a = np.zeros(Q)
            a[i], a[j] = 1, -1
            A.append(a)
    return np.array(S), np.array(A)


@pytest.mark.parametrize("lat,name", [(O.D2Q9, "D2Q9"), (O.D3Q19, "D3Q19")])
def test_subspace_dimensions(lat, name, golden):
    """Tab. lattice_summary / sym_structure / antisym_structure: dim S, dim A, N_G,
    M2, N3 and the antisymmetric completeness dim A = D + N3 (Eq. A_decomp)."""
    row = [r for r in golden("lattice_summary.txt") if r[0] == name][0]
    Q, D, Q0, Qp, dS, dA, NG, N3, M2 = map(int, row[1:])
    info = O.lattice_info(lat)
    assert info["Q"] == Q and info["D"] == D
    Sb, Ab = _sym_antisym_bases(info)
    assert len(Sb) == dS == Q0 + Qp and len(Ab) == dA == Qp
    assert info["NG"] == NG
    n2, n3 = O.hermite_ranks(lat)
    assert n2 == M2 and n3 == N3
    assert D + n3 == dA  # no antisymmetric ghosts (Sec. 2.3.3)
    # numerical ranks from the Hermite tensors themselves
    H2, H3 = O.hermite(lat)
    h2 = np.array([H2[:, a, b] for a in range(D) for b in range(a, D)])
    h3 = np.array([H3[:, a, b, c] for a in range(D) for b in range(a, D) for c in range(b, D)])
    assert np.linalg.matrix_rank(h2, tol=1e-12) == M2
    assert np.linalg.matrix_rank(h3, tol=1e-12) == N3
    e = info["e"][:, :D].astype(float)
    full_A = np.vstack([e.T, h3])
    assert np.linalg.matrix_rank(full_A, tol=1e-12) == dA
    full_S = np.vstack([np.ones(Q), h2, info["phi"]])
    assert np.linalg.matrix_rank(full_S, tol=1e-12) == dS


def _brute_force_ghost_projector(info):
    """Projector onto the w-orthogonal complement of span{1, H2} inside S, by SVD
    in the w^(1/2)-scaled coordinates (brute force, independent of the oracle's
    Gram-Schmidt).  Acts on populations g (which carry the weight): P g."""
    lat = O.D2Q9 if info["Q"] == 9 else O.D3Q19
    w, Q, D = info["w"], info["Q"], info["D"]
    sw = np.sqrt(w)
    H2, _ = O.hermite(lat)
    Sb, _ = _sym_antisym_bases(info)
    # subspaces in scaled coordinates y = h * sqrt(w) for a mode h
    S_sc = (Sb * sw).T  # columns span S
    hyd = np.vstack([np.ones(Q)] + [H2[:, a, b] for a in range(D) for b in range(a, D)])
    hyd_sc = (hyd * sw).T
    # orthonormal basis of S and of hyd
    Us = np.linalg.svd(S_sc, full_matrices=False)[0]
    Uh = np.linalg.svd(hyd_sc, full_matrices=False)[0]
    Uh = Uh[:, :np.linalg.matrix_rank(hyd_sc)]
    Pg_sc = Us @ Us.T - Uh @ Uh.T  # projector onto S minus hydrodynamic span
    # population g = w*h; scaled y = h*sqrt(w) = g / sqrt(w)
    return np.diag(sw) @ Pg_sc @ np.diag(1.0 / sw)


@pytest.mark.parametrize("lat", LATTICES)
def test_ghost_projector_brute_force(lat):
    """The oracle's ghost basis gives the same projector as an SVD construction of
    S minus span{1, H2} (Eq. S_decomp, Eq. ghost_proj)."""
    info = O.lattice_info(lat)
    w = info["w"]
    P_ref = _brute_force_ghost_projector(info)
    P_or = np.zeros_like(P_ref)
    for k in range(info["NG"]):
        phi = info["phi"][k]
        P_or += np.outer(w * phi, phi) / info["phinorm"][k]
    assert np.allclose(P_or, P_ref, atol=1e-14)
    assert np.allclose(P_or @ P_or, P_or, atol=1e-14)  # idempotent


def test_ghost_projector_through_collision():
    """Without the oracle's tables: (f*_TRT - f*_PTRT)/(1 - w+) must equal the
    brute-force ghost projection of fneq (Eq. PTRT versus standard TRT)."""
    rng = np.random.default_rng(7)
    import workloads as W
    for lat in LATTICES:
        info = O.lattice_info(lat)
        P_ref = _brute_force_ghost_projector(info)
        f = W.random_populations(info["w"], (20,), rng, amp=0.2).T.copy()
        kw = dict(omega_plus=1.3, omega_minus=0.9, force=(0.0, 0.0, 0.0))
        a = O.collide(O.Params(lat, 1, 1, 1, collision=O.TRT, **kw), f)
        b = O.collide(O.Params(lat, 1, 1, 1, collision=O.P_TRT, **kw), f)
        e = info["e"][:, :info["D"]].astype(float)
        for n in range(f.shape[0]):
            rho = f[n].sum()
            u = (f[n] @ e) / rho
            feq = O.equilibrium(lat, rho, u)
            pg = P_ref @ (f[n] - feq)
            assert np.allclose((a[n] - b[n]) / (1 - 1.3), pg, atol=1e-15)


def test_d3q19_printed_products_are_not_orthogonal():
    """Why the D3Q19 ghost basis is orthogonalised: the printed products
    (e_a^2 - cs^2)(e_b^2 - cs^2) of App. A.2 have Gram matrix cs^8 [[4,-1,-1],...]
    and overlap H2_zz (<phi_xy, H2_zz>_w = -1/27), contrary to App. A.2."""
    info = O.lattice_info(O.D3Q19)
    e, w = info["e"].astype(float), info["w"]
    prods = [(e[:, a] ** 2 - CS2) * (e[:, b] ** 2 - CS2) for a, b in [(0, 1), (1, 2), (2, 0)]]
    G = np.array([[_w_inner(w, p, q) for q in prods] for p in prods]) * 81
    assert np.allclose(G, [[4, -1, -1], [-1, 4, -1], [-1, -1, 4]], atol=1e-12)
    assert _w_inner(w, prods[0], e[:, 2] ** 2 - CS2) == pytest.approx(-1 / 27, abs=1e-15)
    # the corrected modes phi~_ab = phi_ab + (cs^2/2) H2_cc are orthogonal to 1 and H2
    # and span the same space as the oracle's basis
    corr = [prods[0] + CS2 / 2 * (e[:, 2] ** 2 - CS2), prods[1] + CS2 / 2 * (e[:, 0] ** 2 - CS2),
            prods[2] + CS2 / 2 * (e[:, 1] ** 2 - CS2)]
    H2, _ = O.hermite(O.D3Q19)
    for c in corr:
        assert abs(_w_inner(w, c, np.ones(19))) < 1e-16
        for a, b in product(range(3), range(3)):
            assert abs(_w_inner(w, c, H2[:, a, b])) < 1e-16
    Gc = np.array([[_w_inner(w, p, q) for q in corr] for p in corr]) * 81
    assert np.allclose(Gc, [[3.5, -1, -1], [-1, 3.5, -1], [-1, -1, 3.5]], atol=1e-12)
    both = np.vstack([np.array(corr), info["phi"]])
    assert np.linalg.matrix_rank(both, tol=1e-12) == 3


def _op_matrix(fn, Q):
    return np.array([fn(np.eye(Q)[j]) for j in range(Q)]).T


def test_hermite_contraction_is_projection_only_on_d2q9():
    """Eq. R2R3_hermite's contraction w H3:A3/(6cs^6) is idempotent on D2Q9 but not
    on D3Q19 (H3_xyy and H3_xzz have w-inner product -cs^6 there), which is why the
    TRT-RLB comparator uses the orthogonal projection of Thm 3rd's proof."""
    for lat, q, ok3 in [(O.D2Q9, 9, True), (O.D3Q19, 19, False)]:
        M2 = _op_matrix(lambda g: O.hermite_contraction(lat, g)[0], q)
        M3 = _op_matrix(lambda g: O.hermite_contraction(lat, g)[1], q)
        assert np.allclose(M2 @ M2, M2, atol=1e-14)
        assert np.allclose(M3 @ M3, M3, atol=1e-14) == ok3
    info = O.lattice_info(O.D3Q19)
    e, w = info["e"].astype(float), info["w"]
    xyy = e[:, 0] * (e[:, 1] ** 2 - CS2)
    xzz = e[:, 0] * (e[:, 2] ** 2 - CS2)
    assert _w_inner(w, xyy, xzz) == pytest.approx(-CS2 ** 3, abs=1e-16)
    assert _w_inner(w, xyy, xyy) == pytest.approx(2 * CS2 ** 3, abs=1e-16)


@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_moments(lat):
    """Eq. feq_moments: zeroth to second moments exact on both lattices; on D2Q9
    (the lattice Eq. feq_moments is written for) the third moment is exact for the
    mixed components and aliased for xxx, yyy by exactly -Phi/(3cs^2) = -rho u_a^3.
    (D3Q19 lacks the sixth-order isotropy that would make its mixed third moments
    exact, so only the first three moments are asserted there.)"""
    info = O.lattice_info(lat)
    D = info["D"]
    e = info["e"][:, :D].astype(float)
    rng = np.random.default_rng(11)
    for _ in range(10):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        u = 0.1 * rng.uniform(-1, 1, size=D)
        feq = O.equilibrium(lat, rho, u)
        assert feq.sum() == pytest.approx(rho, abs=1e-15)
        assert np.allclose(feq @ e, rho * u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", feq, e, e),
                           rho * np.outer(u, u) + rho * CS2 * np.eye(D), atol=1e-15)
        if lat != O.D2Q9:
            continue
        m3 = np.einsum("i,ia,ib,ic->abc", feq, e, e, e)
        d = np.eye(D)
        cont = rho * np.einsum("a,b,c->abc", u, u, u) + rho * CS2 * (
            np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d)
            + np.einsum("c,ab->abc", u, d))
        for a, b, c in product(range(D), repeat=3):
            diff = m3[a, b, c] - cont[a, b, c]
            if a == b == c:
                assert diff == pytest.approx(-rho * u[a] ** 3 / (3 * CS2), abs=1e-15)
            else:
                assert abs(diff) < 1e-15


def test_rest_equilibrium_is_weights():
    for lat in LATTICES:
        info = O.lattice_info(lat)
        assert np.allclose(O.equilibrium(lat, 1.3, [0, 0, 0]), 1.3 * info["w"], atol=1e-16)
