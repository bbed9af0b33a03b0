"""GPU parity on D3Q27 (App. D3Q27, Eq. PTRT_D3Q27): the hybrid P-TRT, TRT,
TRT-RLB and the BGK / RLB parameterisations against the FP64 oracle on the same
seeded inputs, element by element (FP64 to 1e-12 in every population; FP32 to
2e-5 in rho and u), with walls, forces, solid nodes, both layouts, the
pipelined and register kernels (bit for bit against each other), and forcing
Scheme II."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_cases import elem_rel, gpu_lattice, oracle_params, scaled_err

pytestmark = pytest.mark.gpu

LAT = O.D3Q27
COLLS = [O.P_TRT, O.TRT, O.TRT_RLB]


@pytest.mark.parametrize("coll", COLLS + [O.BGK, O.RLB])
@pytest.mark.parametrize("shape,periodic", [
    ((9, 10, 12), (1, 1, 1)),
    ((6, 11, 16), (1, 0, 1)),   # y walls
    ((5, 7, 10), (0, 0, 0)),    # closed box
])
def test_d3q27_fp64_walls_force(coll, shape, periodic):
    rng = np.random.default_rng(91)
    rho, u = W.random_macros(shape, 3, rng, umax=0.05)
    F = (2e-5, -1e-5, 1.5e-5)
    g = gpu_lattice(LAT, shape, coll, 0.02, 3 / 16, force=F, periodic=periodic)
    g.init_equilibrium(rho, u)
    g.step(100)
    p = oracle_params(LAT, shape, coll, 0.02, 3 / 16, force=F, periodic=periodic)
    ref = O.step(p, O.init_equilibrium(p, rho, u), 100, nthreads=4)
    assert elem_rel(g.populations().cpu().numpy(), ref) < 1e-12
    assert g.status()[0] == 0


@pytest.mark.parametrize("coll", COLLS)
def test_d3q27_solid_mask_fp64(coll):
    shape = (8, 12, 16)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[2:6, 4:8, 5:9] = 1
    rng = np.random.default_rng(92)
    rho, u = W.random_macros(shape, 3, rng, umax=0.05)
    u = u * (solid == 0)
    g = gpu_lattice(LAT, shape, coll, 0.03, 0.25, periodic=(1, 0, 1), solid=solid)
    g.init_equilibrium(rho, u)
    g.step(60)
    p = oracle_params(LAT, shape, coll, 0.03, 0.25, periodic=(1, 0, 1), solid=solid)
    ref = O.step(p, O.init_equilibrium(p, rho, u), 60, nthreads=4)
    assert elem_rel(g.populations().cpu().numpy(), ref, solid) < 1e-12


@pytest.mark.parametrize("coll", COLLS)
def test_d3q27_fp32_rho_u_after_100_steps(coll):
    shape = (10, 13, 24)
    rng = np.random.default_rng(93)
    rho, u = W.random_macros(shape, 3, rng, umax=0.05)
    F = (1e-5, 0.0, -1e-5)
    g = gpu_lattice(LAT, shape, coll, 0.03, 0.25, storage="F32", force=F, periodic=(1, 0, 1))
    g.init_equilibrium(rho, u)
    g.step(100)
    r_gpu, u_gpu = (t.cpu().numpy() for t in g.macros())
    p = oracle_params(LAT, shape, coll, 0.03, 0.25, force=F, periodic=(1, 0, 1))
    r_ref, u_ref = O.macros(p, O.step(p, O.init_equilibrium(p, rho, u), 100, nthreads=4))
    assert elem_rel(r_gpu, r_ref) < 2e-5
    assert scaled_err(u_gpu, u_ref) < 2e-5


@pytest.mark.parametrize("shape,storage,periodic", [
    ((4, 5, 264), "F32", (1, 0, 1)),   # two 256-node tiles, the second ragged
    ((3, 6, 48), "F32", (0, 1, 0)),    # x and z walls, one tile
    ((4, 4, 272), "F16", (1, 1, 0)),   # adjacent node pairs, z walls
    ((3, 5, 130), "F64", (0, 1, 1)),   # unpacked, 128-node tiles, x walls
])
@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT_RLB])
def test_d3q27_pipelined_matches_register_variants_and_oracle(shape, storage, periodic, coll):
    rng = np.random.default_rng(94)
    rho, u = W.random_macros(shape, 3, rng, umax=0.05)
    F = (1e-5, 2e-6, -1e-5)
    g = gpu_lattice(LAT, shape, coll, 0.03, 0.25, storage=storage, force=F, periodic=periodic)
    names = g.variants()
    tma = [v for v, n in enumerate(names) if n.startswith("tma")]
    reg = [v for v, n in enumerate(names) if not n.startswith("tma")]
    assert tma and reg
    results = {}
    for v in tma + reg[:3]:
        g.variant = v
        g.init_equilibrium(rho, u)
        g.step(9)
        results[names[v]] = g.populations().cpu().numpy()
        assert g.status()[0] == 0
    ref = results[names[reg[0]]]
    for n, r in results.items():
        assert np.array_equal(r, ref), n
    p = oracle_params(LAT, shape, coll, 0.03, 0.25, force=F, periodic=periodic)
    want = O.step(p, O.init_equilibrium(p, rho, u), 9)
    tol = {"F64": 1e-12, "F32": 2e-6, "F16": 2e-3}[storage]
    assert elem_rel(ref, want) < tol


@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_d3q27_aa_layout_matches_ab(storage):
    """In place (AA, even and odd steps) gives the A/B bits after an odd and an
    even number of steps."""
    shape = (6, 7, 32)
    rng = np.random.default_rng(95)
    rho, u = W.random_macros(shape, 3, rng, umax=0.05)
    for steps in (7, 8):
        out = []
        for layout in ("AB", "AA"):
            g = gpu_lattice(LAT, shape, O.P_TRT, 0.03, 0.25, storage=storage,
                            force=(1e-5, 0, 0), periodic=(1, 0, 1), layout=layout)
            g.init_equilibrium(rho, u)
            g.step(steps)
            out.append(g.populations().cpu().numpy())
        assert np.array_equal(out[0], out[1]), steps


@pytest.mark.parametrize("coll", [O.P_TRT, O.TRT_RLB])
def test_d3q27_scheme2_matches_oracle(coll):
    shape = (5, 6, 20)
    rng = np.random.default_rng(96)
    rho, u = W.random_macros(shape, 3, rng, umax=0.06)
    F = (1e-6, 0.0, 2e-6)
    g = gpu_lattice(LAT, shape, coll, 0.03, 3 / 16, force=F, periodic=(1, 0, 1))
    g.set_forcing_scheme(2)
    g.init_equilibrium(rho, u)
    g.step(9)
    p = oracle_params(LAT, shape, coll, 0.03, 3 / 16, force=F, periodic=(1, 0, 1))
    want = O.step_s2(p, O.init_equilibrium(p, rho, u), 9, nthreads=4)
    assert elem_rel(g.populations().cpu().numpy(), want) < 1e-12


def test_d3q27_hybrid_differs_from_trt_rlb_by_the_fifth_order_residual():
    """Two steps from the same equilibrium state (the first collision sees no
    fneq): GPU hybrid minus GPU TRT-RLB equals the oracle's difference, which
    carries the (1 - w-) P5 fneq of the second collision (FP64)."""
    shape = (4, 5, 8)
    rng = np.random.default_rng(97)
    rho, u = W.random_macros(shape, 3, rng, umax=0.08)
    res = {}
    for coll in (O.P_TRT, O.TRT_RLB):
        g = gpu_lattice(LAT, shape, coll, 0.03, 0.25)
        g.init_equilibrium(rho, u)
        g.step(2)
        p = oracle_params(LAT, shape, coll, 0.03, 0.25)
        res[coll] = (g.populations().cpu().numpy(), O.step(p, O.init_equilibrium(p, rho, u), 2))
    d_gpu = res[O.P_TRT][0] - res[O.TRT_RLB][0]
    d_ref = res[O.P_TRT][1] - res[O.TRT_RLB][1]
    assert np.max(np.abs(d_ref)) > 1e-9
    assert np.max(np.abs(d_gpu - d_ref)) < 1e-12 * np.max(np.abs(res[O.P_TRT][1]))
