"""GPU tests of the batched driver: many uneven lattices advanced by one
persistent cooperative kernel (replayed from a CUDA graph) must give, bit for
bit, what each lattice gives when run alone, in every tile shape and in the
sequential one-launch-per-lattice mode; FP64 batches match the oracle; a grid
barrier that cannot complete returns an error status instead of hanging."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _specs(count, seed, storage="F32", side=(40, 130)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx, ny = (int(v) for v in rng.integers(side[0], side[1] + 1, 2))
        Re = float(10 ** rng.uniform(3, 5))
        lam = float(rng.choice([1 / 12, 3 / 16, 0.25]))
        out.append(dict(lattice="D2Q9", nx=nx, ny=ny, nu=0.1 * nx / Re, Lambda=lam,
                        collision="P_TRT", storage=storage))
    return out


def _init(batch, specs):
    fields = []
    for i, s in enumerate(specs):
        rho, u = W.double_shear_rect(s["nx"], s["ny"])
        batch.lattice(i).init_equilibrium(rho, u)
        fields.append((rho, u))
    return fields


def _alone(spec, fields, steps):
    from paper_2602_06686_gb300 import Lattice
    g = Lattice(**spec)
    g.init_equilibrium(*fields)
    g.step(steps)
    return g.populations().cpu().numpy()


@pytest.mark.parametrize("steps", [1, 8, 13])
def test_persistent_batch_equals_single_runs(steps):
    from paper_2602_06686_gb300 import Batch
    specs = _specs(7, 51)
    b = Batch(specs)
    fields = _init(b, specs)
    b.step(steps, mode=0)
    assert b.launches == 1
    for i, s in enumerate(specs):
        got = b.lattice(i).populations().cpu().numpy()
        assert np.array_equal(got, _alone(s, fields[i], steps)), i
        assert b.lattice(i).t == steps


def test_sequential_mode_and_tile_shapes_agree():
    from paper_2602_06686_gb300 import Batch
    specs = _specs(5, 52)
    b = Batch(specs)
    ref = None
    for v in range(len(b.variants())):
        b.set_variant(v)
        _init(b, specs)
        b.step(6, mode=0)
        b.step(5, mode=0)
        got = [b.lattice(i).populations().cpu().numpy() for i in range(len(specs))]
        if ref is None:
            ref = got
        for i in range(len(specs)):
            assert np.array_equal(got[i], ref[i]), (v, i)
    _init(b, specs)
    b.step(11, mode=1)
    assert b.launches == 11 * len(specs)
    for i in range(len(specs)):
        assert np.array_equal(b.lattice(i).populations().cpu().numpy(), ref[i])


@pytest.mark.parametrize("lat,storage,periodic,forced", [
    ("D2Q9", "F16", (1, 0, 1), True),     # walls in y, some lattices forced
    ("D2Q9", "BF16", (0, 1, 1), False),   # walls in x (row ends read from HBM)
    ("D3Q19", "F32", (0, 1, 0), True),    # walls in x and z
    ("D3Q19", "F16", (1, 1, 1), False),
    ("D3Q27", "F32", (1, 0, 1), True),    # walls in y
    ("D3Q27", "BF16", (0, 1, 1), False),
])
def test_every_batch_variant_equals_single_runs(lat, storage, periodic, forced):
    """Every variant of the batched kernel (pipelined and register tiles, any
    extent, unaligned periodic row ends, walls, per-lattice forces) gives what
    each lattice gives alone (comparison up to the sign of zero: unforced
    kernels skip adding zero force terms)."""
    from paper_2602_06686_gb300 import Batch
    rng = np.random.default_rng(56)
    specs = []
    for k in range(5):
        if lat == "D2Q9":
            nx, ny, nz = int(rng.integers(20, 140)), int(rng.integers(6, 40)), 1
        else:
            nx, ny, nz = int(rng.integers(9, 70)), int(rng.integers(4, 12)), int(rng.integers(3, 9))
        F = (2e-5 * (k % 2), -1e-5 * (k % 2), 1e-5 * (k % 2) if lat != "D2Q9" else 0.0)
        specs.append(dict(lattice=lat, nx=nx, ny=ny, nz=nz, nu=0.02 + 0.01 * k, Lambda=3 / 16,
                          collision="P_TRT", storage=storage, periodic=periodic,
                          force=F if forced else (0.0, 0.0, 0.0)))
    fields = []
    for s in specs:
        shape = (s["nz"], s["ny"], s["nx"])
        fields.append(W.random_macros(shape, 2 if lat == "D2Q9" else 3, rng, umax=0.05))
    alone = []
    from paper_2602_06686_gb300 import Lattice
    for s, fl in zip(specs, fields):
        g = Lattice(**s)
        g.init_equilibrium(*fl)
        g.step(7)
        alone.append(g.populations().cpu().numpy())
    b = Batch(specs)
    names = b.variants()
    assert any(n.startswith("tma") for n in names)
    for v, name in enumerate(names):
        b.set_variant(v)
        for i, fl in enumerate(fields):
            b.lattice(i).init_equilibrium(*fl)
        b.step(7, mode=0)
        for i in range(len(specs)):
            got = b.lattice(i).populations().cpu().numpy()
            assert np.array_equal(got, alone[i]), (name, i)
            assert b.lattice(i).status()[0] == 0, (name, i)


def test_fp64_batch_matches_oracle():
    from paper_2602_06686_gb300 import Batch
    specs = _specs(3, 53, storage="F64", side=(20, 40))
    b = Batch(specs)
    fields = _init(b, specs)
    b.step(30)
    for i, s in enumerate(specs):
        wp, wm = O.rates(nu=s["nu"], Lambda=s["Lambda"])
        p = O.Params(O.D2Q9, s["nx"], s["ny"], 1, collision=O.P_TRT, omega_plus=wp,
                     omega_minus=wm)
        ref = O.step(p, O.init_equilibrium(p, *fields[i]), 30)
        got = b.lattice(i).populations().cpu().numpy()
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12
        d = b.lattice(i).diagnostics()
        assert d["step"] == 30 and d["nan_flag"] == 0


def test_barrier_timeout_returns_error_and_context_recovers():
    """The barrier waits for one arrival that never comes: every block gives up
    after the limit (0.3 s), the call reports LBM_ERR_TIMEOUT, and the batch runs
    normally again afterwards."""
    from paper_2602_06686_gb300 import Batch, LBMError
    specs = _specs(3, 54)
    b = Batch(specs)
    fields = _init(b, specs)
    b.set_barrier(0.3, extra=1)
    with pytest.raises(LBMError) as e:
        b.step(3, mode=0)
    assert e.value.code == -4
    b.set_barrier(2.0, extra=0)
    _init(b, specs)
    b.step(4, mode=0)
    for i, s in enumerate(specs):
        assert np.array_equal(b.lattice(i).populations().cpu().numpy(),
                              _alone(s, fields[i], 4))


def test_batch_autotune_and_view_diagnostics():
    from paper_2602_06686_gb300 import Batch
    specs = _specs(4, 55)
    b = Batch(specs)
    _init(b, specs)
    chosen, times = b.autotune(steps=4)
    assert 0 <= chosen < len(b.variants()) and all(t > 0 for t in times)
    _init(b, specs)
    b.step(10)
    for i in range(len(specs)):
        d = b.lattice(i).diagnostics()
        assert d["nan_flag"] == 0 and d["step"] == 10
        assert b.lattice(i).status()[0] == 0
    with pytest.raises(RuntimeError):
        b.lattice(0).step(1)
