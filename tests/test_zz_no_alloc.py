"""The allocation-free diagnostics entry point, for callers that cannot give
the library a scratch buffer (their device memory belongs to someone else's
pool, or they must not change a running simulation's footprint).  It must
return what lbm_diagnostics returns for the same state -- the same bits, since
both run the same kernels with the same reduction order -- on two calls in a
row (the fixed working array is reused and keeps the previous call's
contents), apply the open boundaries when told to, and refuse lattices larger
than its fixed capacity.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CAPACITY = 262144

CASES = [
    # lattice, shape (nz, ny, nx), storage, layout, periodic, force, solid block
    ("D2Q9", (1, 96, 128), "F32", "AB", (1, 1, 1), (0.0, 0.0, 0.0), False),
    ("D2Q9", (1, 60, 80), "F64", "AA", (1, 0, 1), (1e-5, 0.0, 0.0), True),
    ("D3Q19", (12, 16, 20), "F32", "AB", (1, 0, 1), (1e-5, 0.0, 0.0), False),
    ("D3Q19", (10, 12, 16), "F16", "AA", (1, 1, 1), (0.0, 0.0, 0.0), True),
    # exactly at capacity: the last velocity plane ends at the end of the array
    ("D2Q9", (1, 512, 512), "F64", "AB", (1, 1, 1), (0.0, 0.0, 0.0), False),
    ("D3Q27", (64, 64, 64), "BF16", "AB", (1, 0, 1), (0.0, 1e-5, 0.0), False),
]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _state(g):
    """The buffer holding the current state (A/B: the one the next step reads)."""
    return g.pop_a if (g.p.layout == 1 or g.t % 2 == 0) else g.pop_b


def _noalloc(lib, g, out, open_bc=None):
    ob = None if open_bc is None else (ctypes.c_double * 2)(*open_bc)
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(g.p), _ptr(_state(g)),
                                     _ptr(g.mask) if g.mask is not None else None, ob, g.t,
                                     _ptr(out), ctypes.c_void_p(g.stream.cuda_stream))
    assert rc == 0, lib.lbm_last_error()


def _same_as_diagnostics(got, ref, t):
    assert got[0] == ref["mass"]
    assert np.array_equal(got[1:4], ref["momentum"])
    assert got[4] == ref["kinetic_energy"]
    assert got[5] == ref["enstrophy"]
    assert got[6] == ref["nan_flag"] == 0
    assert got[7] == t == ref["step"]


@pytest.mark.parametrize("lat,shape,storage,layout,periodic,force,solid", CASES)
def test_matches_lbm_diagnostics_on_two_calls(lat, shape, storage, layout, periodic, force, solid):
    import torch
    from paper_2602_06686_gb300 import Lattice
    from paper_2602_06686_gb300.lbm import load_library
    lib = load_library()
    nz, ny, nx = shape
    mask = None
    if solid:
        mask = np.zeros(shape, dtype=np.uint8)
        mask[:, ny // 3:ny // 3 + 4, nx // 3:nx // 3 + 5] = 1
    rng = np.random.default_rng(61)
    D = 2 if lat == "D2Q9" else 3
    rho, u = W.random_macros(shape, D, rng, umax=0.05)
    g = Lattice(lattice=lat, nx=nx, ny=ny, nz=nz, nu=0.03, Lambda=0.25, collision="P_TRT",
                storage=storage, layout=layout, periodic=periodic, force=force, solid=mask)
    g.init_equilibrium(rho, u)
    out = torch.full((8,), -7.0, dtype=torch.float64, device="cuda")
    for steps in (6, 5):  # an even then an odd step count (A/B buffer, AA parity)
        g.step(steps)
        _noalloc(lib, g, out)
        torch.cuda.synchronize()
        _same_as_diagnostics(out.cpu().numpy(), g.diagnostics(), g.t)


def test_open_boundaries_as_lbm_diagnostics():
    """A lattice stepped with the moving-wall inlet and Zou-He outlet: with
    open_bc the values equal lbm_diagnostics' (which applies the boundary rules
    to the gathered state); without it they differ; for the state just written
    (not yet streamed) lbm_diagnostics applies no rule and open_bc = NULL
    matches it."""
    import torch
    from paper_2602_06686_gb300 import Lattice
    from paper_2602_06686_gb300.lbm import load_library
    lib = load_library()
    shape = (1, 24, 48)
    solid = np.zeros(shape, dtype=np.uint8)
    solid[0, 9:15, 16:22] = 1
    rng = np.random.default_rng(83)
    rho, u = W.random_macros(shape, 2, rng, umax=0.02)
    u = u * (solid == 0)
    g = Lattice(lattice="D2Q9", nx=48, ny=24, nz=1, nu=0.05, Lambda=3 / 16, collision="P_TRT",
                storage="F64", periodic=(0, 1, 1), solid=solid)
    g.set_open_boundaries(0.03, 0.99)
    g.init_equilibrium(rho, u)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    _noalloc(lib, g, out)
    torch.cuda.synchronize()
    _same_as_diagnostics(out.cpu().numpy(), g.diagnostics(), 0)
    for steps in (40, 7):
        g.step(steps)
        _noalloc(lib, g, out, open_bc=(0.03, 0.99))
        torch.cuda.synchronize()
        ref = g.diagnostics()
        _same_as_diagnostics(out.cpu().numpy(), ref, g.t)
        _noalloc(lib, g, out)
        torch.cuda.synchronize()
        assert out.cpu().numpy()[0] != ref["mass"]


def test_rejects_lattices_beyond_capacity_and_bad_open_boundaries():
    import torch
    from paper_2602_06686_gb300.lbm import LBMError, _check, load_library, make_params
    lib = load_library()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    # one node beyond the capacity (5 x 52429 = 262145)
    p = make_params("D2Q9", 5, 52429, nu=0.01, Lambda=0.25, storage="F32")
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(p), _ptr(dummy), None, None, 0, _ptr(out), None)
    assert rc == -1
    assert str(CAPACITY).encode() in lib.lbm_last_error()
    with pytest.raises(LBMError):
        _check(rc, "lbm_diagnostics_noalloc")
    # open boundaries need a non-periodic x axis (and D2Q9, A/B)
    ob = (ctypes.c_double * 2)(0.03, 0.99)
    p = make_params("D2Q9", 32, 16, nu=0.01, Lambda=0.25, storage="F32")
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(p), _ptr(dummy), None, ob, 1, _ptr(out), None)
    assert rc == -1
    p3 = make_params("D3Q19", 8, 4, 4, nu=0.01, Lambda=0.25, storage="F32", periodic=(0, 1, 1))
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(p3), _ptr(dummy), None, ob, 1, _ptr(out), None)
    assert rc == -5
