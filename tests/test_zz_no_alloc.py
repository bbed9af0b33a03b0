"""The allocation-free diagnostics entry point, for callers that cannot give
the library a scratch buffer (their device memory belongs to someone else's
pool, or they must not change a running simulation's footprint).  It must
return what lbm_diagnostics returns for the same state, on two calls in a row
(the fixed working array is reused and keeps the previous call's contents), and
refuse lattices larger than its fixed capacity.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    # lattice, shape (nz, ny, nx), storage, layout, periodic, force, solid block
    ("D2Q9", (1, 96, 128), "F32", "AB", (1, 1, 1), (0.0, 0.0, 0.0), False),
    ("D2Q9", (1, 60, 80), "F64", "AA", (1, 0, 1), (1e-5, 0.0, 0.0), True),
    ("D3Q19", (12, 16, 20), "F32", "AB", (1, 0, 1), (1e-5, 0.0, 0.0), False),
    ("D3Q19", (10, 12, 16), "F16", "AA", (1, 1, 1), (0.0, 0.0, 0.0), True),
]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


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
    stream = ctypes.c_void_p(g.stream.cuda_stream)
    for steps in (6, 5):  # an even then an odd step count (A/B buffer, AA parity)
        g.step(steps)
        t = g.t
        state = g.pop_a if (layout == "AA" or t % 2 == 0) else g.pop_b
        rc = lib.lbm_diagnostics_noalloc(ctypes.byref(g.p), _ptr(state),
                                         _ptr(g.mask) if g.mask is not None else None, t,
                                         _ptr(out), stream)
        assert rc == 0, lib.lbm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = g.diagnostics()
        for k, idx in (("mass", 0), ("kinetic_energy", 4), ("enstrophy", 5)):
            assert got[idx] == pytest.approx(ref[k], rel=1e-12), k
        assert np.allclose(got[1:4], ref["momentum"], rtol=1e-10, atol=1e-12)
        assert got[6] == ref["nan_flag"] == 0
        assert got[7] == t == ref["step"]


def test_rejects_lattices_beyond_capacity():
    import torch
    from paper_2602_06686_gb300.lbm import LBMError, _check, load_library, make_params
    lib = load_library()
    p = make_params("D2Q9", 1024, 512, nu=0.01, Lambda=0.25, storage="F32")
    dummy = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(p), _ptr(dummy), None, 0, _ptr(out), None)
    assert rc == -1
    assert b"262144" in lib.lbm_last_error()
    with pytest.raises(LBMError):
        _check(rc, "lbm_diagnostics_noalloc")
