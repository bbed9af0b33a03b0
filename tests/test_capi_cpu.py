"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/lbm.h, and its host-only calls (parameter validation,
buffer plan, error strings) behave as documented.  No GPU compute is called."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_06686_gb300 import build, lbm
    build.build()
    return lbm.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2602_06686_gb300 import lbm
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.EXPORTED) == names


def test_version_and_strerror(lib):
    assert lib.lbm_version() >= 100
    for code in range(0, -8, -1):
        assert lib.lbm_strerror(code)
    assert b"unknown" in lib.lbm_strerror(-99)


def test_buffer_plan(lib):
    from paper_2602_06686_gb300.lbm import buffer_sizes, make_params
    pop, scr = buffer_sizes(make_params("D2Q9", 64, 64, nu=0.01, Lambda=0.25, storage="F64"))
    assert pop == 9 * 64 * 64 * 8
    pop, _ = buffer_sizes(make_params("D2Q9", 4096, 4096, nu=0.004, Lambda=0.25, storage="F32"))
    assert pop == 9 * 4096 * 4096 * 4
    # rows padded to 16 bytes, planes to 256 bytes
    pop, _ = buffer_sizes(make_params("D3Q19", 30, 7, 5, nu=0.01, Lambda=0.25, storage="F16"))
    plane = ((32 * 7 * 5 + 127) // 128) * 128
    assert pop == 19 * plane * 2
    _, scr = buffer_sizes(make_params("D3Q19", 10, 10, 10, nu=0.01, Lambda=0.25))
    assert scr >= 4 * 1000 * 8
    # D3Q27: 27 planes; the scratch field area also holds the Scheme II rho u^3 field
    pop, scr = buffer_sizes(make_params("D3Q27", 24, 6, 5, nu=0.01, Lambda=0.25, storage="F32"))
    plane = ((24 * 6 * 5 + 63) // 64) * 64
    assert pop == 27 * plane * 4
    assert scr >= 4 * 24 * 6 * 5 * 8


@pytest.mark.parametrize("kw", [
    dict(lattice="D2Q9", nx=8, ny=8, nz=2),
    dict(lattice="D2Q9", nx=0, ny=8),
    dict(lattice="D2Q9", nx=8, ny=8, tau_plus=0.8),          # nu and tau_plus both given
    dict(lattice="D2Q9", nx=8, ny=8, Lambda=0.0),            # neither Lambda nor tau_minus
    dict(lattice="D2Q9", nx=8, ny=8, collision=7),
    dict(lattice="D2Q9", nx=8, ny=8, storage=9),
    dict(lattice="D2Q9", nx=8, ny=8, rho0=0.0),
    dict(lattice="D2Q9", nx=8, ny=8, force=(0, 0, 1e-3)),
    dict(lattice="D2Q9", nx=8, ny=8, periodic=(2, 1, 1)),
    dict(lattice=3, nx=8, ny=8, nz=8),                        # no fourth lattice
])
def test_invalid_parameters_rejected(lib, kw):
    from paper_2602_06686_gb300.lbm import LBMError, buffer_sizes, make_params
    base = dict(nu=0.05, Lambda=0.25)
    base.update(kw)
    with pytest.raises(LBMError) as e:
        buffer_sizes(make_params(**base))
    assert e.value.code == -1


def test_null_handles_and_outputs_are_argument_errors():
    """Every entry point given a NULL context, batch, parameter block or
    required output returns LBM_ERR_ARG before any CUDA call (this machine may
    have no GPU); destroying NULL is a no-op."""
    import ctypes

    from paper_2602_06686_gb300 import build
    raw = ctypes.CDLL(build.build())  # no argtypes: every argument spelled out
    d, sz, ll = ctypes.c_double, ctypes.c_size_t, ctypes.c_longlong
    calls = {
        "lbm_buffer_sizes": (None, None, None),
        "lbm_create": (None, None, None),
        "lbm_bind_buffers": (None, None, None, None, None),
        "lbm_init_equilibrium": (None, None, None),
        "lbm_init_equilibrium_host": (None, None, None),
        "lbm_step": (None, 1),
        "lbm_macros": (None, None, None),
        "lbm_macros_host": (None, None, None),
        "lbm_get_populations": (None, None),
        "lbm_set_populations": (None, None),
        "lbm_diagnostics": (None, None),
        "lbm_velocity_l2": (None, None, None),
        "lbm_set_open_boundaries": (None, d(0.01), d(1.0)),
        "lbm_set_forcing_scheme": (None, 2),
        "lbm_momentum_exchange": (None, None),
        "lbm_status": (None, None),
        "lbm_diagnostics_noalloc": (None, None, None, None, ll(0), None, None),
        "lbm_step_count": (None, None),
        "lbm_checkpoint": (None, None, sz(0), None),
        "lbm_restore": (None, None, sz(0), ll(0)),
        "lbm_launch_count": (None, None),
        "lbm_set_wait_limit": (None, d(1.0), 0),
        "lbm_variant_count": (None, None),
        "lbm_variant_name": (None, 0, None, sz(0)),
        "lbm_get_variant": (None, None),
        "lbm_set_variant": (None, 0),
        "lbm_autotune": (None, 1, None, None),
        "lbm_copy_ceiling": (None, None, sz(16), None),
        "lbm_batch_buffer_sizes": (0, None, None, None),
        "lbm_batch_create": (0, None, None, None),
        "lbm_batch_bind": (None, None, None, None),
        "lbm_batch_lattice": (None, 0, None),
        "lbm_batch_step": (None, 1, 0),
        "lbm_batch_variant_count": (None, None),
        "lbm_batch_variant_name": (None, 0, None, sz(0)),
        "lbm_batch_set_variant": (None, 0),
        "lbm_batch_autotune": (None, 1, None, None),
        "lbm_batch_set_barrier": (None, d(1.0), 0),
        "lbm_batch_launches": (None, None),
    }
    raw.lbm_last_error.restype = ctypes.c_char_p
    for name, args in calls.items():
        assert getattr(raw, name)(*args) == -1, name
        assert raw.lbm_last_error(), name
    assert raw.lbm_destroy(None) == 0
    assert raw.lbm_batch_destroy(None) == 0
    # every entry point that takes a handle or a parameter block is covered
    takes_handle = {n for n in _declared()
                    if n not in ("lbm_version", "lbm_strerror", "lbm_last_error",
                                 "lbm_destroy", "lbm_batch_destroy")}
    assert takes_handle == set(calls)


def test_noalloc_diagnostics_refuses_misaligned_buffers(lib):
    """The no-scratch diagnostics checks the alignment lbm_bind_buffers asks
    of the state and mask (256 bytes) and of its FP64 output (8 bytes) before
    any CUDA call; the addresses are never dereferenced here."""
    import ctypes

    from paper_2602_06686_gb300.lbm import make_params
    p = make_params("D2Q9", 64, 64, nu=0.01, Lambda=0.25, storage="F32")
    base = 1 << 20  # a 256-byte aligned address value
    cases = [(base + 16, None, base), (base, base + 1, base), (base, None, base + 4)]
    for state, mask, out in cases:
        rc = lib.lbm_diagnostics_noalloc(ctypes.byref(p), ctypes.c_void_p(state), ctypes.c_void_p(mask),
                                         None, 0, ctypes.c_void_p(out), None)
        assert rc == -7, (state, mask, out)
    # a lattice beyond the static array's capacity is refused first by size
    big = make_params("D2Q9", 1024, 1024, nu=0.01, Lambda=0.25, storage="F32")
    assert lib.lbm_diagnostics_noalloc(ctypes.byref(big), ctypes.c_void_p(base), None, None, 0,
                                       ctypes.c_void_p(base), None) == -1
