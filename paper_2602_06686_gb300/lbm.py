"""ctypes binding of ``include/lbm.h`` (argument marshalling only).

PyTorch supplies device memory and the CUDA stream; every step of the update
runs in the sm_103a kernels of ``_lib/liblbm.so``.  There is no fallback: if
the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbm.so")

LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"TRT": 0, "TRT_RLB": 1, "P_TRT": 2, "BGK": 3, "RLB": 4}
STORAGES = {"F64": 0, "F32": 1, "F16": 2, "BF16": 3}
LAYOUTS = {"AB": 0, "AA": 1}
Q_OF = {0: 9, 1: 19, 2: 27}
D_OF = {0: 2, 1: 3, 2: 3}

LBM_OK = 0
LBM_ERR_DIVERGED = -3
LBM_ERR_TIMEOUT = -4

EXPORTED = [
    "lbm_version", "lbm_strerror", "lbm_last_error", "lbm_buffer_sizes", "lbm_create",
    "lbm_bind_buffers", "lbm_init_equilibrium", "lbm_init_equilibrium_host", "lbm_step",
    "lbm_macros", "lbm_macros_host", "lbm_get_populations", "lbm_set_populations",
    "lbm_diagnostics", "lbm_velocity_l2", "lbm_status", "lbm_step_count", "lbm_checkpoint",
    "lbm_restore", "lbm_launch_count", "lbm_set_wait_limit", "lbm_variant_count", "lbm_variant_name",
    "lbm_get_variant", "lbm_set_variant", "lbm_autotune", "lbm_destroy", "lbm_copy_ceiling",
    "lbm_batch_buffer_sizes", "lbm_batch_create", "lbm_batch_bind", "lbm_batch_lattice",
    "lbm_batch_step", "lbm_batch_variant_count", "lbm_batch_variant_name",
    "lbm_batch_set_variant", "lbm_batch_autotune", "lbm_batch_set_barrier",
    "lbm_batch_launches", "lbm_batch_destroy", "lbm_diagnostics_noalloc",
    "lbm_set_open_boundaries", "lbm_momentum_exchange", "lbm_set_forcing_scheme",
]


class LBMError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {code} ({detail})")


class Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nu", ctypes.c_double), ("tau_plus", ctypes.c_double),
        ("Lambda", ctypes.c_double), ("tau_minus", ctypes.c_double),
        ("collision", ctypes.c_int),
        ("force", ctypes.c_double * 3),
        ("rho0", ctypes.c_double),
        ("periodic", ctypes.c_int * 3),
        ("storage", ctypes.c_int),
        ("layout", ctypes.c_int),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads liblbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2602_06686_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    ll = ctypes.POINTER(ctypes.c_longlong)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(Params)
    sig = {
        "lbm_version": ([], ctypes.c_int),
        "lbm_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "lbm_last_error": ([], ctypes.c_char_p),
        "lbm_buffer_sizes": ([pp, ctypes.POINTER(sz), ctypes.POINTER(sz)], ctypes.c_int),
        "lbm_create": ([pp, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "lbm_bind_buffers": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "lbm_init_equilibrium": ([vp, vp, vp], ctypes.c_int),
        "lbm_init_equilibrium_host": ([vp, dp, dp], ctypes.c_int),
        "lbm_step": ([vp, ctypes.c_int], ctypes.c_int),
        "lbm_macros": ([vp, vp, vp], ctypes.c_int),
        "lbm_macros_host": ([vp, dp, dp], ctypes.c_int),
        "lbm_get_populations": ([vp, vp], ctypes.c_int),
        "lbm_set_populations": ([vp, vp], ctypes.c_int),
        "lbm_diagnostics": ([vp, dp], ctypes.c_int),
        "lbm_velocity_l2": ([vp, vp, dp], ctypes.c_int),
        "lbm_status": ([vp, ll], ctypes.c_int),
        "lbm_step_count": ([vp, ll], ctypes.c_int),
        "lbm_checkpoint": ([vp, vp, sz, ll], ctypes.c_int),
        "lbm_restore": ([vp, vp, sz, ctypes.c_longlong], ctypes.c_int),
        "lbm_launch_count": ([vp, ll], ctypes.c_int),
        "lbm_set_wait_limit": ([vp, ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "lbm_variant_count": ([vp, ip], ctypes.c_int),
        "lbm_variant_name": ([vp, ctypes.c_int, ctypes.c_char_p, sz], ctypes.c_int),
        "lbm_get_variant": ([vp, ip], ctypes.c_int),
        "lbm_set_variant": ([vp, ctypes.c_int], ctypes.c_int),
        "lbm_autotune": ([vp, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "lbm_destroy": ([vp], ctypes.c_int),
        "lbm_copy_ceiling": ([vp, vp, sz, vp], ctypes.c_int),
        "lbm_batch_buffer_sizes": ([ctypes.c_int, pp, ctypes.POINTER(sz), ctypes.POINTER(sz)],
                                   ctypes.c_int),
        "lbm_batch_create": ([ctypes.c_int, pp, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "lbm_batch_bind": ([vp, vp, vp, vp], ctypes.c_int),
        "lbm_batch_lattice": ([vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "lbm_batch_step": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "lbm_batch_variant_count": ([vp, ip], ctypes.c_int),
        "lbm_batch_variant_name": ([vp, ctypes.c_int, ctypes.c_char_p, sz], ctypes.c_int),
        "lbm_batch_set_variant": ([vp, ctypes.c_int], ctypes.c_int),
        "lbm_batch_autotune": ([vp, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_float)],
                               ctypes.c_int),
        "lbm_batch_set_barrier": ([vp, ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "lbm_batch_launches": ([vp, ll], ctypes.c_int),
        "lbm_batch_destroy": ([vp], ctypes.c_int),
        "lbm_diagnostics_noalloc": ([pp, vp, vp, dp, ctypes.c_longlong, vp, vp], ctypes.c_int),
        "lbm_set_open_boundaries": ([vp, ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "lbm_momentum_exchange": ([vp, dp], ctypes.c_int),
        "lbm_set_forcing_scheme": ([vp, ctypes.c_int], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != LBM_OK:
        lib = load_library()
        raise LBMError(rc, what, (lib.lbm_strerror(rc) or b"").decode() + "; "
                       + (lib.lbm_last_error() or b"").decode())


def _code(table: dict, v):
    return table[v] if isinstance(v, str) else int(v)


def make_params(lattice="D2Q9", nx=64, ny=64, nz=1, nu=0.0, tau_plus=0.0, Lambda=0.0,
                tau_minus=0.0, collision="P_TRT", force=(0.0, 0.0, 0.0), rho0=1.0,
                periodic=(1, 1, 1), storage="F32", layout="AB") -> Params:
    p = Params()
    p.lattice = _code(LATTICES, lattice)
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.nu, p.tau_plus, p.Lambda, p.tau_minus = float(nu), float(tau_plus), float(Lambda), float(
        tau_minus)
    p.collision = _code(COLLISIONS, collision)
    for a in range(3):
        p.force[a] = float(force[a])
        p.periodic[a] = int(periodic[a])
    p.rho0 = float(rho0)
    p.storage = _code(STORAGES, storage)
    p.layout = _code(LAYOUTS, layout)
    return p


def buffer_sizes(p: Params):
    lib = load_library()
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib.lbm_buffer_sizes(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b)),
           "lbm_buffer_sizes")
    return a.value, b.value


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class Lattice:
    """One lattice bound to torch-allocated device buffers."""

    def __init__(self, solid=None, stream=None, **kw):
        import torch
        self.lib = load_library()
        self.p = make_params(**kw)
        self.Q = Q_OF[self.p.lattice]
        self.D = D_OF[self.p.lattice]
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = self.p.nx * self.p.ny * self.p.nz
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.pop_bytes, self.scratch_bytes = buffer_sizes(self.p)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.pop_a = torch.empty(self.pop_bytes, dtype=torch.uint8, device=dev)
        self.pop_b = (torch.empty(self.pop_bytes, dtype=torch.uint8, device=dev)
                      if self.p.layout == 0 else None)
        self.scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=dev)
        self.mask = None
        if solid is not None:
            m = torch.as_tensor(np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.shape))
            self.mask = m.to(dev).contiguous()
        self.ctx = ctypes.c_void_p()
        _check(self.lib.lbm_create(ctypes.byref(self.p), _stream_handle(self.stream),
                                   ctypes.byref(self.ctx)), "lbm_create")
        _check(self.lib.lbm_bind_buffers(
            self.ctx, _dev_ptr(self.pop_a),
            _dev_ptr(self.pop_b) if self.pop_b is not None else None,
            _dev_ptr(self.mask) if self.mask is not None else None,
            _dev_ptr(self.scratch)), "lbm_bind_buffers")

    # -- state
    def _dev64(self, a, shape):
        import torch
        if isinstance(a, np.ndarray) and not a.flags.writeable:
            a = a.copy()
        t = torch.as_tensor(a, dtype=torch.float64)
        return t.to(self.pop_a.device).reshape(shape).contiguous()

    def init_equilibrium(self, rho, u):
        self._keep = (self._dev64(rho, self.shape), self._dev64(u, (self.D,) + self.shape))
        _check(self.lib.lbm_init_equilibrium(self.ctx, _dev_ptr(self._keep[0]),
                                             _dev_ptr(self._keep[1])), "lbm_init_equilibrium")

    def init_equilibrium_host(self, rho: np.ndarray, u: np.ndarray):
        dp = ctypes.POINTER(ctypes.c_double)
        r = np.ascontiguousarray(rho, dtype=np.float64)
        v = np.ascontiguousarray(u, dtype=np.float64)
        assert r.size == self.N and v.size == self.D * self.N
        _check(self.lib.lbm_init_equilibrium_host(self.ctx, r.ctypes.data_as(dp),
                                                  v.ctypes.data_as(dp)),
               "lbm_init_equilibrium_host")

    def init_equilibrium_host_ptr(self, rho_ptr: int, u_ptr: int):
        """Host-pointer variant for pinned buffers (e.g. torch pin_memory tensors)."""
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self.lib.lbm_init_equilibrium_host(self.ctx, ctypes.cast(rho_ptr, dp),
                                                  ctypes.cast(u_ptr, dp)),
               "lbm_init_equilibrium_host")

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self.ctx, int(n)), "lbm_step")

    def macros(self):
        import torch
        rho = torch.empty(self.shape, dtype=torch.float64, device=self.pop_a.device)
        u = torch.empty((self.D,) + self.shape, dtype=torch.float64, device=self.pop_a.device)
        _check(self.lib.lbm_macros(self.ctx, _dev_ptr(rho), _dev_ptr(u)), "lbm_macros")
        return rho, u

    def macros_host(self, rho_out: np.ndarray | None = None, u_out: np.ndarray | None = None):
        dp = ctypes.POINTER(ctypes.c_double)
        rho = rho_out if rho_out is not None else np.empty(self.shape)
        u = u_out if u_out is not None else np.empty((self.D,) + self.shape)
        _check(self.lib.lbm_macros_host(self.ctx, rho.ctypes.data_as(dp), u.ctypes.data_as(dp)),
               "lbm_macros_host")
        return rho, u

    def macros_host_ptr(self, rho_ptr: int, u_ptr: int):
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self.lib.lbm_macros_host(self.ctx, ctypes.cast(rho_ptr, dp),
                                        ctypes.cast(u_ptr, dp)), "lbm_macros_host")

    def populations(self):
        import torch
        f = torch.empty((self.Q,) + self.shape, dtype=torch.float64, device=self.pop_a.device)
        _check(self.lib.lbm_get_populations(self.ctx, _dev_ptr(f)), "lbm_get_populations")
        return f

    def set_populations(self, f):
        self._keepf = self._dev64(f, (self.Q,) + self.shape)
        _check(self.lib.lbm_set_populations(self.ctx, _dev_ptr(self._keepf)),
               "lbm_set_populations")

    def diagnostics(self) -> dict:
        out = (ctypes.c_double * 8)()
        _check(self.lib.lbm_diagnostics(self.ctx, out), "lbm_diagnostics")
        return {"mass": out[0], "momentum": np.array(out[1:4]), "kinetic_energy": out[4],
                "enstrophy": out[5], "nan_flag": out[6], "step": int(out[7])}

    def set_open_boundaries(self, u_in: float, rho_out: float):
        """Moving-wall inlet (u_in, 0) at the left, Zou-He outlet (rho_out) at the
        right (D2Q9, A/B, x non-periodic); rho_out <= 0 turns them off."""
        _check(self.lib.lbm_set_open_boundaries(self.ctx, float(u_in), float(rho_out)),
               "lbm_set_open_boundaries")

    def set_forcing_scheme(self, scheme: int):
        """1: Guo source (default); 2: the simplified projection with the cubic
        correction G_i (Eq. source_simple, Eq. Gi), two launches per step."""
        _check(self.lib.lbm_set_forcing_scheme(self.ctx, int(scheme)), "lbm_set_forcing_scheme")

    def momentum_exchange(self) -> np.ndarray:
        """Force on the solid nodes by momentum exchange, FP64 (3 components)."""
        out = (ctypes.c_double * 3)()
        _check(self.lib.lbm_momentum_exchange(self.ctx, out), "lbm_momentum_exchange")
        return np.array(out[:])

    def velocity_l2(self, u_ref) -> float:
        ur = self._dev64(u_ref, (self.D,) + self.shape)
        out = ctypes.c_double()
        _check(self.lib.lbm_velocity_l2(self.ctx, _dev_ptr(ur), ctypes.byref(out)),
               "lbm_velocity_l2")
        return out.value

    def status(self):
        first = ctypes.c_longlong()
        rc = self.lib.lbm_status(self.ctx, ctypes.byref(first))
        if rc not in (LBM_OK, LBM_ERR_DIVERGED):
            _check(rc, "lbm_status")
        return rc, first.value

    @property
    def t(self) -> int:
        v = ctypes.c_longlong()
        _check(self.lib.lbm_step_count(self.ctx, ctypes.byref(v)), "lbm_step_count")
        return v.value

    @property
    def launches(self) -> int:
        v = ctypes.c_longlong()
        _check(self.lib.lbm_launch_count(self.ctx, ctypes.byref(v)), "lbm_launch_count")
        return v.value

    def checkpoint(self):
        import torch
        buf = torch.empty(self.pop_bytes, dtype=torch.uint8, device=self.pop_a.device)
        t = ctypes.c_longlong()
        _check(self.lib.lbm_checkpoint(self.ctx, _dev_ptr(buf), self.pop_bytes, ctypes.byref(t)),
               "lbm_checkpoint")
        return buf, t.value

    def restore(self, snap):
        buf, t = snap
        _check(self.lib.lbm_restore(self.ctx, _dev_ptr(buf), self.pop_bytes, int(t)),
               "lbm_restore")

    def set_wait_limit(self, seconds: float, test_extra_bytes: int = 0):
        _check(self.lib.lbm_set_wait_limit(self.ctx, float(seconds), int(test_extra_bytes)),
               "lbm_set_wait_limit")

    # -- kernel variants
    def variants(self):
        n = ctypes.c_int()
        _check(self.lib.lbm_variant_count(self.ctx, ctypes.byref(n)), "lbm_variant_count")
        names = []
        buf = ctypes.create_string_buffer(64)
        for v in range(n.value):
            _check(self.lib.lbm_variant_name(self.ctx, v, buf, 64), "lbm_variant_name")
            names.append(buf.value.decode())
        return names

    @property
    def variant(self) -> int:
        v = ctypes.c_int()
        _check(self.lib.lbm_get_variant(self.ctx, ctypes.byref(v)), "lbm_get_variant")
        return v.value

    @variant.setter
    def variant(self, v: int):
        _check(self.lib.lbm_set_variant(self.ctx, int(v)), "lbm_set_variant")

    def autotune(self, reps: int = 5, report: bool = True):
        n = len(self.variants())
        times = (ctypes.c_float * n)() if report else None
        chosen = ctypes.c_int()
        _check(self.lib.lbm_autotune(self.ctx, int(reps), ctypes.byref(chosen), times),
               "lbm_autotune")
        return chosen.value, (list(times) if report else None)

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.lbm_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _View(Lattice):
    """Lattice i of a Batch: shares the batch's arenas and scratch."""

    def __init__(self, batch, i, ctx, params):
        self.lib = batch.lib
        self.p = params
        self.Q = Q_OF[params.lattice]
        self.D = D_OF[params.lattice]
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self.stream = batch.stream
        self.pop_a = batch.pop_a  # for the device of temporaries
        self.ctx = ctx
        self._batch = batch

    def step(self, n: int = 1):
        raise RuntimeError("lattices of a batch advance together: use Batch.step")

    def close(self):
        self.ctx = ctypes.c_void_p()


class Batch:
    """Many independent lattices advanced by one persistent kernel."""

    def __init__(self, params: list, stream=None):
        import torch
        self.lib = load_library()
        self.n = len(params)
        arr = (Params * self.n)()
        for i, kw in enumerate(params):
            arr[i] = make_params(**kw)
        self.params = arr
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self.lib.lbm_batch_buffer_sizes(self.n, arr, ctypes.byref(a), ctypes.byref(b)),
               "lbm_batch_buffer_sizes")
        self.pop_bytes, self.scratch_bytes = a.value, b.value
        dev = torch.device("cuda", torch.cuda.current_device())
        self.pop_a = torch.empty(self.pop_bytes, dtype=torch.uint8, device=dev)
        self.pop_b = torch.empty(self.pop_bytes, dtype=torch.uint8, device=dev)
        self.scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=dev)
        self.h = ctypes.c_void_p()
        _check(self.lib.lbm_batch_create(self.n, arr, _stream_handle(self.stream),
                                         ctypes.byref(self.h)), "lbm_batch_create")
        _check(self.lib.lbm_batch_bind(self.h, _dev_ptr(self.pop_a), _dev_ptr(self.pop_b),
                                       _dev_ptr(self.scratch)), "lbm_batch_bind")
        self.views = []
        for i in range(self.n):
            v = ctypes.c_void_p()
            _check(self.lib.lbm_batch_lattice(self.h, i, ctypes.byref(v)), "lbm_batch_lattice")
            self.views.append(_View(self, i, v, arr[i]))

    @property
    def nodes(self) -> int:
        return sum(v.N for v in self.views)

    def lattice(self, i: int) -> Lattice:
        return self.views[i]

    def step(self, n: int, mode: int = 0):
        _check(self.lib.lbm_batch_step(self.h, int(n), int(mode)), "lbm_batch_step")

    def variants(self):
        n = ctypes.c_int()
        _check(self.lib.lbm_batch_variant_count(self.h, ctypes.byref(n)), "variant count")
        buf = ctypes.create_string_buffer(64)
        out = []
        for v in range(n.value):
            _check(self.lib.lbm_batch_variant_name(self.h, v, buf, 64), "variant name")
            out.append(buf.value.decode())
        return out

    def set_variant(self, v: int):
        _check(self.lib.lbm_batch_set_variant(self.h, int(v)), "lbm_batch_set_variant")

    def autotune(self, steps: int = 4):
        n = len(self.variants())
        times = (ctypes.c_float * n)()
        chosen = ctypes.c_int()
        _check(self.lib.lbm_batch_autotune(self.h, int(steps), ctypes.byref(chosen), times),
               "lbm_batch_autotune")
        return chosen.value, list(times)

    def set_barrier(self, timeout_s: float, extra: int = 0):
        _check(self.lib.lbm_batch_set_barrier(self.h, float(timeout_s), int(extra)),
               "lbm_batch_set_barrier")

    @property
    def launches(self) -> int:
        v = ctypes.c_longlong()
        _check(self.lib.lbm_batch_launches(self.h, ctypes.byref(v)), "lbm_batch_launches")
        return v.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            for v in self.views:
                v.close()
            self.lib.lbm_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def copy_ceiling(src, dst, nbytes: int, stream=None):
    lib = load_library()
    _check(lib.lbm_copy_ceiling(_dev_ptr(src), _dev_ptr(dst), int(nbytes), _stream_handle(stream)),
           "lbm_copy_ceiling")
