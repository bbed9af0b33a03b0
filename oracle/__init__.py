"""FP64 CPU oracle of the P-TRT lattice Boltzmann update (arXiv 2602.06686).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
CUDA library never links, loads or calls it, and this package imports nothing
from the CUDA side.

The arithmetic lives in ``oracle.c`` (plain C, FP64, node by node, generic
tables); this module only builds it with gcc and marshals numpy arrays.

Array conventions: populations ``f`` have shape ``(Q, nz, ny, nx)`` (x fastest),
density ``(nz, ny, nx)``, velocity ``(D, nz, ny, nx)``; 2-D lattices use nz = 1.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, printed tables, theorems or brute force (see each test's
docstring).  The FP16/BF16 storage error budget has no pin in the paper and is
reported, not asserted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
TRT, TRT_RLB, P_TRT, BGK, RLB = 0, 1, 2, 3, 4
COLLISIONS = {"TRT": TRT, "TRT_RLB": TRT_RLB, "P_TRT": P_TRT, "BGK": BGK, "RLB": RLB}
Q_OF = {D2Q9: 9, D3Q19: 19, D3Q27: 27}
D_OF = {D2Q9: 2, D3Q19: 3, D3Q27: 3}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, FP64, no FMA contraction
    so that x86 and Arm hosts give bit-identical results)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(_CParams)
        lib.oracle_lattice_info.argtypes = [ctypes.c_int, ip, ip, ip, ip, dp, ip, dp, dp]
        lib.oracle_hermite.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_rates.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        lib.oracle_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        lib.oracle_collide.argtypes = [pp, dp, dp]
        lib.oracle_collide_many.argtypes = [pp, ctypes.c_int, dp, dp]
        lib.oracle_init_equilibrium.argtypes = [pp, dp, dp, dp]
        lib.oracle_step.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_macros.argtypes = [pp, dp, dp, dp]
        lib.oracle_diagnostics.argtypes = [pp, dp, dp]
        lib.oracle_l2.argtypes = [ctypes.c_long, dp, dp]
        lib.oracle_l2.restype = ctypes.c_double
        lib.oracle_hermite_contraction.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.oracle_hermite_ranks.argtypes = [ctypes.c_int, ip, ip]
        lib.oracle_step_open.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_momentum_exchange.argtypes = [pp, dp, dp]
        lib.oracle_cubic_flux_gradient.argtypes = [pp, dp, dp]
        lib.oracle_collide_s2.argtypes = [pp, dp, dp, dp]
        lib.oracle_step_s2.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_fifth_order_projection.argtypes = [ctypes.c_int, dp, dp]
        _lib = lib
    return _lib


class _CParams(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("omega_plus", ctypes.c_double),
        ("omega_minus", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("solid", ctypes.POINTER(ctypes.c_uint8)),
    ]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """One lattice run.  ``omega_plus`` = 1/tau_s1, ``omega_minus`` = 1/tau_s2."""
    lattice: int
    nx: int
    ny: int
    nz: int = 1
    collision: int = P_TRT
    omega_plus: float = 1.0
    omega_minus: float = 1.0
    force: tuple = (0.0, 0.0, 0.0)
    periodic: tuple = (1, 1, 1)
    solid: np.ndarray | None = None  # uint8 (nz, ny, nx), nonzero = solid
    _keep: list = field(default_factory=list, repr=False)

    @property
    def Q(self) -> int:
        return Q_OF[self.lattice]

    @property
    def D(self) -> int:
        return D_OF[self.lattice]

    @property
    def shape(self) -> tuple:
        return (self.nz, self.ny, self.nx)

    def c(self) -> _CParams:
        p = _CParams()
        p.lattice = self.lattice
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.collision = self.collision
        for a in range(3):
            p.periodic[a] = int(self.periodic[a])
            p.force[a] = float(self.force[a])
        p.omega_plus = self.omega_plus
        p.omega_minus = self.omega_minus
        if self.solid is not None:
            s = np.ascontiguousarray(self.solid, dtype=np.uint8).reshape(self.shape)
            self._keep[:] = [s]
            p.solid = s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        else:
            p.solid = None
        return p


def lattice_info(lattice: int) -> dict:
    lib = _load()
    Q = Q_OF[lattice]
    D, Qo, NG = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    phi = np.zeros((7, Q))
    nrm = np.zeros(7)
    rc = lib.oracle_lattice_info(lattice, ctypes.byref(D), ctypes.byref(Qo), ctypes.byref(NG),
                                 e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                                 opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(phi),
                                 _dp(nrm))
    if rc:
        raise RuntimeError(f"oracle_lattice_info failed: {rc}")
    ng = NG.value
    return {"D": D.value, "Q": Qo.value, "NG": ng, "e": e.astype(np.int64), "w": w,
            "opp": opp.astype(np.int64), "phi": phi[:ng].copy(), "phinorm": nrm[:ng].copy()}


def hermite(lattice: int):
    lib = _load()
    Q = Q_OF[lattice]
    H2 = np.zeros((Q, 3, 3))
    H3 = np.zeros((Q, 3, 3, 3))
    if lib.oracle_hermite(lattice, _dp(H2), _dp(H3)):
        raise RuntimeError("oracle_hermite failed")
    return H2, H3


def hermite_contraction(lattice: int, g: np.ndarray):
    """The literal contractions w H2:A2/(2cs^4), w H3:A3/(6cs^6) of Eq. R2R3_hermite."""
    lib = _load()
    g = np.ascontiguousarray(g, dtype=np.float64)
    r2, r3 = np.zeros_like(g), np.zeros_like(g)
    if lib.oracle_hermite_contraction(lattice, _dp(g), _dp(r2), _dp(r3)):
        raise RuntimeError("oracle_hermite_contraction failed")
    return r2, r3


def fifth_order_projection(lattice: int, g: np.ndarray) -> np.ndarray:
    """P^(5) g on D3Q27: projection onto the fifth-order antisymmetric modes of
    App. D3Q27 (the residual the hybrid P-TRT keeps in R3)."""
    lib = _load()
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(g)
    if lib.oracle_fifth_order_projection(lattice, _dp(g), _dp(out)):
        raise RuntimeError("oracle_fifth_order_projection failed")
    return out


def hermite_ranks(lattice: int):
    lib = _load()
    n2, n3 = ctypes.c_int(), ctypes.c_int()
    if lib.oracle_hermite_ranks(lattice, ctypes.byref(n2), ctypes.byref(n3)):
        raise RuntimeError("oracle_hermite_ranks failed")
    return n2.value, n3.value


def rates(nu: float = 0.0, tau_plus: float = 0.0, Lambda: float = 0.0,
          tau_minus: float = 0.0):
    """(omega_plus, omega_minus) from (nu or tau+) and (Lambda or tau-)."""
    lib = _load()
    wp, wm = ctypes.c_double(), ctypes.c_double()
    if lib.oracle_rates(nu, tau_plus, Lambda, tau_minus, ctypes.byref(wp), ctypes.byref(wm)):
        raise ValueError("invalid relaxation parameters")
    return wp.value, wm.value


def equilibrium(lattice: int, rho: float, u) -> np.ndarray:
    lib = _load()
    u3 = np.zeros(3)
    u3[:len(u)] = u
    feq = np.zeros(Q_OF[lattice])
    if lib.oracle_equilibrium(lattice, float(rho), _dp(u3), _dp(feq)):
        raise RuntimeError("oracle_equilibrium failed")
    return feq


def collide(p: Params, f: np.ndarray) -> np.ndarray:
    """Post-collision populations of one node (shape (Q,)) or many ((n, Q))."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    cp = p.c()
    if f.ndim == 1:
        rc = lib.oracle_collide(ctypes.byref(cp), _dp(f), _dp(out))
    else:
        rc = lib.oracle_collide_many(ctypes.byref(cp), f.shape[0], _dp(f), _dp(out))
    if rc:
        raise RuntimeError(f"oracle_collide failed: {rc}")
    return out


def init_equilibrium(p: Params, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    lib = _load()
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(p.shape)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape((p.D,) + p.shape)
    f = np.zeros((p.Q,) + p.shape)
    cp = p.c()
    if lib.oracle_init_equilibrium(ctypes.byref(cp), _dp(rho), _dp(u), _dp(f)):
        raise RuntimeError("oracle_init_equilibrium failed")
    return f


def step(p: Params, f: np.ndarray, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """Returns the pre-collision state after ``nsteps`` updates (input untouched)."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True).reshape((p.Q,) + p.shape)
    cp = p.c()
    rc = lib.oracle_step(ctypes.byref(cp), _dp(g), int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_step failed: {rc}")
    return g


def step_open(p: Params, f: np.ndarray, nsteps: int, u_in: float, rho_out: float,
              rho_w: float = 1.0, nthreads: int = 1) -> np.ndarray:
    """As step, with the open boundaries of Sec. 3.4 on D2Q9 (x non-periodic):
    moving-wall bounce-back inlet at the left (velocity u_in, wall density
    rho_w) and a Zou-He constant-density outlet (rho_out) at x = nx - 1."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True).reshape((p.Q,) + p.shape)
    cp = p.c()
    rc = lib.oracle_step_open(ctypes.byref(cp), float(u_in), float(rho_w), float(rho_out), _dp(g),
                              int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_step_open failed: {rc}")
    return g


def momentum_exchange(p: Params, f: np.ndarray) -> np.ndarray:
    """Force on the solid nodes by momentum exchange (Sec. 3.4) for the
    pre-collision state f: sum over fluid-to-solid links of 2 e_i f*_i."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(3)
    cp = p.c()
    if lib.oracle_momentum_exchange(ctypes.byref(cp), _dp(f), _dp(out)):
        raise RuntimeError("oracle_momentum_exchange failed")
    return out


def cubic_flux_gradient(p: Params, f: np.ndarray) -> np.ndarray:
    """d_a (rho u_a^3) of the pre-collision state f, shape (D, nz, ny, nx): the
    non-zero entries of d_g Phi_abg in G_i (Eq. Gi), by central differences,
    one-sided next to a solid node or a non-periodic edge."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((p.D,) + p.shape)
    cp = p.c()
    if lib.oracle_cubic_flux_gradient(ctypes.byref(cp), _dp(f), _dp(out)):
        raise RuntimeError("oracle_cubic_flux_gradient failed")
    return out


def collide_s2(p: Params, f: np.ndarray, dphi) -> np.ndarray:
    """Post-collision populations of one node with the Scheme II source
    (Eq. source_simple, Eq. Gi); dphi (3, 3) = d_g Phi_abg."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    d = np.ascontiguousarray(np.asarray(dphi, dtype=np.float64).reshape(3, 3))
    out = np.empty_like(f)
    cp = p.c()
    if lib.oracle_collide_s2(ctypes.byref(cp), _dp(f), _dp(d), _dp(out)):
        raise RuntimeError("oracle_collide_s2 failed")
    return out


def step_s2(p: Params, f: np.ndarray, nsteps: int, nthreads: int = 1) -> np.ndarray:
    """As step, with the Scheme II source (Eq. source_simple, Eq. Gi) instead of
    the Guo source; d_g Phi from the pre-collision state of each step."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True).reshape((p.Q,) + p.shape)
    cp = p.c()
    rc = lib.oracle_step_s2(ctypes.byref(cp), _dp(g), int(nsteps), int(nthreads))
    if rc:
        raise RuntimeError(f"oracle_step_s2 failed: {rc}")
    return g


def macros(p: Params, f: np.ndarray):
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(p.shape)
    u = np.zeros((p.D,) + p.shape)
    cp = p.c()
    if lib.oracle_macros(ctypes.byref(cp), _dp(f), _dp(rho), _dp(u)):
        raise RuntimeError("oracle_macros failed")
    return rho, u


def diagnostics(p: Params, f: np.ndarray) -> dict:
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(7)
    cp = p.c()
    if lib.oracle_diagnostics(ctypes.byref(cp), _dp(f), _dp(out)):
        raise RuntimeError("oracle_diagnostics failed")
    return {"mass": out[0], "momentum": out[1:4].copy(), "kinetic_energy": out[4],
            "enstrophy": out[5], "nan_flag": out[6]}


def l2(qn: np.ndarray, qa: np.ndarray) -> float:
    """Relative L2 error norm of Sec. 3."""
    lib = _load()
    qn = np.ascontiguousarray(qn, dtype=np.float64).ravel()
    qa = np.ascontiguousarray(qa, dtype=np.float64).ravel()
    return lib.oracle_l2(qn.size, _dp(qn), _dp(qa))


def pull_sample(p: Params, fstate, nodes) -> np.ndarray:
    """Pre-collision populations f(x, t+1) at a few sample nodes, from the
    pre-collision state f(., t) of a lattice too large to step whole.

    ``fstate(points)`` returns the (n, Q) pre-collision populations at integer
    node coordinates ``points`` ((n, 3) as x, y, z).  Each sample node needs the
    post-collision state of itself and of its Q - 1 upstream neighbours; the
    streaming rule is the one of ``oracle_step`` (periodic wrap, halfway
    bounce-back at solids and non-periodic edges)."""
    info = lattice_info(p.lattice)
    e, opp, Q = info["e"], info["opp"], info["Q"]
    ext = np.array([p.nx, p.ny, p.nz])
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1, 3)
    solid = None if p.solid is None else np.asarray(p.solid).reshape(p.shape)
    out = np.zeros((len(nodes), Q))
    for k, x in enumerate(nodes):
        src, bounce = [], []
        for i in range(Q):
            s = x - e[i]
            b = False
            for a in range(3):
                if s[a] < 0 or s[a] >= ext[a]:
                    if p.periodic[a]:
                        s[a] %= ext[a]
                    else:
                        b = True
            if not b and solid is not None and solid[s[2], s[1], s[0]]:
                b = True
            bounce.append(b)
            src.append(x if b else s)
        pts = np.array(src)
        fpre = np.asarray(fstate(pts), dtype=np.float64).reshape(Q, Q)
        fpost = collide(p, fpre)
        for i in range(Q):
            out[k, i] = fpost[i, opp[i]] if bounce[i] else fpost[i, i]
    return out
