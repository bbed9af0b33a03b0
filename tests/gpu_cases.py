"""Shared helpers of the GPU tests: build a lattice through the C ABI binding
and the matching oracle run on the same seeded inputs."""
import numpy as np

import oracle as O

COLL_NAMES = {O.TRT: "TRT", O.TRT_RLB: "TRT_RLB", O.P_TRT: "P_TRT", O.BGK: "BGK", O.RLB: "RLB"}
LAT_NAMES = {O.D2Q9: "D2Q9", O.D3Q19: "D3Q19", O.D3Q27: "D3Q27"}


def gpu_lattice(lat, shape, coll, nu, Lam, storage="F64", force=(0.0, 0.0, 0.0),
                periodic=(1, 1, 1), solid=None, layout="AB"):
    from paper_2602_06686_gb300 import Lattice
    nz, ny, nx = shape
    return Lattice(lattice=LAT_NAMES[lat], nx=nx, ny=ny, nz=nz, nu=nu, Lambda=Lam,
                   collision=COLL_NAMES[coll], force=force, periodic=periodic, storage=storage,
                   layout=layout, solid=solid)


def oracle_params(lat, shape, coll, nu, Lam, force=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
                  solid=None):
    nz, ny, nx = shape
    wp, wm = O.rates(nu=nu, Lambda=Lam)
    return O.Params(lat, nx, ny, nz, collision=coll, omega_plus=wp, omega_minus=wm, force=force,
                    periodic=periodic, solid=solid)


def fluid(a, solid):
    """Values at fluid nodes (all nodes if there is no solid mask)."""
    a = np.asarray(a)
    if solid is None:
        return a
    return a[..., np.asarray(solid).reshape(a.shape[-3:]) == 0]


def elem_rel(a, b, solid=None):
    """max |a - b| / |b| element by element (populations are positive)."""
    a, b = fluid(a, solid), fluid(b, solid)
    return float(np.max(np.abs(a - b) / np.abs(b)))


def scaled_err(a, b, solid=None):
    """max |a - b| / max |b| (for fields that cross zero, e.g. velocity)."""
    a, b = fluid(a, solid), fluid(b, solid)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
