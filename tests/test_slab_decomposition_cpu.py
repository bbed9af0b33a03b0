"""Design check of the single-lattice domain decomposition (a slab per rank
along the slowest axis, one halo exchange of whole rows per step), run on CPU
with two gloo ranks and the FP64 oracle as each rank's update: the gathered
result must equal the single-domain run bit for bit, with a solid block and
walls crossing the cuts.  Only the exchange pattern is exercised here; the GPU
path runs one replica per rank (no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case(lat):
    """Lattice, initial populations and mask of the single-domain run; the
    decomposed axis is y for D2Q9 and z for D3Q19 (the slowest one)."""
    import oracle as O
    import workloads as W
    shape = (1, 16, 21) if lat == O.D2Q9 else (12, 7, 9)
    solid = np.zeros(shape, dtype=np.uint8)
    if lat == O.D2Q9:
        solid[0, 6:10, 4:8] = 1      # straddles the cut at y = 8
    else:
        solid[5:8, 2:5, 3:6] = 1     # straddles the cut at z = 6
    periodic = (1, 0, 1) if lat == O.D2Q9 else (0, 1, 1)
    wp, wm = O.rates(nu=0.03, Lambda=3 / 16)
    p = O.Params(lat, shape[2], shape[1], shape[0], collision=O.P_TRT, omega_plus=wp,
                 omega_minus=wm, force=(1e-4, -5e-5, 2e-5 if lat == O.D3Q19 else 0.0),
                 periodic=periodic, solid=solid)
    rng = np.random.default_rng(61)
    rho, u = W.random_macros(shape, O.D_OF[lat], rng, umax=0.05)
    u = u * (solid == 0)
    return p, O.init_equilibrium(p, rho, u), solid


def _axis(lat):
    import oracle as O
    return 2 if lat == O.D2Q9 else 1  # index of y (D2Q9) / z (D3Q19) in (Q, nz, ny, nx)


def _worker(rank, world, port, lat, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle as O
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    p, f, solid = _case(lat)
    ax = _axis(lat)
    n = f.shape[ax]
    lo, hi = n * rank // world, n * (rank + 1) // world
    per = bool(p.periodic[1] if lat == O.D2Q9 else p.periodic[2])

    def take(a, idx, axis):
        return np.take(a, idx, axis=axis)

    own = take(f, np.arange(lo, hi), ax)
    # the extended slab: one halo row (plane) on each side; beyond a wall the
    # halo is a solid layer, so the oracle's own bounce-back applies there
    rows = [(lo - 1) % n if (per or lo > 0) else None, (hi) % n if (per or hi < n) else None]
    msk = take(solid, np.arange(lo, hi), ax - 1)
    halo_solid = [take(solid, [r], ax - 1) if r is not None else np.ones_like(take(solid, [0], ax - 1))
                  for r in rows]
    ext_solid = np.concatenate([halo_solid[0], msk, halo_solid[1]], axis=ax - 1)
    if lat == O.D2Q9:
        pe = O.Params(lat, p.nx, hi - lo + 2, 1, collision=p.collision, omega_plus=p.omega_plus,
                      omega_minus=p.omega_minus, force=p.force, periodic=(p.periodic[0], 0, 1),
                      solid=ext_solid)
    else:
        pe = O.Params(lat, p.nx, p.ny, hi - lo + 2, collision=p.collision,
                      omega_plus=p.omega_plus, omega_minus=p.omega_minus, force=p.force,
                      periodic=(p.periodic[0], p.periodic[1], 0), solid=ext_solid)
    for _ in range(STEPS):
        # halo exchange: every rank publishes its first and last owned row
        first = torch.from_numpy(np.ascontiguousarray(take(own, [0], ax)))
        last = torch.from_numpy(np.ascontiguousarray(take(own, [own.shape[ax] - 1], ax)))
        firsts = [torch.empty_like(first) for _ in range(world)]
        lasts = [torch.empty_like(last) for _ in range(world)]
        dist.all_gather(firsts, first)
        dist.all_gather(lasts, last)
        below = lasts[(rank - 1) % world].numpy()   # row lo - 1
        above = firsts[(rank + 1) % world].numpy()  # row hi
        if rows[0] is None:
            below = np.zeros_like(below)
        if rows[1] is None:
            above = np.zeros_like(above)
        ext = np.concatenate([below, own, above], axis=ax)
        ext = O.step(pe, np.ascontiguousarray(ext), 1)
        own = take(ext, np.arange(1, ext.shape[ax] - 1), ax)
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, own))
    if rank == 0:
        out["parts"] = parts
    dist.destroy_process_group()


@pytest.mark.parametrize("lat", [0, 1])
def test_slab_decomposition_is_bitwise_single_domain(lat):
    import sys
    sys.path.insert(0, ROOT)
    import oracle as O
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, lat, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    p, f, solid = _case(lat)
    ref = O.step(p, f, STEPS)
    ax = _axis(lat)
    got = np.concatenate([part[2] for part in sorted(out["parts"], key=lambda t: t[0])], axis=ax)
    fluid = np.broadcast_to(solid == 0, ref.shape)
    assert np.array_equal(got[fluid], ref[fluid])
