"""Benchmark of the P-TRT lattice Boltzmann hot path on GB300.

One benchmark "step" is one pass of the whole hot path over the workload:
``--inner`` fused stream-collide updates of the lattice followed by the FP64
diagnostics reduction (mass, momentum, kinetic energy, enstrophy, NaN flag).

Workload (default): D2Q9 P-TRT double shear layer, 4096 x 4096 periodic, FP32
shifted storage, U0 = 0.1, kappa = 80, delta = 0.05, Re = U0 N / nu = 1e5,
1/tau- = 1.6, A/B buffers (2 x 604 MB, far larger than the 129 MB L2, so no
flush is needed between iterations).  Metric: MLUPS (million lattice-node
updates per second, all nodes) and the fraction of the HBM roofline
(72 bytes per D2Q9 FP32 node update) of the fused kernel.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own replica (weak scaling); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "P-TRT MLUPS & % HBM roofline (D3Q19/D2Q9); FP16-store vs FP32 at set error"
BYTES_PER_NODE = {("D2Q9", "F64"): 144, ("D2Q9", "F32"): 72, ("D2Q9", "F16"): 36,
                  ("D2Q9", "BF16"): 36, ("D3Q19", "F64"): 304, ("D3Q19", "F32"): 152,
                  ("D3Q19", "F16"): 76, ("D3Q19", "BF16"): 76, ("D3Q27", "F64"): 432,
                  ("D3Q27", "F32"): 216, ("D3Q27", "F16"): 108, ("D3Q27", "BF16"): 108}
PROFILE = os.path.join(ROOT, "profiles", "stream_collide_d2q9_f32_4096.md")
# FP64 instructions (DADD + DMUL + DFMA) per node update of the FP64 update, by
# lattice and collision: ncu counts on D3Q19 128^3 and D2Q9 2048x1024
# (profiles/stream_collide_d3q19_f64_128.md).  With GB300's 2 FP64 lanes per
# SM they give the FP64-pipe roofline of the FP64 runs.
FP64_INSTR_PER_NODE = {("D3Q19", "P_TRT"): 242, ("D3Q19", "TRT_RLB"): 301, ("D3Q19", "TRT"): 192,
                       ("D2Q9", "P_TRT"): 103, ("D2Q9", "TRT_RLB"): 129, ("D2Q9", "TRT"): 93}
FP64_LANES_PER_SM = 2


def fp64_peak_instr_per_s() -> float:
    """FP64 instructions per second of the device: SMs x max SM clock x lanes."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = measured_peaks()["sm_max_mhz"]
    return sms * mhz * 1e6 * FP64_LANES_PER_SM


EXTRA_LEGEND = ("d2q9_*: double shear 4096^2 Re=1e5 1/tau-=1.6; d3q19_*/d3q27_*: Taylor-Green "
                "384^3 Re=1600 Lambda=1/4; collision P-TRT unless named; frac: algorithmic bytes "
                "/ measured HBM peak; copy: / copy ceiling at the buffer size; alu_frac (FP64): "
                "FP64 instructions / (SMs x clock x 2 lanes); v: kernel variant")


# Device code of the pipelined fused kernel: the committed ncu counters of the
# headline kernel are used only while these files are unchanged.
KERNEL_SOURCES = ("tma.cuh", "collide_v.cuh", "storage.cuh", "lattice.cuh", "kernels.cuh")


def csrc_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2602_06686_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured",
                "sm_max_mhz": float(d.get("sm_max_mhz") or 2070.0)}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


def profile_traffic(kernel_hash: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    with open(PROFILE) as fh:
        for line in fh:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("csrc_hash") != kernel_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self, wait_s: float = 5.0):
        """Start nvidia-smi and wait (up to wait_s) for its first sample, so that
        the timed region is covered from its beginning."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < wait_s:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0: float | None = None, t1: float | None = None) -> dict | None:
        """Median SM clock and the throttle reasons seen in [t0, t1] (wall clock,
        time.perf_counter), widened by one sampling period on each side."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if t0 is not None and (ts < t0 - 0.1 or ts > t1 + 0.1):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(units: float, seconds: float, group=None):
    """Whole-job totals across ranks: units summed, time = max over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()), float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(seconds_target: float = 12.0, n: int = 512, threads: int | None = None):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload:
    the same double shear layer on an n x n lattice, D2Q9 P-TRT."""
    import oracle as O
    import workloads as W
    threads = threads or len(os.sched_getaffinity(0))
    nu = 0.1 * n / 1e5
    wp, wm = O.rates(nu=nu, tau_minus=1 / 1.6)
    p = O.Params(O.D2Q9, n, n, 1, collision=O.P_TRT, omega_plus=wp, omega_minus=wm)
    rho, u = W.double_shear(n)
    f = O.init_equilibrium(p, rho, u)
    t0 = time.perf_counter()
    O.step(p, f, 1, nthreads=threads)
    one = time.perf_counter() - t0
    steps = max(1, int(seconds_target / max(one, 1e-6)))
    t0 = time.perf_counter()
    O.step(p, f, steps, nthreads=threads)
    dt = time.perf_counter() - t0
    # the same oracle on one core (a shorter sample)
    g1 = O.init_equilibrium(p, rho, u)
    t1 = time.perf_counter()
    O.step(p, g1, 1, nthreads=1)
    one1 = time.perf_counter() - t1
    steps1 = max(1, int(seconds_target / 3 / max(one1, 1e-6)))
    t1 = time.perf_counter()
    O.step(p, g1, steps1, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": f"D2Q9 P-TRT FP64 double shear {n}x{n}, {steps} steps ({dt:.1f} s)",
            "single_core_value": n * n * steps1 / dt1 / 1e6,
            "single_core_sample": f"{steps1} steps ({dt1:.1f} s) on 1 core"}


def headline_workload(n: int) -> str:
    """The headline workload's name, shared by both arms of the benchmark."""
    return (f"D2Q9 P-TRT double shear layer {n}x{n}, FP32 shifted storage, "
            f"Re=1e5, 1/tau-=1.6, A/B buffers")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W
    threads = len(os.sched_getaffinity(0))
    n = 512
    nu = 0.1 * n / 1e5
    wp, wm = O.rates(nu=nu, tau_minus=1 / 1.6)
    p = O.Params(O.D2Q9, n, n, 1, collision=O.P_TRT, omega_plus=wp, omega_minus=wm)
    rho, u = W.double_shear(n)
    f = O.init_equilibrium(p, rho, u)
    inner = 2
    for _ in range(args.warmup):
        f = O.step(p, f, inner, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(p, f, inner, nthreads=threads)
    dt = time.perf_counter() - t0
    value = n * n * inner * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": headline_workload(4096),
                   "sample": f"the same flow on {n}x{n} (same Re and rates), FP64 oracle",
                   "updates_per_step": inner},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"D2Q9 P-TRT FP64 double shear {n}x{n}, {inner} updates "
                                   f"per step, {args.steps} steps"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def workload_fields(kind: str, n: int):
    import workloads as W
    if kind == "double_shear":
        return W.double_shear(n, U0=0.1)
    return W.taylor_green_3d(n, u0=0.05)


def make_lattice(lat: str, n: int, storage: str, collision: str = "P_TRT", layout: str = "AB",
                 tau_minus: float | None = None):
    """D2Q9: double shear layer, Re = U0 N / nu = 1e5, 1/tau- = 1.6 (the stability
    optimum of Sec. 3.1).  D3Q19 / D3Q27: Taylor-Green vortex at Re = 1600
    (L = N / 2 pi), Lambda = 1/4 unless tau_minus is given."""
    from paper_2602_06686_gb300 import Lattice
    if lat == "D2Q9":
        return Lattice(lattice="D2Q9", nx=n, ny=n, nz=1, nu=0.1 * n / 1e5, tau_minus=1 / 1.6,
                       collision=collision, storage=storage, layout=layout)
    rates = dict(tau_minus=tau_minus) if tau_minus else dict(Lambda=0.25)
    return Lattice(lattice=lat, nx=n, ny=n, nz=n, nu=0.05 * n / (2 * math.pi * 1600),
                   collision=collision, storage=storage, layout=layout, **rates)


def time_kernel(lat_obj, inner: int, reps: int):
    """Average duration of one fused update (CUDA events on the lattice's stream)."""
    import torch
    st = lat_obj.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat_obj.step(inner)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        lat_obj.step(inner)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / (reps * inner) * 1e-3


def copy_ceiling_at(nbytes: int, reps: int = 20) -> dict:
    """Copy bandwidth (read + write bytes / time) at one population buffer's size:
    the library's 128-bit copy kernel and torch's copy_, CUDA events, best of
    `reps` after warm-up."""
    import torch
    from paper_2602_06686_gb300 import copy_ceiling
    n = (nbytes // 16) * 16
    a = torch.empty(n, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1)
    st = torch.cuda.current_stream()
    out = {"bytes": n}
    for name, fn in (("lbm_copy", lambda: copy_ceiling(a, b, n, st)),
                     ("torch_copy", lambda: b.copy_(a))):
        for _ in range(3):
            fn()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        out[name + "_gbs"] = 2 * n / best / 1e9
    del a, b
    torch.cuda.empty_cache()
    return out


def scheme2_bytes_per_node(lat: str, storage: str) -> int:
    """Algorithmic bytes of one Scheme II update per node: the rho u_a^3 pass
    reads Q populations and writes D values, the update reads Q populations and
    the D values (each once from memory; the neighbours' through L2) and writes
    Q populations."""
    D = 2 if lat == "D2Q9" else 3
    r = 8 if storage == "F64" else 4
    return 3 * BYTES_PER_NODE[(lat, storage)] // 2 + 2 * D * r


def secondary(lat: str, n: int, storage: str, kind: str, peak: float, collision="P_TRT",
              layout: str = "AB", scheme: int = 1):
    """MLUPS and roofline fraction of another workload (kernel-only, few steps):
    mlups, frac (of the measured HBM peak, algorithmic bytes), copy (of the
    larger copy ceiling measured at the buffer's size), v (kernel variant)."""
    import torch
    g = make_lattice(lat, n, storage, collision, layout)
    rho, u = workload_fields(kind, n)
    g.init_equilibrium(rho, u)
    if scheme == 2:
        g.set_forcing_scheme(2)
    g.autotune(reps=3, report=False)
    reps = 1 if storage == "F64" and lat != "D2Q9" else 3
    dt = time_kernel(g, 10, reps)
    N = g.N
    bpn = BYTES_PER_NODE[(lat, storage)] if scheme == 1 else scheme2_bytes_per_node(lat, storage)
    gbs = bpn * N / dt / 1e9
    out = {"mlups": N / dt / 1e6, "frac": gbs / peak, "v": g.variants()[g.variant]}
    if storage == "F64" and (lat, collision) in FP64_INSTR_PER_NODE:
        out["bound"] = "alu"
        out["alu_frac"] = N / dt * FP64_INSTR_PER_NODE[(lat, collision)] / fp64_peak_instr_per_s()
    if scheme == 2:
        out["bytes_per_node"] = bpn
    rc, _ = g.status()
    if rc != 0:
        out["diverged"] = True
    del g
    torch.cuda.empty_cache()
    cc = copy_ceiling_at(BYTES_PER_NODE[(lat, storage)] * N // 2)
    out["copy"] = gbs / max(cc["lbm_copy_gbs"], cc["torch_copy_gbs"])
    return out


def compact(v, digits: int = 4):
    """Floats rounded to `digits` significant digits (recursively), so that the
    bench line stays short."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}") if math.isfinite(v) else v
    if isinstance(v, dict):
        return {k: compact(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [compact(x, digits) for x in v]
    return v


def batched(peak: float, count: int = 256, steps: int = 500):
    """256 uneven D2Q9 P-TRT double shear lattices (side lengths U{64..1024}, Re
    log-uniform in [1e3, 1e7], Lambda in {1/12, 3/16, 1/4}, seeded), FP32, advanced
    `steps` steps by the persistent kernel in a CUDA graph versus one launch per
    lattice per step.  Many of these lattices diverge (small Lambda at high Re),
    so the aggregate over the lattices that stayed finite is reported as well,
    and the same seeded shapes and Reynolds numbers are run once more at
    1/tau- = 1.6 (the stability optimum of Sec. 3.1), where they survive."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Batch
    lats = W.batch_lattices(count)
    out = {"lattices": count, "steps": steps}
    for label, rate in (("lambda_draw", None), ("inv_tau_minus_1.6", 1 / 1.6)):
        specs = []
        for d in lats:
            r = dict(Lambda=d["Lambda"]) if rate is None else dict(tau_minus=rate)
            specs.append(dict(lattice="D2Q9", nx=d["nx"], ny=d["ny"], nu=0.1 * d["nx"] / d["Re"],
                              collision="P_TRT", storage="F32", **r))
        b = Batch(specs)

        def init():
            for i, s in enumerate(specs):
                b.lattice(i).init_equilibrium(*W.double_shear_rect(s["nx"], s["ny"]))

        init()
        chosen, _ = b.autotune(steps=4)
        modes = ((0, "persistent"), (1, "sequential")) if rate is None else ((0, "persistent"),)
        res = {"tile": b.variants()[chosen]}
        for mode, name in modes:
            init()
            b.step(2, mode)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step(steps, mode)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[name + "_mlups"] = b.nodes * steps / dt / 1e6
            if mode == 0:
                res["seconds"] = dt
        bad = [i for i in range(count) if b.lattice(i).status()[0] != 0]
        live = sum(specs[i]["nx"] * specs[i]["ny"] for i in range(count) if i not in set(bad))
        res["frac"] = res["persistent_mlups"] * 1e6 * 72 / 1e9 / peak
        res["diverged"] = len(bad)
        res["finite_lattice_mlups"] = live * steps / res["seconds"] / 1e6
        if rate is None:
            res["speedup_vs_sequential"] = res["persistent_mlups"] / res["sequential_mlups"]
            out["nodes"] = b.nodes
        out[label] = res
        b.close()
        del b
        torch.cuda.empty_cache()
    return out


PRECISION_STORAGES = ("F64", "F32", "F16", "BF16")


def channel_relax_steps(h: int, nu: float, efolds: float = 30.0) -> int:
    """Steps for the slowest diffusive mode of a channel of height h to decay by
    exp(-efolds) (time constant h^2 / (pi^2 nu))."""
    return int(math.ceil(efolds * h * h / (math.pi ** 2 * nu)))


def precision_channel(nus=(0.1,), h: int = 64, u_c: float = 0.05, with_oracle: bool = False):
    """Accuracy of the shifted storage formats on the force-driven D3Q19 channel
    (halfway bounce-back walls normal to y, periodic in x and z, Lambda = 3/16,
    body force F = 8 nu u_c / h^2), run from rest to steady state.

    The flow is invariant in x and z and the update is per node, so a narrow
    32 x h x 4 slab computes, column for column, exactly what the full
    512 x h x 512 channel does; only throughput depends on the extent.  Each
    storage format reports the relative L2 error of u_x against the discrete
    analytic profile (which the FP64 update reaches to rounding at Lambda = 3/16)
    and against the FP64 run of the same length; with ``with_oracle`` the FP64
    CPU oracle is run on one column as well."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Lattice
    out = []
    exact = W.poiseuille_profile(h, u_c)
    for nu in nus:
        F = 8.0 * nu * u_c / (h * h)
        T = channel_relax_steps(h, nu)
        shape = (4, h, 32)
        rho, u = W.channel_at_rest(shape, 3)
        ux = {}
        for st in PRECISION_STORAGES:
            g = Lattice(lattice="D3Q19", nx=32, ny=h, nz=4, nu=nu, Lambda=3 / 16,
                        collision="P_TRT", storage=st, force=(F, 0.0, 0.0), periodic=(1, 0, 1))
            g.init_equilibrium(rho, u)
            g.step(T)
            _, uu = g.macros()
            ux[st] = uu[0].double().cpu().numpy()
            rc, _ = g.status()
            del g
            if rc != 0:
                ux[st] = None
        torch.cuda.synchronize()
        row = {"nu": nu, "force": F, "steps": T}
        ref = np.broadcast_to(exact[None, :, None], shape)
        for st in PRECISION_STORAGES:
            if ux[st] is None:
                row[st] = {"diverged": True}
                continue
            row[st] = {"l2_vs_analytic": rel_l2(ux[st], ref),
                       "l2_vs_fp64": rel_l2(ux[st], ux["F64"])}
        if with_oracle:
            import oracle as O
            wp, wm = O.rates(nu=nu, Lambda=3 / 16)
            p = O.Params(O.D3Q19, 1, h, 1, collision=O.P_TRT, omega_plus=wp, omega_minus=wm,
                         force=(F, 0.0, 0.0), periodic=(1, 0, 1))
            r0, u0 = W.channel_at_rest(p.shape, 3)
            _, uo = O.macros(p, O.step(p, O.init_equilibrium(p, r0, u0), T, nthreads=1))
            col = uo[0][:, :, 0:1]
            row["oracle"] = {"l2_vs_analytic": rel_l2(col, exact[None, :, None]),
                             "gpu_fp64_vs_oracle": rel_l2(ux["F64"][:, :, 0:1][0:1], col)}
            for st in ("F32", "F16", "BF16"):
                if ux[st] is not None:
                    row[st]["l2_vs_oracle"] = rel_l2(ux[st][0:1, :, 0:1], col)
        out.append(row)
    return out


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = float(np.sqrt(np.sum(b * b)))
    return float(np.sqrt(np.sum((a - b) ** 2)) / den) if den > 0 else float("nan")


def precision_throughput(peak: float, nx: int = 512, h: int = 64, nz: int = 512):
    """MLUPS of the full force-driven D3Q19 channel (nx x h x nz, walls normal to
    y) per storage format, FP32 arithmetic, kernel-only."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Lattice
    out = {}
    nu, u_c = 0.1, 0.05
    F = 8.0 * nu * u_c / (h * h)
    for st in ("F32", "F16", "BF16"):
        g = Lattice(lattice="D3Q19", nx=nx, ny=h, nz=nz, nu=nu, Lambda=3 / 16,
                    collision="P_TRT", storage=st, force=(F, 0.0, 0.0), periodic=(1, 0, 1))
        rho, u = W.channel_at_rest((nz, h, nx), 3)
        g.init_equilibrium(rho, u)
        g.autotune(reps=3, report=False)
        dt = time_kernel(g, 10, 3)
        bpn = BYTES_PER_NODE[("D3Q19", st)]
        out[st] = {"mlups": g.N / dt / 1e6, "kernel_ms": dt * 1e3,
                   "frac": bpn * g.N / dt / 1e9 / peak, "variant": g.variants()[g.variant]}
        del g
        torch.cuda.empty_cache()
    out["f16_over_f32"] = out["F16"]["mlups"] / out["F32"]["mlups"]
    out["workload"] = f"D3Q19 P-TRT force-driven channel {nx}x{h}x{nz}, Lambda=3/16"
    return out


def precision_cylinder(steps: int = 0, nx: int = 2048, ny: int = 1024, side: int = 64,
                       re: float = 0.1, ma: float = 0.1, cdmu: float = 8.252):
    """D2Q9 creeping flow through a periodic array of square cylinders: a centred
    side x side halfway bounce-back square in a fully periodic nx x ny lattice,
    Ma = u0 / cs = 0.1 and Re = u0 side / nu = 0.1 (so nu = u0 side / Re and
    tau+ = 1/2 + 3 nu, about 111), Lambda = 3/16, driven by a uniform body force
    sized from the Stokes drag F_x = Cd,mu rho u0 nu / 2 with the paper's
    Cd,mu = 8.252, spread over the fluid nodes.  Every storage format runs
    `steps` steps from rest (default: 30 e-folds of the slowest diffusive mode,
    ny^2 / (pi^2 nu) steps each); reported are the relative L2 error of the fluid
    velocity against the FP64 run of the same length, the Reynolds number that
    run reaches (mean fluid u_x), and the MLUPS of each format."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Lattice
    u0 = ma / math.sqrt(3.0)
    nu = u0 * side / re
    solid = W.square_cylinder_mask(nx, ny, side)
    fluid = solid[0] == 0
    F = cdmu * u0 * nu / 2.0 / float(fluid.sum())
    if steps <= 0:
        steps = int(math.ceil(30.0 * ny * ny / (math.pi ** 2 * nu)))
    shape = (1, ny, nx)
    rho, u = W.channel_at_rest(shape, 2)
    vel, rates = {}, {}
    for st in PRECISION_STORAGES:
        g = Lattice(lattice="D2Q9", nx=nx, ny=ny, nu=nu, Lambda=3 / 16, collision="P_TRT",
                    storage=st, force=(F, 0.0, 0.0), periodic=(1, 1, 1), solid=solid)
        g.init_equilibrium(rho, u)
        g.step(steps)
        _, uu = g.macros()
        vel[st] = uu.double().cpu().numpy()
        rc, _ = g.status()
        dt = time_kernel(g, 10, 3)
        rates[st] = {"mlups": g.N / dt / 1e6, "diverged": rc != 0}
        del g
        torch.cuda.empty_cache()
    ux64 = vel["F64"][0, 0][fluid]
    out = {"workload": f"D2Q9 P-TRT periodic square-cylinder array {nx}x{ny}, side {side}, "
                       f"Ma={ma}, Re={re} (nu={nu:.4g}, tau+={0.5 + 3 * nu:.4g}), "
                       f"Lambda=3/16, {steps} steps from rest",
           "force": F, "re_reached_fp64": float(ux64.mean()) * side / nu}
    for st in PRECISION_STORAGES:
        out[st] = dict(rates[st])
        out[st]["l2_vs_fp64"] = rel_l2(vel[st][:, 0][:, fluid], vel["F64"][:, 0][:, fluid])
    return out


def precision_flow(kind: str, n: int, steps: int):
    """Relative L2 error of the velocity of each storage format against the FP64
    run of the same workload and length: the 3-D Taylor-Green vortex (D3Q19,
    Re = 1600, n^3, 1/tau- = 1.6: with Lambda = 1/4 the minus rate is tiny at
    this Reynolds number and the run diverges, see taylor_green_run) or the
    double shear layer (D2Q9, Re = 1e5, 1/tau- = 1.6, n^2)."""
    import torch
    lat = "D3Q19" if kind == "taylor_green_3d" else "D2Q9"
    rho, u = workload_fields(kind, n)
    vel = {}
    for st in PRECISION_STORAGES:
        g = make_lattice(lat, n, st, tau_minus=1 / 1.6 if lat == "D3Q19" else None)
        g.init_equilibrium(rho, u)
        g.step(steps)
        _, uu = g.macros()
        vel[st] = uu.double().cpu().numpy()
        rc, _ = g.status()
        if rc != 0:
            vel[st] = None
        del g
        torch.cuda.empty_cache()
    out = {"workload": f"{lat} P-TRT {kind} {n}^{3 if lat == 'D3Q19' else 2}, {steps} steps"}
    for st in ("F32", "F16", "BF16"):
        out[st] = ({"l2_vs_fp64": rel_l2(vel[st], vel["F64"])} if vel[st] is not None
                   and vel["F64"] is not None else {"diverged": True})
    return out


STABILITY_COLLISIONS = ("P_TRT", "TRT_RLB", "TRT", "RLB", "BGK")


def critical_mach(collision: str, cases, n: int = 128, dma: float = 0.01, ma_hi: float = 1.0,
                  storage: str = "F32"):
    """Largest stable Mach number Ma_c (Sec. 3.1) of the double shear layer on an
    n x n periodic lattice for each (Re, 1/tau-) case, by bisection to dma: a run
    at Ma (u_c = Ma cs, nu = u_c n / Re) is stable if it reaches t = 2 t_c =
    2 n / u_c steps without divergence (NaN/Inf, rho <= 0 or |u| > 1, the
    per-lattice flag).  Every bisection round advances all cases together as one
    batch in one persistent launch.  1/tau- is ignored by BGK and RLB (their
    minus rate is tied to the plus rate or to 1).  Returns Ma_c per case (0.0:
    unstable at every tested Ma; ma_hi: stable at ma_hi) and the round count."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Batch
    cs = 1.0 / math.sqrt(3.0)
    lo = [0.0] * len(cases)
    hi = [ma_hi] * len(cases)
    probe = [ma_hi] * len(cases)  # the first round tries ma_hi itself
    rounds = 0
    while True:
        specs, steps = [], []
        for (re, itm), ma in zip(cases, probe):
            uc = ma * cs
            specs.append(dict(lattice="D2Q9", nx=n, ny=n, nu=uc * n / re, tau_minus=1.0 / itm,
                              collision=collision, storage=storage))
            steps.append(int(math.ceil(2.0 * n / uc)))
        b = Batch(specs)
        for i in range(len(specs)):
            b.lattice(i).init_equilibrium(*W.double_shear_rect(n, n, U0=probe[i] * cs))
        b.step(max(steps), mode=0)
        torch.cuda.synchronize()
        for i in range(len(cases)):
            rc, first = b.lattice(i).status()
            if rc == 0 or first >= steps[i]:
                lo[i] = probe[i]
            else:
                hi[i] = probe[i]
        b.close()
        del b
        torch.cuda.empty_cache()
        rounds += 1
        if all(h - l <= dma + 1e-12 or l >= ma_hi for l, h in zip(lo, hi)):
            break
        probe = [(l + h) / 2 if h - l > dma + 1e-12 and l < ma_hi else l for l, h in zip(lo, hi)]
    return lo, rounds


def stability_sweep(res=(1e4, 5e4, 1e5, 1e6, 1e7), itms=None, n: int = 128):
    """Ma_c against 1/tau- for P-TRT, TRT-RLB and TRT (and the single-rate BGK
    and RLB, whose Ma_c does not depend on tau-) at each Reynolds number."""
    if itms is None:  # 0.1 .. 1.9 and 1.99 (1/tau- = 2 is tau- = 1/2, not a valid rate)
        itms = [round(0.1 * k, 1) for k in range(1, 20)] + [1.99]
    out = {"n": n, "re": list(res), "inv_tau_minus": itms, "ma_c": {}, "seconds": {},
           "rounds": {}}
    for coll in STABILITY_COLLISIONS:
        grid = [(re, itm) for re in res
                for itm in (itms if coll in ("P_TRT", "TRT_RLB", "TRT") else [1.0])]
        t0 = time.perf_counter()
        mac, rounds = critical_mach(coll, grid, n=n)
        table = {}
        for (re, itm), m in zip(grid, mac):
            table.setdefault(f"{re:g}", {})[f"{itm:g}"] = m
        out["ma_c"][coll] = table
        out["seconds"][coll] = time.perf_counter() - t0
        out["rounds"][coll] = rounds
    return out


def run_stability_study(args):
    """Critical Mach number sweep of the double shear layer (Sec. 3.1)."""
    from paper_2602_06686_gb300 import build
    build.build()
    print(json.dumps({"study": "stability", **stability_sweep()}), flush=True)
    return 0


def taylor_green_run(n: int = 384, steps: int = 2000, every: int = 100):
    """The 3-D Taylor-Green vortex at Re = 1600 on n^3 (u0 = 0.05), 2000 steps,
    kinetic energy and enstrophy reduced in FP64 every `every` steps: FP32
    storage with Lambda = 1/4 and with 1/tau- = 1.6, and FP64 storage with
    1/tau- = 1.6.  Reports the histories and the first diverged step."""
    import torch
    rho, u = workload_fields("taylor_green_3d", n)
    out = {"workload": f"D3Q19 P-TRT Taylor-Green {n}^3, Re = 1600, u0 = 0.05, {steps} steps"}
    for name, st, tm in (("F32_Lambda_1/4", "F32", None), ("F32_inv_tau_minus_1.6", "F32", 1 / 1.6),
                         ("F64_inv_tau_minus_1.6", "F64", 1 / 1.6)):
        g = make_lattice("D3Q19", n, st, tau_minus=tm)
        g.init_equilibrium(rho, u)
        ke, ens = [], []
        for _ in range(steps // every):
            g.step(every)
            d = g.diagnostics()
            ke.append(d["kinetic_energy"])
            ens.append(d["enstrophy"])
        rc, first = g.status()
        out[name] = {"kinetic_energy": ke, "enstrophy": ens, "first_diverged_step": first}
        del g
        torch.cuda.empty_cache()
    return out


def double_shear_run(n: int, re: float, collision: str, rate: dict, tc: float = 10.0,
                     every_tc: float = 0.25, storage: str = "F32"):
    """One run of the double shear layer of Sec. 3.1 on an n x n periodic
    lattice (U0 = 0.1, kappa = 80, delta = 0.05, nu = U0 n / Re) to `tc`
    convective times (t_c = n / U0 steps) or until the update flags divergence
    (reading 12).  Kinetic energy and enstrophy (FP64) every `every_tc`
    convective times, normalised by their initial values."""
    import torch
    from paper_2602_06686_gb300 import Lattice
    g = Lattice(lattice="D2Q9", nx=n, ny=n, nz=1, nu=0.1 * n / re, collision=collision,
                storage=storage, **rate)
    g.init_equilibrium(*workload_fields("double_shear", n))
    d0 = g.diagnostics()
    steps = int(round(tc * n / 0.1))
    every = max(1, int(round(every_tc * n / 0.1)))
    ke, ens, t = [], [], 0
    first = -1
    while t < steps:
        k = min(every, steps - t)
        g.step(k)
        t += k
        d = g.diagnostics()
        rc, first = g.status()
        if rc != 0:
            break
        ke.append(d["kinetic_energy"] / d0["kinetic_energy"])
        ens.append(d["enstrophy"] / d0["enstrophy"])
    out = {"n": n, "re": re, "collision": collision, "rate": list(rate.items())[0],
           "steps": steps, "first_diverged_step": first if first >= 0 else None,
           "ke": ke[-1] if ke else None, "enstrophy": ens[-1] if ens else None,
           "ke_history": ke, "enstrophy_history": ens}
    del g
    torch.cuda.empty_cache()
    return out


def run_reynolds_study(args):
    """The double shear layer sweep of Sec. 3.1 (the second workload): 1024^2 and
    4096^2, Re = 1e4 .. 1e7, P-TRT vs TRT vs TRT-RLB, FP32, 1/tau- = 1.6 and
    Lambda = 1/4, to 10 convective times or divergence."""
    from paper_2602_06686_gb300 import build
    build.build()
    sizes = [int(v) for v in args.sizes.split(",")]
    rows = []
    for n in sizes:
        for re in (1e4, 1e5, 1e6, 1e7):
            for coll in ("P_TRT", "TRT_RLB", "TRT"):
                for rate in ({"tau_minus": 1 / 1.6}, {"Lambda": 0.25}):
                    t0 = time.perf_counter()
                    r = double_shear_run(n, re, coll, rate)
                    r["seconds"] = time.perf_counter() - t0
                    brief = {k: v for k, v in r.items() if not k.endswith("history")}
                    print(json.dumps(compact(brief, 6)), flush=True)
                    rows.append(r)
    print(json.dumps({"study": "reynolds", "rows": compact(rows, 6)}), flush=True)
    return 0


def cylinder_lattice(re: float, d: int = 21, lfac: int = 50, storage: str = "F32",
                     collision: str = "P_TRT"):
    """The square-cylinder lattice of Sec. 3.4 started from the uniform stream:
    side d centred in an (lfac d)^2 domain, moving-wall inlet at u_c on the
    left, Zou-He outlet (rho = 1) on the right, y periodic, Lambda = 3/16,
    Ma = min(0.1, sqrt(0.1 Re)) (T = Ma^2/Re = 0.1 in the low-Re regime of
    Tab. 3), nu = u_c d / Re.  Returns (lattice, u_c, Ma, nu); the drag
    coefficient is C_d = 2 F_x / (rho0 u_c^2 d) with F_x from
    lattice.momentum_exchange()."""
    import workloads as W
    from paper_2602_06686_gb300 import Lattice
    n = lfac * d
    ma = min(0.1, math.sqrt(0.1 * re))
    uc = ma / math.sqrt(3.0)
    nu = uc * d / re
    solid = W.square_cylinder_mask(n, n, d)
    g = Lattice(lattice="D2Q9", nx=n, ny=n, nu=nu, Lambda=3 / 16, collision=collision,
                storage=storage, periodic=(0, 1, 1), solid=solid)
    g.set_open_boundaries(uc, 1.0)
    rho = np.ones((1, n, n))
    u = np.zeros((2, 1, n, n))
    u[0] = uc * (solid == 0)
    g.init_equilibrium(rho, u)
    return g, uc, ma, nu


def cylinder_drag(re: float, d: int = 21, lfac: int = 50, storage: str = "F32",
                  check: int = 5000, tol: float = 1e-6, max_steps: int = 400000,
                  collision: str = "P_TRT", criterion: str = "cd"):
    """Drag of the square cylinder of Sec. 3.4: side d centred in an (lfac d)^2
    domain, moving-wall inlet at u_c on the left, Zou-He outlet (rho = 1) on the
    right, y periodic, Lambda = 3/16, Ma = min(0.1, sqrt(0.1 Re)) (T = Ma^2/Re =
    0.1 in the low-Re regime of Tab. 3), nu = u_c d / Re.  Starts from the
    uniform stream and steps `check` steps at a time until converged:
    criterion "cd": C_d = 2 F_x / (rho0 u_c^2 d) changes by less than tol
    (relative) over `check` steps; criterion "l2": the relative L2 norm of
    Sec. 3 between the velocity fields `check` steps apart is below tol (the
    paper's L2 < 1e-9 for this flow, with check = 10000).  Returns C_d,
    C_d,mu = C_d Re, the steps taken, the last L2 and, for 2 <= Re <= 40, Sen's
    C_d = 0.7496 + 10.5767 Re^-0.66."""
    import torch
    g, uc, ma, nu = cylinder_lattice(re, d, lfac, storage, collision)
    cd_prev, steps, cd, l2 = None, 0, float("nan"), float("nan")
    u_prev = g.macros()[1] if criterion == "l2" else None
    converged = False
    t0 = time.perf_counter()
    while steps < max_steps:
        g.step(check)
        steps += check
        cd = 2.0 * g.momentum_exchange()[0] / (uc * uc * d)
        if criterion == "l2":
            l2 = g.velocity_l2(u_prev)
            u_prev = g.macros()[1]
            if l2 < tol:
                converged = True
                break
        else:
            if cd_prev is not None and abs(cd - cd_prev) <= tol * abs(cd):
                converged = True
                break
            cd_prev = cd
        if g.status()[0] != 0:
            break
    torch.cuda.synchronize()
    out = {"re": re, "ma": ma, "tau_plus": 0.5 + 3 * nu, "collision": collision,
           "storage": storage, "cd": cd, "cd_mu": cd * re, "steps": steps,
           "converged": converged, "seconds": time.perf_counter() - t0,
           "diverged": g.status()[0] != 0}
    if criterion == "l2":
        out["l2_last"] = l2
    if 2 <= re <= 40:
        out["cd_sen"] = 0.7496 + 10.5767 * re ** -0.66
    del g
    torch.cuda.empty_cache()
    return out


TAB3_RE = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)
TAB3_PRINTED = {1e-1: 8.449, 1e-2: 8.260, 1e-3: 8.253, 1e-4: 8.253, 1e-5: 8.252, 1e-6: 8.252}


def tab3_row(re: float, collision: str, max_steps: int = 1_600_000):
    """One row of Tab. 3 (Sec. 3.4): FP64 storage (the steady state is
    converged to the paper's L2 < 1e-9 between fields 10000 steps apart, below
    what FP32 storage resolves at u_c = 1.8e-4) and the printed C_d,mu."""
    r = cylinder_drag(re, storage="F64", check=10000, tol=1e-9, max_steps=max_steps,
                      collision=collision, criterion="l2")
    r["cd_mu_printed"] = TAB3_PRINTED.get(re)
    return r


def run_cylinder_study(args):
    """Square-cylinder drag (Sec. 3.4), D = 21, L = 50 D: every row of Tab. 3
    (Re = 1e-1 .. 1e-6, tau+ up to 11503) for P-TRT and TRT-RLB in FP64 to
    the paper's L2 < 1e-9, the Re = 0.1 row in FP32 as well, and C_d at
    Re = 2..20 against Sen's law."""
    from paper_2602_06686_gb300 import build
    build.build()
    rows = []
    for re in TAB3_RE:
        pair = {c: tab3_row(re, c) for c in ("P_TRT", "TRT_RLB")}
        pair["P_TRT"]["cd_rel_diff_trt_rlb"] = (abs(pair["P_TRT"]["cd"] - pair["TRT_RLB"]["cd"])
                                               / abs(pair["TRT_RLB"]["cd"]))
        rows += [pair["P_TRT"], pair["TRT_RLB"]]
        print(json.dumps(compact(pair, 6)), flush=True)
    res = {"study": "cylinder", "tab3": rows,
           "low_re_f32": cylinder_drag(0.1, storage="F32"),
           "sen": [cylinder_drag(re) for re in (2.0, 5.0, 10.0, 20.0)]}
    print(json.dumps(compact(res, 6)), flush=True)
    return 0


def run_precision_study(args):
    """Full precision study (minutes): channel at nu = 0.1, 0.01, 0.001 (the FP64
    oracle on one column at nu = 0.1), the full-channel throughput per format,
    and the square cylinder."""
    import torch
    from paper_2602_06686_gb300 import build
    build.build()
    peak = measured_peaks()["hbm_gbs"]
    res = {"study": "precision",
           "channel": precision_channel((0.1, 0.01, 0.001), with_oracle=False),
           "channel_oracle": precision_channel((0.1,), with_oracle=True),
           "throughput": precision_throughput(peak),
           "taylor_green_3d": precision_flow("taylor_green_3d", 128, 2000),
           "taylor_green_384": taylor_green_run(),
           "double_shear": precision_flow("double_shear", 1024, 10240),
           "cylinder": precision_cylinder(args.cyl_steps)}
    torch.cuda.synchronize()
    print(json.dumps(res), flush=True)
    return 0


def run_case(args):
    """One lattice configuration for a profiler: LATTICE:STORAGE:NX,NY,NZ[:COLLISION[:LAYOUT]],
    LAYOUT AB, AA or S2 (A/B with forcing scheme II),
    fixed kernel variant (by name; the default variant otherwise), ``--warmup``
    updates then ``--inner`` updates."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import build, Lattice
    build.build()
    parts = args.case.split(":")
    lat, st = parts[0], parts[1]
    dims = [int(v) for v in parts[2].split(",")]
    coll = parts[3] if len(parts) > 3 else "P_TRT"
    layout = parts[4] if len(parts) > 4 else "AB"
    scheme = 2 if layout == "S2" else 1
    layout = "AB" if layout == "S2" else layout
    nx, ny = dims[0], dims[1]
    nz = dims[2] if len(dims) > 2 else 1
    if lat == "D2Q9":
        g = Lattice(lattice="D2Q9", nx=nx, ny=ny, nu=0.1 * nx / 1e5, tau_minus=1 / 1.6,
                    collision=coll, storage=st, layout=layout)
        rho, u = W.double_shear_rect(nx, ny)
    else:
        g = Lattice(lattice=lat, nx=nx, ny=ny, nz=nz, nu=0.05 * nx / (2 * math.pi * 1600),
                    Lambda=0.25, collision=coll, storage=st, layout=layout)
        rho, u = W.channel_at_rest((nz, ny, nx), 3)
        u[0] = 0.02
    g.init_equilibrium(rho, u)
    if scheme == 2:
        g.set_forcing_scheme(2)
    if args.variant:
        g.variant = g.variants().index(args.variant)
    g.step(args.warmup)
    g.step(args.inner)
    torch.cuda.synchronize()
    rc, first = g.status()
    print(json.dumps({"case": args.case, "variant": g.variants()[g.variant],
                      "updates": args.warmup + args.inner, "status": rc}), flush=True)
    return 0 if rc == 0 else 1


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2602_06686_gb300 import build
    if rank == 0:
        build.build()
    barrier()
    from paper_2602_06686_gb300 import Lattice  # noqa: F401

    n = args.n
    inner = args.inner
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"]
    g = make_lattice("D2Q9", n, "F32")
    rho, u = workload_fields("double_shear", n)
    g.init_equilibrium(rho, u)
    chosen, times = g.autotune(reps=3)
    variant = g.variants()[chosen]
    names = g.variants()
    tune = dict(sorted(((names[v], round(t, 4)) for v, t in enumerate(times)), key=lambda kv: kv[1])[:8])
    N = g.N
    st = g.stream

    def one_step():
        g.step(inner)
        return g.diagnostics()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    launches0 = g.launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    w_start = time.perf_counter()
    t_start.record(st)
    diag = None
    for k in range(args.steps):
        ev[k][0].record(st)
        g.step(inner)
        ev[k][1].record(st)
        diag = g.diagnostics()  # FP64 reduction, synchronises
    t_end.record(st)
    t_end.synchronize()
    w_end = time.perf_counter()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop(w_start, w_end)
    launches = g.launches - launches0
    rc, first = g.status()
    total_s = t_start.elapsed_time(t_end) * 1e-3
    kernel_s = sum(a.elapsed_time(b) for a, b in ev) * 1e-3 / (args.steps * inner)
    units = float(N) * inner * args.steps
    units_all, total_all = aggregate(units, total_s)
    value = units_all / total_all / 1e6

    # e2e through the public API with host buffers (pinned), copies inside the region
    rho_h = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float64)).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    g.init_equilibrium_host_ptr(rho_h.data_ptr(), u_h.data_ptr())
    g.step(inner)
    g.macros_host_ptr(rho_o.data_ptr(), u_o.data_ptr())
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.init_equilibrium_host_ptr(rho_h.data_ptr(), u_h.data_ptr())
        g.step(inner)
        g.diagnostics()
        g.macros_host_ptr(rho_o.data_ptr(), u_o.data_ptr())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_units, e2e_all = aggregate(float(N) * inner * e2e_steps, e2e_s)
    e2e_value = e2e_units / e2e_all / 1e6
    h2d = rho_h.numel() * 8 + u_h.numel() * 8
    d2h = rho_o.numel() * 8 + u_o.numel() * 8 + 64
    # where the end-to-end time goes: the host-link copies of one step, each
    # timed alone (both calls synchronise; the init / macros kernels included)
    t0 = time.perf_counter()
    g.init_equilibrium_host_ptr(rho_h.data_ptr(), u_h.data_ptr())
    t_h2d = time.perf_counter() - t0
    g.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.macros_host_ptr(rho_o.data_ptr(), u_o.data_ptr())
    t_d2h = time.perf_counter() - t0

    bpn = BYTES_PER_NODE[("D2Q9", "F32")]
    achieved = bpn * N / kernel_s / 1e9
    khash = csrc_hash()
    ceiling = copy_ceiling_at(bpn * N // 2) if rank == 0 else None
    extra = {}
    if rank == 0 and not args.no_extra:
        del g
        torch.cuda.empty_cache()
        jobs = [
            ("d3q19_f32", lambda: secondary("D3Q19", 384, "F32", "taylor_green_3d", peak)),
            ("d3q19_f16", lambda: secondary("D3Q19", 384, "F16", "taylor_green_3d", peak)),
            ("d3q19_bf16", lambda: secondary("D3Q19", 384, "BF16", "taylor_green_3d", peak)),
            ("d2q9_f16", lambda: secondary("D2Q9", n, "F16", "double_shear", peak)),
            ("d2q9_trt_rlb_f32",
             lambda: secondary("D2Q9", n, "F32", "double_shear", peak, "TRT_RLB")),
            ("d2q9_trt_f32", lambda: secondary("D2Q9", n, "F32", "double_shear", peak, "TRT")),
            ("d3q19_trt_rlb_f32",
             lambda: secondary("D3Q19", 384, "F32", "taylor_green_3d", peak, "TRT_RLB")),
            ("d3q19_f64", lambda: secondary("D3Q19", 384, "F64", "taylor_green_3d", peak)),
            ("d3q19_f64_trt_rlb",
             lambda: secondary("D3Q19", 384, "F64", "taylor_green_3d", peak, "TRT_RLB")),
            ("d3q19_f64_trt",
             lambda: secondary("D3Q19", 384, "F64", "taylor_green_3d", peak, "TRT")),
            ("d2q9_f64", lambda: secondary("D2Q9", n, "F64", "double_shear", peak)),
            ("d2q9_f64_trt_rlb",
             lambda: secondary("D2Q9", n, "F64", "double_shear", peak, "TRT_RLB")),
            ("d2q9_f64_trt", lambda: secondary("D2Q9", n, "F64", "double_shear", peak, "TRT")),
            ("d3q19_f32_aa",
             lambda: secondary("D3Q19", 384, "F32", "taylor_green_3d", peak, layout="AA")),
            ("d3q27_f32", lambda: secondary("D3Q27", 384, "F32", "taylor_green_3d", peak)),
            ("d3q27_f16", lambda: secondary("D3Q27", 384, "F16", "taylor_green_3d", peak)),
            ("d3q27_trt_rlb_f32",
             lambda: secondary("D3Q27", 384, "F32", "taylor_green_3d", peak, "TRT_RLB")),
            ("d2q9_f32_scheme2",
             lambda: secondary("D2Q9", n, "F32", "double_shear", peak, scheme=2)),
            ("d3q19_f32_scheme2",
             lambda: secondary("D3Q19", 384, "F32", "taylor_green_3d", peak, scheme=2)),
            ("batch256", lambda: batched(peak)),
            ("precision", lambda: {"channel": precision_channel((0.1,)),
                                   "taylor_green_3d": precision_flow("taylor_green_3d", 96, 1000),
                                   "throughput": precision_throughput(peak)}),
        ]
        for key, fn in jobs:
            try:
                extra[key] = fn()
            except Exception as e:  # a failed side measurement must not lose the headline
                extra[key] = {"error": f"{type(e).__name__}: {e}"}
                torch.cuda.synchronize()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args.cpu_seconds)
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_all / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": headline_workload(n),
                   "updates_per_step": inner, "diagnostics_per_step": 1,
                   "l2": "inputs larger than L2 (2 x 604 MB population buffers)",
                   "variant": variant, "autotune_ms": tune,
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profile_traffic(khash),
                     "peak_source": peaks["source"], "bytes_per_node": bpn,
                     "kernel_ms": kernel_s * 1e3, "copy_ceiling": ceiling,
                     "frac_of_copy_ceiling": (achieved / max(ceiling["lbm_copy_gbs"],
                                                             ceiling["torch_copy_gbs"])
                                              if ceiling else None)},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "h2d_gbs": h2d / t_h2d / 1e9,
                "d2h_gbs": (d2h - 64) / t_d2h / 1e9},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "diverged": rc != 0,
        "diagnostics_last": {"mass": diag["mass"], "kinetic_energy": diag["kinetic_energy"],
                             "enstrophy": diag["enstrophy"]} if diag else None,
        "csrc_hash": khash,
        "extra_legend": EXTRA_LEGEND,
        "extra": compact(extra),
    }
    # the D3Q19 384^3 Taylor-Green figures last, so that a reader of the end of
    # the line sees the lattice the throughput target is stated for
    d3 = {k[6:] or "F32": extra[k] for k in ("d3q19_f32", "d3q19_f16", "d3q19_bf16", "d3q19_f64",
                                           "d3q19_f32_aa") if k in extra}
    if d3:
        d3 = {k.upper(): {f: v.get(f) for f in ("mlups", "frac", "copy", "alu_frac") if f in v}
              for k, v in d3.items()}
        if "F16" in d3 and d3["F16"]["mlups"] and d3.get("F32", {}).get("mlups"):
            d3["f16_over_f32"] = d3["F16"]["mlups"] / d3["F32"]["mlups"]
        line["d3q19_384"] = compact(dict(workload="D3Q19 P-TRT Taylor-Green 384^3, Re=1600, A/B "
                                                  "(F32_AA: in place)", **d3))
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--inner", type=int, default=100)
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--study", choices=["precision", "stability", "cylinder", "reynolds"],
                    default=None,
                    help="run the precision study or the critical-Mach stability sweep "
                         "instead of the benchmark")
    ap.add_argument("--sizes", default="1024,4096",
                    help="lattice sides of the Reynolds-number study")
    ap.add_argument("--cyl-steps", type=int, default=0,
                    help="square-cylinder steps (0: 30 diffusive e-folds)")
    ap.add_argument("--case", default=None,
                    help="LATTICE:STORAGE:NX,NY,NZ[:COLLISION[:LAYOUT]]: run one configuration "
                         "(--warmup + --inner updates) for a profiler and exit")
    ap.add_argument("--variant", default=None, help="kernel variant name for --case")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.study == "precision":
        return run_precision_study(args)
    if args.study == "stability":
        return run_stability_study(args)
    if args.study == "cylinder":
        return run_cylinder_study(args)
    if args.study == "reynolds":
        return run_reynolds_study(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
