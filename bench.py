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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "P-TRT MLUPS & % HBM roofline (D3Q19/D2Q9); FP16-store vs FP32 at set error"
BYTES_PER_NODE = {("D2Q9", "F64"): 144, ("D2Q9", "F32"): 72, ("D2Q9", "F16"): 36,
                  ("D2Q9", "BF16"): 36, ("D3Q19", "F64"): 304, ("D3Q19", "F32"): 152,
                  ("D3Q19", "F16"): 76, ("D3Q19", "BF16"): 76}
PROFILE = os.path.join(ROOT, "profiles", "stream_collide_d2q9_f32_4096.md")


def csrc_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2602_06686_gb300", "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


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

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
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
        for ln in self.lines:
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
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": f"D2Q9 P-TRT FP64 double shear {n}x{n}, {steps} steps ({dt:.1f} s)"}


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
        "config": {"workload": "D2Q9 P-TRT double shear layer (bounded CPU sample)",
                   "nx": n, "ny": n, "updates_per_step": inner},
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


def make_lattice(lat: str, n: int, storage: str, collision: str = "P_TRT"):
    from paper_2602_06686_gb300 import Lattice
    if lat == "D2Q9":
        # double shear layer: Re = U0 N / nu = 1e5, 1/tau- = 1.6 (the stability optimum of Sec. 3.1)
        return Lattice(lattice="D2Q9", nx=n, ny=n, nz=1, nu=0.1 * n / 1e5, tau_minus=1 / 1.6,
                       collision=collision, storage=storage)
    return Lattice(lattice="D3Q19", nx=n, ny=n, nz=n, nu=0.05 * n / (2 * math.pi * 1600),
                   Lambda=0.25, collision=collision, storage=storage)


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


def secondary(lat: str, n: int, storage: str, kind: str, peak: float, collision="P_TRT"):
    """MLUPS and roofline fraction of another workload (kernel-only, few steps)."""
    import torch
    g = make_lattice(lat, n, storage, collision)
    rho, u = workload_fields(kind, n)
    g.init_equilibrium(rho, u)
    g.autotune(reps=3, report=False)
    dt = time_kernel(g, 10, 3)
    N = g.N
    bpn = BYTES_PER_NODE[(lat, storage)]
    out = {"workload": f"{lat} {collision} {kind} {n}^{2 if lat == 'D2Q9' else 3} {storage}",
           "mlups": N / dt / 1e6, "kernel_ms": dt * 1e3,
           "achieved_gbs": bpn * N / dt / 1e9, "frac": bpn * N / dt / 1e9 / peak,
           "variant": g.variants()[g.variant]}
    rc, _ = g.status()
    out["diverged"] = rc != 0
    del g
    torch.cuda.empty_cache()
    return out


def batched(peak: float, count: int = 256, steps: int = 500):
    """256 uneven D2Q9 P-TRT double shear lattices (side lengths U{64..1024}, Re
    log-uniform in [1e3, 1e7], Lambda in {1/12, 3/16, 1/4}, seeded), FP32, advanced
    `steps` steps by the persistent kernel in a CUDA graph versus one launch per
    lattice per step."""
    import torch
    import workloads as W
    from paper_2602_06686_gb300 import Batch
    specs = []
    for d in W.batch_lattices(count):
        specs.append(dict(lattice="D2Q9", nx=d["nx"], ny=d["ny"], nu=0.1 * d["nx"] / d["Re"],
                          Lambda=d["Lambda"], collision="P_TRT", storage="F32"))
    b = Batch(specs)

    def init():
        for i, s in enumerate(specs):
            b.lattice(i).init_equilibrium(*W.double_shear_rect(s["nx"], s["ny"]))

    init()
    chosen, _ = b.autotune(steps=4)
    out = {"lattices": count, "nodes": b.nodes, "steps": steps,
           "tile": b.variants()[chosen]}
    for mode, name in ((0, "persistent_graph"), (1, "sequential_launches")):
        init()
        b.step(2, mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(steps, mode)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"mlups": b.nodes * steps / dt / 1e6, "seconds": dt,
                     "launches": b.launches}
    out["frac_persistent"] = out["persistent_graph"]["mlups"] * 1e6 * 72 / 1e9 / peak
    out["speedup_vs_sequential"] = (out["persistent_graph"]["mlups"]
                                    / out["sequential_launches"]["mlups"])
    out["diverged"] = [i for i in range(count) if b.lattice(i).status()[0] != 0]
    b.close()
    del b
    torch.cuda.empty_cache()
    return out


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
    t_start.record(st)
    diag = None
    for k in range(args.steps):
        ev[k][0].record(st)
        g.step(inner)
        ev[k][1].record(st)
        diag = g.diagnostics()  # FP64 reduction, synchronises
    t_end.record(st)
    t_end.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
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

    bpn = BYTES_PER_NODE[("D2Q9", "F32")]
    achieved = bpn * N / kernel_s / 1e9
    khash = csrc_hash()
    extra = {}
    if rank == 0 and not args.no_extra:
        del g
        torch.cuda.empty_cache()
        extra["d3q19_f32"] = secondary("D3Q19", 384, "F32", "taylor_green_3d", peak)
        extra["d3q19_f16"] = secondary("D3Q19", 384, "F16", "taylor_green_3d", peak)
        extra["d3q19_bf16"] = secondary("D3Q19", 384, "BF16", "taylor_green_3d", peak)
        extra["d2q9_f16"] = secondary("D2Q9", n, "F16", "double_shear", peak)
        extra["d2q9_trt_rlb_f32"] = secondary("D2Q9", n, "F32", "double_shear", peak, "TRT_RLB")
        extra["d2q9_trt_f32"] = secondary("D2Q9", n, "F32", "double_shear", peak, "TRT")
        extra["d3q19_trt_rlb_f32"] = secondary("D3Q19", 384, "F32", "taylor_green_3d", peak,
                                               "TRT_RLB")
        extra["d3q19_f64"] = secondary("D3Q19", 384, "F64", "taylor_green_3d", peak)
        extra["batch256"] = batched(peak)
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
        "config": {"workload": f"D2Q9 P-TRT double shear layer {n}x{n}, FP32 shifted storage, "
                               f"Re=1e5, 1/tau-=1.6, A/B buffers",
                   "updates_per_step": inner, "diagnostics_per_step": 1,
                   "l2": "inputs larger than L2 (2 x 604 MB population buffers)",
                   "variant": variant, "autotune_ms": tune,
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profile_traffic(khash),
                     "peak_source": peaks["source"], "bytes_per_node": bpn,
                     "kernel_ms": kernel_s * 1e3},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "diverged": rc != 0,
        "diagnostics_last": {"mass": diag["mass"], "kinetic_energy": diag["kinetic_energy"],
                             "enstrophy": diag["enstrophy"]} if diag else None,
        "extra": extra, "csrc_hash": khash,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--inner", type=int, default=100)
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
