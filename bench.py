"""Throughput of the fused RMRT-LB collide-and-stream step on GB300.

Workload (default): rD2Q9 Navier-Stokes on a periodic 4096 x 2048 grid,
dx = 1, dy = 0.6, c_s^2 = 0.12, four seeded Taylor-Green modes with
amplitudes in [0.005, 0.02], nu = 0.01, bulk viscosity 0.02, free rates
1.1, FP32 compute and storage, FP64 check every 100 steps.  One bench step
is one lattice time step over the whole grid.  The working set (two FP32
population lattices, 604 MB) is larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  Extra per-lattice lines are measured in the
same run and reported under "variants".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(lattice="D2Q9", shape=(4096, 2048, 1), spacing=(1.0, 0.6, 1.0), storage="f32", basis="raw",
                kind="nse", nu=0.01, nu_bulk=0.02, s_free=1.1, rho0=1.0, seed=1)
VARIANTS = [
    # (name, lattice, shape, spacing, storage, basis, kind)
    ("rD2Q9-f16", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "f16", "raw", "nse"),
    ("rD2Q9-bf16", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "bf16", "raw", "nse"),
    ("rD2Q9-ncde-quad-f32", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "f32", "raw", "ncde_quad"),
    ("rD3Q19-raw-f32", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "raw", "nse"),
    ("rD3Q19-central-f32", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "central", "nse"),
    ("rD3Q19-raw-f16", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "f16", "raw", "nse"),
    ("rD3Q19-central-f16", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "f16", "central", "nse"),
    ("rD3Q27-raw-f32", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "raw", "nse"),
    ("rD3Q27-central-f32", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "central", "nse"),
    ("rD3Q27-raw-f16", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f16", "raw", "nse"),
    ("rD3Q27-central-f16", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f16", "central", "nse"),
    ("rD3Q27-hermite-f32", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "hermite", "nse"),
    ("rD3Q27-central-hermite-f32", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f32", "central_hermite", "nse"),
    ("rD2Q9-f64", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "f64", "raw", "nse"),
    ("rD3Q27-raw-f64", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "f64", "raw", "nse"),
    ("rD2Q9-e3m12", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "e3m12", "raw", "nse"),
    ("rD2Q9-ncde-quad-e3m12", "D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "e3m12", "raw", "ncde_quad"),
    ("rD3Q19-raw-e3m12", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "e3m12", "raw", "nse"),
    ("rD3Q19-central-e3m12", "D3Q19", (256, 256, 128), (1.0, 1.0, 0.5), "e3m12", "central", "nse"),
    ("rD3Q27-raw-e3m12", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "e3m12", "raw", "nse"),
    ("rD3Q27-central-e3m12", "D3Q27", (256, 256, 128), (1.0, 1.0, 0.5), "e3m12", "central", "nse"),
]
Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
ESIZE = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "e3m12": 2}

# The stored oracle run each workload's accuracy is measured on: the same
# lattice, basis, physics and step count on a downscaled grid (the oracle
# cannot run the full grids), written by tests/golden/long_runs.py.
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def golden_for(lattice, basis, kind):
    if lattice == "D2Q9":
        return {"nse": "d2q9_nse_modes", "ncde_linear": "d2q9_ncde_linear_hill",
                "ncde_quad": "d2q9_ncde_quad_hill"}[kind]
    return f"{lattice.lower()}_{basis}"


def _golden(name):
    """(meta, arrays) of a stored oracle run, or None when it is absent."""
    sys.path.insert(0, GOLDEN_DIR)
    import store
    if not store.available(name):
        return None
    return store.load(name)


def oracle_error(lattice, storage, basis, kind):
    """Error against the FP64 oracle of one workload variant: the same
    kernel, storage and physics run on the stored oracle run's grid to its
    step count (the workload's own), compared node by node.  NSE: largest
    component error of u over max |u| (u_of_max), the largest of the
    components' errors each over its own maximum (u_per_component) and the
    normwise error of rho; NCDE: normwise phi."""
    import torch
    name = golden_for(lattice, basis, kind)
    g = _golden(name)
    if g is None:
        return {"case": name, "unavailable": "stored oracle run not present"}
    meta, a = g
    shape = tuple(meta["shape"])
    sp = tuple(meta["spacing"])
    s = make_solver(lattice, shape, sp, storage, basis, kind, 0)
    r_, u_ = initial_fields(lattice, shape, sp, kind, 1)
    s.init_equilibrium(torch.from_numpy(r_).cuda(), torch.from_numpy(u_).cuda())
    s.step(int(meta["steps"]))
    rho, u = s.moments()
    ro, uo = a["rho"], a["u"]
    out = {"case": name, "grid": list(shape), "steps": int(meta["steps"])}
    if kind.startswith("ncde"):
        out["phi"] = float(np.abs(rho - ro).max() / np.abs(ro).max())
        return out
    umax = float(np.sqrt((uo * uo).sum(axis=0)).max())
    per = []
    for c in range(uo.shape[0]):
        den = float(np.abs(uo[c]).max())
        per.append(float(np.abs(u[c] - uo[c]).max() / (den if den >= 0.01 * umax else umax)))
    # u_of_max is the measure the 16-bit gate (2e-3 of max |u|) applies to;
    # u_per_component divides each component's error by its own maximum
    out.update({"u_of_max": float(np.abs(u - uo).max() / umax), "u_per_component": max(per),
                "rho": float(np.abs(rho - ro).max() / np.abs(ro).max())})
    return out
CHECK_EVERY = 100
FALLBACK_HBM_GBS = 6800.0
TO_STEADY_CAP = 600000     # batched cavities: steps at most to residual 1e-6


STEP_KERNEL_SOURCES = ("rmrt_device.cuh", "rmrt_params.h", "rmrt_tuning.h", "rmrt_launch.cuh", "build.py")


def kernel_source_hash() -> str:
    """Hash of the files that define the step kernels and how they are built."""
    pkg = os.path.join(ROOT, "paper_2206_00366_gb300")
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        path = os.path.join(pkg, "csrc", f) if f != "build.py" else os.path.join(pkg, f)
        h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d and d[k]:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def profiled_entry(name: str):
    """The committed ncu summary of one step workload, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return d.get("workloads", {}).get(name)


def profiled_traffic(name: str):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    ent = profiled_entry(name)
    return ent.get("dram_bytes_per_launch") if ent else None


# FP64 pipe of GB300: 1.25 TFLOP/s nominal = 625 G DFMA instructions/s; a
# DADD or DMUL takes one pipe slot like a DFMA, so the FP64 step kernels are
# measured in pipe instructions against 625 G/s.
FP64_PIPE_GINST = 625.0


def fp64_alu_roof(name: str, nodes: int, kernel_ms: float):
    """ALU roofline of an FP64 step kernel from its ncu-counted DADD, DFMA
    and DMUL per node (None without a current profile)."""
    ent = profiled_entry(name)
    if not ent or "fp64_inst_per_node" not in ent:
        return None
    rate = nodes / (kernel_ms * 1e-3)
    ach = ent["fp64_inst_per_node"] * rate / 1e9
    return {"bound": "alu", "unit": "G FP64 inst/s", "achieved": round(ach, 1), "peak": FP64_PIPE_GINST,
            "frac": round(ach / FP64_PIPE_GINST, 4), "fp64_inst_per_node": ent["fp64_inst_per_node"],
            "gflops": round(ent["fp64_flop_per_node"] * rate / 1e9, 1),
            "peak_source": "nominal 1.25 TFLOP/s FP64 (DFMA) = 625 G pipe instructions/s"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        import shutil
        import tempfile
        if shutil.which("nvidia-smi") is None:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def solver_params(lattice, kind, check_every):
    return dict(rho0=1.0 if kind.startswith("nse") else 0.0, nu=0.01 if lattice == "D2Q9" else 0.005,
                nu_bulk=0.02 if lattice == "D2Q9" else 0.01, s_free=1.1, diffusivity=0.005,
                adv=(0.05, 0.02, 0.0), check_every=check_every)


def make_solver(lattice, shape, spacing, storage, basis, kind, check_every):
    from paper_2206_00366_gb300.rmrtlb import Solver
    return Solver(lattice, shape, spacing, 1.0, solver_params(lattice, kind, check_every), kind, basis, storage)


class SlabRun:
    """One rank's slab of the N-rank grid: the benched 4096 x 2048 grid
    stacked N times along y (each rank's slab holds the seeded single-GPU
    field, so the whole grid is that field repeated, periodic in y), with
    the halo exchange after every step.  One rank: the single grid."""

    def __init__(self, wl, rank, world, check_every):
        from paper_2206_00366_gb300.slab import Slab
        nx, ny, nz = wl["shape"]
        self.slab = Slab(wl["lattice"], (nx, ny * world, nz), wl["spacing"], 1.0,
                         solver_params(wl["lattice"], wl["kind"], check_every), wl["kind"], wl["basis"],
                         wl["storage"], rank=rank, world=world)
        self.solver = self.slab.solver
        self.stream = self.solver.stream

    def init_equilibrium(self, rho, u):
        self.solver.init_equilibrium(rho, u)            # this slab's part of the stacked field

    def step(self, n=1):
        self.slab.step(n)              # the last step's exchange stays in flight (lands in the next step)

    def finish(self):
        self.slab.finish()

    def moments(self, rho=None, u=None):
        self.finish()
        return self.solver.moments(rho, u)

    def last_check(self):
        self.finish()
        return self.solver.last_check()


def initial_fields(lattice, shape, spacing, kind, seed):
    import workloads as W
    nx, ny, nz = shape
    if kind.startswith("ncde"):
        phi = W.gaussian_hill((nz, ny, nx), spacing[:2], sigma0=40.0, peak=1.0)
        return phi, np.zeros((2, nz, ny, nx))
    if lattice == "D2Q9":
        cs2 = min(spacing[0], spacing[1]) ** 2 / 3
        return W.taylor_green_2d_modes(nx, ny, spacing[0], spacing[1], 1.0, cs2, seed=seed)
    return W.taylor_green_3d(nx, ny, nz, spacing[0], spacing[1], spacing[2], 0.02, 1.0)


def time_solver(solver, steps, warmup):
    """Device time of `steps` steps (no periodic check) with CUDA events on the
    solver's stream: (total ms, mean per-step ms)."""
    import torch
    stream = solver.stream
    for _ in range(warmup):
        solver.step(1)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        solver.step(1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    durs = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[steps]), statistics.mean(durs)


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over the ranks of the initialised process group (x
    itself on one rank): the timing rule of a replicated run."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job MLUPS of `world` ranks (slabs of one grid) that each
    advanced `nodes` nodes `steps` times, timed by the slowest rank."""
    return world * nodes * steps / seconds / 1e6


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2206_00366_gb300 import build as _build
    if rank == 0 or local == 0:
        _build.build()
    if world > 1:
        dist.barrier()

    wl = WORKLOAD
    nx, ny, nz = wl["shape"]
    nodes = nx * ny * nz
    rho, u = initial_fields(wl["lattice"], wl["shape"], wl["spacing"], wl["kind"], wl["seed"])
    solver = SlabRun(wl, rank, world, CHECK_EVERY)
    solver.init_equilibrium(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        solver.step(1)
    solver.finish()
    torch.cuda.synchronize()
    # timed region: barrier + synchronize on both sides, events on the solver's stream
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stream = solver.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            solver.step(1)
            if i == args.steps - 1:
                solver.finish()        # the last exchange lands inside the region
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = ev[0].elapsed_time(ev[args.steps])
    durs = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    plain = [d for i, d in enumerate(durs) if (args.warmup + i + 1) % CHECK_EVERY != 0]
    kern_ms = statistics.mean(plain) if plain else total_ms / args.steps
    checks_in_region = args.steps - len(plain)
    # The FP64 check runs every CHECK_EVERY steps; a timed region shorter
    # than that holds fewer checks than its share.  Time one step that ends
    # in a check and add the missing share, so that value is the throughput
    # of the workload with its checks.
    done = args.warmup + args.steps
    to_next = CHECK_EVERY - done % CHECK_EVERY
    if to_next > 1:
        solver.step(to_next - 1)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    solver.step(1)
    solver.finish()                    # the check runs once the step's exchange has landed
    c1.record(stream)
    torch.cuda.synchronize()
    check_ms = max(0.0, c0.elapsed_time(c1) - kern_ms)
    added_ms = max(0.0, args.steps / CHECK_EVERY - checks_in_region) * check_ms
    total_ms = max_over_ranks(total_ms + added_ms, "cuda")
    chk = solver.last_check()
    ms_per_step = total_ms / args.steps
    mlups = replica_mlups(world, nodes, args.steps, total_ms * 1e-3)

    # end to end through the C ABI with pinned host buffers
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    e2e_solver = SlabRun(wl, rank, world, CHECK_EVERY)
    e2e_solver.init_equilibrium(rho_h, u_h)
    e2e_solver.step(3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_solver.init_equilibrium(rho_h, u_h)           # host -> device inside the call
    e2e_solver.step(args.steps)
    e2e_solver.moments(rho_o, u_o)                     # device -> host inside the call
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, "cuda")
    d = 2 if wl["lattice"] == "D2Q9" else 3
    e2e = {"value": replica_mlups(world, nodes, args.steps, e2e_s), "unit": "MLUPS",
           "h2d_bytes_per_step": (1 + d) * nodes * 8 / args.steps,
           "d2h_bytes_per_step": (1 + d) * nodes * 8 / args.steps,
           "note": "init_equilibrium from pinned host rho,u + K steps + moments to pinned host"}
    del e2e_solver

    q = Q[wl["lattice"]]
    bytes_per_launch = 2 * q * ESIZE[wl["storage"]] * nodes
    peak, peak_kind = hbm_peak()
    achieved = bytes_per_launch / (kern_ms * 1e-3) / 1e9
    traffic = profiled_traffic("rD2Q9-f32")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_kind,
                "kernel": "step_kernel_x2<0, float, float, 0, 0, 1> (rD2Q9, FP32 storage and compute, raw "
                          "moments, unforced, NSE; two nodes per thread)",
                "algorithmic_bytes_per_launch": bytes_per_launch, "kernel_ms": round(kern_ms, 5)}
    accuracy = None
    if rank == 0:
        try:
            accuracy = oracle_error(wl["lattice"], wl["storage"], wl["basis"], wl["kind"])
        except Exception as ex:  # report, do not hide
            accuracy = {"error": str(ex)}

    variants = {}
    if rank == 0 and not args.no_variants:
        del solver
        torch.cuda.empty_cache()
        for name, lat, shape, sp, st, basis, kind in VARIANTS:
            try:
                s = make_solver(lat, shape, sp, st, basis, kind, 0)
                r_, u_ = initial_fields(lat, shape, sp, kind, 1)
                s.init_equilibrium(torch.from_numpy(r_).cuda(), torch.from_numpy(u_).cuda())
                nsteps = max(20, min(200, args.steps))
                tot, km = time_solver(s, nsteps, 5)
                n = shape[0] * shape[1] * shape[2]
                b = 2 * Q[lat] * ESIZE[st] * n
                ach = b / (km * 1e-3) / 1e9
                variants[name] = {"mlups": round(n * nsteps / (tot * 1e-3) / 1e6, 1),
                                  "kernel_ms": round(km, 5), "achieved_gbs": round(ach, 1),
                                  "frac_hbm": round(ach / peak, 4), "bytes_per_node": 2 * Q[lat] * ESIZE[st],
                                  "traffic": profiled_traffic(name)}
                if st == "f64":
                    variants[name]["alu"] = fp64_alu_roof(name, n, km)
                del s
                torch.cuda.empty_cache()
                variants[name]["oracle_err"] = oracle_error(lat, st, basis, kind)
            except Exception as ex:  # report, do not hide
                variants[name] = {"error": str(ex)}

    batched = warm = None
    if rank == 0 and not args.no_variants:
        try:
            batched = run_batched(args)
        except Exception as ex:  # report, do not hide
            batched = {"error": str(ex)}
        try:
            warm = run_warmstart(args)
        except Exception as ex:
            warm = {"error": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(budget_s=20.0)

    if rank == 0:
        launches = args.steps + 2 * (sum(1 for i in range(args.steps) if (args.warmup + i + 1) % CHECK_EVERY == 0))
        line = {
            "metric": "MLUPS", "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "rD2Q9 NSE Taylor-Green modes 4096x2048 dx=1 dy=0.6 FP32 storage",
                       "lattice": "rD2Q9", "nx": nx, "ny": ny, "storage": "f32", "basis": "raw",
                       "check_every": CHECK_EVERY,
                       "check_in_value": {"checks_in_timed_region": checks_in_region,
                                          "check_ms": round(check_ms, 5), "added_ms": round(added_ms, 5),
                                          "note": "the FP64 check every 100 steps is included in value: timed "
                                                  "in the region, or its share added when the region holds "
                                                  "fewer checks than steps/100"},
                       "l2": "working set 604 MB > L2 (129 MB); no flush",
                       "parallelism": (f"slab decomposition along y over {world} ranks (4096 x {2048 * world} "
                                       f"periodic grid, one 4096 x 2048 slab per GPU), NCCL halo exchange of "
                                       f"the crossing populations after every step" if world > 1 else "single")},
            "oracle_err": accuracy,
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "cpu_baseline": cpu, "variants": variants, "batched": batched,
            "warm_start": warm,
            "last_check": {"mass": chk[0], "residual": chk[5], "step": chk[6], "flags": chk[7]},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def batched_oracle_error(storage="f32"):
    """Error against the FP64 oracle of the batch kernels: the stored
    cavities of the batched workload (the smallest seeded ones that stay
    stable), 1,000 steps from rest in one batch, each against its oracle
    run; the largest normwise rho or u error over the cavities."""
    import workloads as W
    from paper_2206_00366_gb300.rmrtlb import Batch
    g = _golden("cavities")
    if g is None:
        return {"case": "cavities", "unavailable": "stored oracle run not present"}
    meta, a = g
    doms = W.cavity_domains(512, seed=4)
    idx = meta["indices"]
    b = Batch([doms[k] for k in idx], storage=storage, check_every=100, tol=1e-300)   # never converged
    b.tune(5)
    b.reset()
    b.step(int(meta["steps"]))
    worst = 0.0
    for i, k in enumerate(idx):
        rg, ug = b.fields(i)
        ro, uo = a[f"rho_{k}"], a[f"u_{k}"]
        worst = max(worst, float(np.abs(rg - ro).max() / np.abs(ro).max()),
                    float(np.abs(ug - uo).max() / np.abs(uo).max()))
    return {"case": "cavities", "domains": [int(k) for k in idx], "steps": int(meta["steps"]),
            "storage": storage, "max_normwise": worst,
            "oracle_unstable": {k: int(v) for k, v in meta["unstable"].items()}}


def run_batched(args):
    """Batched lid-driven cavities (512 seeded domains: sizes 32..512, dy/dx
    in {1/4..4}, Re 100..1000): throughput after tuning the launch shape,
    and cold-start time to residual 1e-6 of all 512 (capped at
    TO_STEADY_CAP steps), with the oracle error of the batch kernels."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2206_00366_gb300.rmrtlb import Batch
    out = {}
    doms = W.cavity_domains(512, seed=4)
    nodes = sum(d["nx"] * d["ny"] for d in doms)
    b = Batch(doms, storage="f32", check_every=100, tol=1e-6)
    width = b.tune(10)
    b.step(100)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nsteps = max(100, (args.steps // 100) * 100)
    e0.record(b.stream)
    b.step(nsteps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res, conv, act, done = b.status()
    out["throughput"] = {"domains": len(doms), "nodes": nodes, "tile_width": width, "tile_rows": b.tile_rows,
                         "nodes_per_thread": b.nodes_per_thread, "steps": nsteps,
                         "mlups": round(nodes * nsteps / (ms * 1e-3) / 1e6, 1),
                         "achieved_gbs": round(72 * nodes * nsteps / (ms * 1e-3) / 1e9, 1),
                         "unstable_domains": int((act == -1).sum()),
                         "note": "FP32, check every 100 steps in a CUDA graph; MLUPS counts every node of every "
                                 "domain while it is stepped"}
    # all 512 to steady state from rest (the same batch, reset)
    b.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issued = b.run(TO_STEADY_CAP)
    wall = time.perf_counter() - t0
    res, conv, act, done = b.status()
    ok = conv[act == 0]
    nn = np.array([d["nx"] * d["ny"] for d in doms])
    work = float((nn * np.where(act == 0, conv, issued)).sum())
    out["time_to_steady"] = {"domains": len(doms), "tol": 1e-6, "start": "cold (rest)",
                             "distribution": "sizes 32..512, dy/dx in {1/4,1/2,1,2,4}, Re 100..1000 (seed 4)",
                             "cap_steps": TO_STEADY_CAP, "steps_issued": int(issued), "wall_s": round(wall, 2),
                             "converged": int((act == 0).sum()), "unstable": int((act == -1).sum()),
                             "capped": int((act == 1).sum()),
                             "median_steps_to_tol": int(np.median(ok)) if len(ok) else None,
                             "p90_steps_to_tol": int(np.percentile(ok, 90)) if len(ok) else None,
                             "max_steps_to_tol": int(ok.max()) if len(ok) else None,
                             "node_updates": work, "mlups_effective": round(work / wall / 1e6, 1)}
    del b
    torch.cuda.empty_cache()
    out["oracle_err"] = batched_oracle_error()
    return out


def cavity3d_oracle_error(storage="f32"):
    """Error against the FP64 oracle of the rD3Q27 batch kernels the warm
    start runs on: the stored 32 x 32 x 16 lid-driven cavity (Re 300), 1,000
    steps from rest, normwise rho and u."""
    from paper_2206_00366_gb300.rmrtlb import Batch
    g = _golden("cavity3d")
    if g is None:
        return {"case": "cavity3d", "unavailable": "stored oracle run not present"}
    meta, a = g
    b = Batch([meta["domain"]], storage=storage, check_every=100, tol=1e-300, lattice="D3Q27")
    b.reset()
    b.step(int(meta["steps"]))
    rg, ug = b.fields(0)
    ro, uo = a["rho"], a["u"]
    return {"case": "cavity3d", "grid": [meta["domain"][k] for k in ("nx", "ny", "nz")], "steps": int(meta["steps"]),
            "storage": storage, "rho": float(np.abs(rg - ro).max() / np.abs(ro).max()),
            "u": float(np.abs(ug - uo).max() / np.abs(uo).max())}


def run_warmstart(args, re_seed=0):
    """rD3Q27 lid-driven cavity, 192 x 192 x 96 cells (dz/dx = 0.5, lid on
    the top z face moving +x at 0.05), Re drawn from [100, 1500] by seed:
    steps and wall time to residual 1e-6 from rest and from the committed
    network's prediction (its inference, upsampling and the f^eq + f^ne
    initialisation inside the warm time)."""
    import numpy as np

    from paper_2206_00366_gb300 import warmstart as WS
    if not os.path.exists(WS.WEIGHTS):
        return {"unavailable": "no trained weights committed"}
    net = WS.Net.load(WS.WEIGHTS)
    re = float(np.random.default_rng(re_seed).uniform(*WS.RE_RANGE))
    dom = WS.cavity((96, 192, 192), re)
    cold = WS.time_to_steady(dom, re, max_steps=400000)
    warm = WS.time_to_steady(dom, re, net=net, coarse=tuple(net.meta["shape"]), max_steps=400000)
    cu, wu = cold["u"], warm["u"]
    diff = float((wu - cu).abs().max() / cu.abs().max())
    ok = cold["state"] == 0 and warm["state"] == 0
    return {"workload": "rD3Q27 cavity 192x192x96, dz/dx=0.5, FP32 storage, raw moments", "re": round(re, 1),
            "re_seed": re_seed, "tol": 1e-6,
            "cold": {"steps": cold["steps"], "state": cold["state"], "wall_s": round(cold["wall_s"], 2)},
            "warm": {"steps": warm["steps"], "state": warm["state"], "wall_s": round(warm["wall_s"], 2),
                     "inference_and_init_s": round(warm["init_s"], 4)},
            "step_ratio_warm_over_cold": round(warm["steps"] / cold["steps"], 3) if ok else None,
            "time_ratio_warm_over_cold": round(warm["wall_s"] / cold["wall_s"], 3) if ok else None,
            "final_u_maxdiff_rel": diff,
            "oracle_err": cavity3d_oracle_error(),
            "network": {k: net.meta.get(k) for k in ("states", "converged", "shape", "epochs", "final_loss",
                                                      "holdout_u_rel_l2_median")}}


# ---------------------------------------------------------------- oracle timing
def _oracle_worker(nx, ny, steps, sync=False):
    """Runs in a child process with one BLAS thread: oracle steps on an
    nx x ny band of the workload; prints seconds.  With sync, prints "ready"
    after the set-up and one untimed step and waits for a line on stdin
    before the timed steps (so that concurrent workers overlap)."""
    import oracle.rmrt as R
    import workloads as W
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, 0.01, 0.02, 1.1))
    m = R.Model()
    rho, u = W.taylor_green_2d_modes(4096, 2048, 1.0, 0.6, 1.0, lat.cs2, seed=1)
    f = R.init_equilibrium(lat, m, S, rho[:, :ny, :nx].copy(), u[:, :, :ny, :nx].copy())
    f = R.step(lat, m, S, f, 1)
    if sync:
        print("ready", flush=True)
        sys.stdin.readline()
    t0 = time.perf_counter()
    R.step(lat, m, S, f, steps)
    print(json.dumps({"seconds": time.perf_counter() - t0}), flush=True)


def _one_thread_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def _oracle_child(nx, ny, steps):
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(nx), str(ny), str(steps)],
                       capture_output=True, text=True, env=_one_thread_env(), cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["seconds"]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_children(nx, ny, steps, procs):
    """`procs` concurrent one-thread oracle processes, each stepping its own
    nx x ny band `steps` times after a common start signal; returns the wall
    seconds from the signal until the last one finished."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", str(nx), str(ny), str(steps), "sync"]
    ps = [subprocess.Popen(cmd, stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=_one_thread_env(), cwd=ROOT) for _ in range(procs)]
    try:
        for p in ps:
            if p.stdout.readline().strip() != "ready":
                raise RuntimeError(p.stderr.read()[-2000:])
        t0 = time.perf_counter()
        for p in ps:
            p.stdin.write("go\n")
            p.stdin.flush()
        outs = [p.communicate() for p in ps]
        wall = time.perf_counter() - t0
    finally:
        for p in ps:
            if p.poll() is None:
                p.kill()
    for p, (out, err) in zip(ps, outs):
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
    return wall


def cpu_baseline(budget_s=20.0):
    """The oracle on the host: one core, and every core (one process per
    core, each on its own band of the workload)."""
    nx, ny = 1024, 512
    probe = _oracle_child(nx, ny, 1)
    steps = max(1, int(budget_s / max(probe, 1e-3)))
    secs = _oracle_child(nx, ny, steps)
    single = {"value": round(nx * ny * steps / secs / 1e6, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
              "sample": f"{steps} oracle steps on a {nx}x{ny} periodic band of the 4096x2048 workload "
                        f"(FP64 numpy, one BLAS thread), {secs:.1f} s"}
    procs = host_cores()
    if procs <= 1:
        return single
    wall = _oracle_children(nx, ny, steps, procs)
    return {"value": round(procs * nx * ny * steps / wall / 1e6, 4), "unit": "MLUPS", "cores": procs,
            "kind": "oracle",
            "sample": f"{procs} concurrent processes, one per host core, each {steps} oracle steps on its own "
                      f"{nx}x{ny} periodic band of the 4096x2048 workload (FP64 numpy, one BLAS thread each), "
                      f"{wall:.1f} s wall",
            "single_core": single}


def run_reference(args):
    """The oracle as it stands, on the host cores: each bench step is one
    oracle step on a band of the workload sized so that the K steps take
    about a minute."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nx = 512
    probe = _oracle_child(nx, 256, 1)
    t_node = probe / (nx * 256)
    ny = int(max(8, min(256, 60.0 / max(args.steps, 1) / t_node / nx)))
    procs = host_cores()
    # one process per host core on its own band; one untimed step inside each
    secs = _oracle_children(nx, ny, args.steps, procs)
    mlups = procs * nx * ny * args.steps / secs / 1e6
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    line = {
        "metric": "MLUPS", "value": round(mlups, 4), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "rD2Q9 NSE Taylor-Green modes 4096x2048 dx=1 dy=0.6 FP32 storage",
                   "lattice": "rD2Q9", "nx": 4096, "ny": 2048, "storage": "f32", "basis": "raw",
                   "check_every": CHECK_EVERY,
                   "l2": "working set 604 MB > L2 (129 MB); no flush",
                   "parallelism": "replicas" if world > 1 else "single"},
        "device": "host cores (the oracle runs on the CPU; no GPU is used by this arm)",
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": procs, "kind": "oracle",
                         "sample": f"each step: one FP64 oracle step in each of {procs} concurrent processes "
                                   f"(one per host core), each on its own {nx}x{ny} periodic band of the "
                                   f"4096x2048 workload, one BLAS thread each"},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_only(args):
    """One workload by name, no e2e / variants / oracle: the command the ncu
    summaries under profiles/ were taken with."""
    import torch
    from paper_2206_00366_gb300 import build as _build
    _build.build()
    if args.only == "batched-cavities":
        return run_only_batched(args)
    if args.only == "warmstart-train-step":
        return run_only_train_step(args)
    if args.only == "batched-to-steady":
        return run_only_batched_to_steady(args)
    table = {"rD2Q9-f32": ("D2Q9", (4096, 2048, 1), (1.0, 0.6, 1.0), "f32", "raw", "nse")}
    table.update({v[0]: v[1:] for v in VARIANTS})
    lat, shape, sp, st, basis, kind = table[args.only]
    s = make_solver(lat, shape, sp, st, basis, kind, 0)
    r_, u_ = initial_fields(lat, shape, sp, kind, 1)
    s.init_equilibrium(torch.from_numpy(r_).cuda(), torch.from_numpy(u_).cuda())
    tot, km = time_solver(s, args.steps, args.warmup)
    n = shape[0] * shape[1] * shape[2]
    b = 2 * Q[lat] * ESIZE[st] * n
    print(json.dumps({"only": args.only, "steps": args.steps, "mlups": round(n * args.steps / (tot * 1e-3) / 1e6, 1),
                      "kernel_ms": round(km, 5), "achieved_gbs": round(b / (km * 1e-3) / 1e9, 1),
                      "bytes_per_launch": b}))


def run_only_batched(args):
    """The 512 seeded rD2Q9 cavities, 128 x 1 tiles (no tuning), direct
    launches: `steps` steps after `warmup`."""
    import torch

    import workloads as W
    from paper_2206_00366_gb300.rmrtlb import Batch
    doms = W.cavity_domains(512, seed=4)
    b = Batch(doms, storage="f32", check_every=1000000, tol=1e-6, use_graphs=False)
    b.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nodes = sum(d["nx"] * d["ny"] for d in doms)
    print(json.dumps({"only": args.only, "steps": args.steps, "nodes": nodes,
                      "mlups": round(nodes * args.steps / (ms * 1e-3) / 1e6, 1),
                      "achieved_gbs": round(72 * nodes * args.steps / (ms * 1e-3) / 1e9, 1)}))


def run_only_batched_to_steady(args):
    """All 512 seeded rD2Q9 cavities from rest to residual 1e-6 (FP32, check
    every 100 steps, CUDA graphs, tuned tiles, tile queue; moment basis
    --basis), at most `steps` steps: wall time, how many converged or were
    retired as unstable, the distribution of steps to converge, and the
    residuals of those still stepping."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2206_00366_gb300.rmrtlb import Batch
    doms = W.cavity_domains(512, seed=4)
    b = Batch(doms, storage="f32", check_every=100, tol=1e-6, basis=args.basis)
    w = b.tune(5)
    b.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issued = b.run(args.steps)
    wall = time.perf_counter() - t0
    res, conv, act, _ = b.status()
    ok = conv[act == 0]
    nodes = np.array([d["nx"] * d["ny"] for d in doms])
    work = float((nodes * np.where(act == 0, conv, issued)).sum())
    stepping = res[act == 1]
    print(json.dumps({"only": args.only, "basis": args.basis, "domains": len(doms), "max_steps": args.steps,
                      "steps_issued": int(issued),
                      "wall_s": round(wall, 1), "tile": [w, b.tile_rows], "converged": int((act == 0).sum()),
                      "unstable": int((act == -1).sum()), "still_stepping": int((act == 1).sum()),
                      "steps_to_tol_median": int(np.median(ok)) if len(ok) else None,
                      "steps_to_tol_p90": int(np.percentile(ok, 90)) if len(ok) else None,
                      "steps_to_tol_max": int(ok.max()) if len(ok) else None,
                      "still_stepping_residual_q10_q50_q90": [float(np.quantile(stepping, x)) for x in (0.1, 0.5, 0.9)]
                      if len(stepping) else None,
                      "node_updates": work, "mlups_effective": round(work / wall / 1e6, 1)}))


def run_only_train_step(args):
    """Training steps of the warm-start network on a batch of 4 cavities of
    32 x 64 x 64 cells (zero targets): 4 forward, 3 input-gradient and 4
    weight-gradient convolutions on the tensor cores, MSE, Adam."""
    import torch

    from paper_2206_00366_gb300 import warmstart as WS
    net = WS.Net(seed=0)
    shape = (32, 64, 64)
    T = torch.zeros((4,) + shape + (4,), dtype=torch.float32, device="cuda")
    re = [200.0, 500.0, 800.0, 1100.0]
    for _ in range(args.warmup):
        net.train_step(re, shape, T, 1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.train_step(re, shape, T, 1e-3)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    fl = sum(2.0 * 4 * 32 * 64 * 64 * 27 * WS.CH[k] * WS.CH[k + 1] for k in range(4))
    print(json.dumps({"only": args.only, "steps": args.steps, "ms_per_step": round(ms, 3),
                      "conv_tflops": round(3 * fl / (ms * 1e-3) / 1e12, 1)}))


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--oracle-worker":
        _oracle_worker(int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]),
                       sync=len(sys.argv) > 5 and sys.argv[5] == "sync")
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default=None, help="time one named workload only (profiling)")
    ap.add_argument("--basis", default="raw", choices=["raw", "central", "hermite", "central_hermite"],
                    help="moment basis of --only batched-to-steady")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
