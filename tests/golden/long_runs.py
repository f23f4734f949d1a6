"""Long oracle runs at the workloads' own step counts, stored for the GPU
parity tests and for the accuracy figures of the bench.

Writes ``tests/golden/long_<name>.npz`` by running ONLY the FP64 oracle
(``oracle.rmrt``) on seeded inputs from ``workloads``; no value comes from
the CUDA path.  Each file holds the final (rho or phi, u) on the full grid,
the same fields on a sub-lattice at intermediate steps (the error-vs-steps
record), and the case description.

Cases (the grids are downscales of the benched ones, the physics and the
step counts are the workloads' own):

* ``d2q9_nse_modes``: rD2Q9 NSE, 512 x 256, dx = 1, dy = 0.6 (c_s^2 = 0.12),
  four seeded Taylor-Green modes (seed 1, amplitudes in [0.005, 0.02]),
  nu = 0.01, nu_b = 0.02, free rates 1.1, 10,000 steps.
* ``d2q9_ncde_linear_hill`` / ``d2q9_ncde_quad_hill``: rD2Q9 NCDE with the
  linear (B = u phi) and quadratic (B = u phi^2 / 2) flux, Gaussian hill of
  peak 1 and sigma0 = 40, advection (0.05, 0.02), D = 0.005, phi0 = 0, same
  grid, 10,000 steps.
* ``d3q19_raw`` ... ``d3q27_central_hermite``: 3-D Taylor-Green, 64 x 64 x 32,
  dx = dy = 1, dz = 0.5 (c_s^2 = 1/12), u0 = 0.02, nu = 0.005, nu_b = 0.01,
  free rates 1.1, in the raw, central, Hermite and central-Hermite bases,
  2,000 steps.
* ``cavities``: the smallest of the 512 seeded lid-driven cavities of the
  batched workload (seed 4: sizes in [32, 512], dy/dx in {1/4 .. 4}, Re in
  [100, 1000], lid 0.05), each stepped alone from rest for 1,000 steps
  between half-way bounce-back walls with the moving lid: the first eight
  that stay stable are stored, the unstable ones smaller than those are
  listed with the step by which they left the method's range.  Each stored
  cavity also carries the run continued from its step-100 state rounded to
  FP32 (what the discrete problem does to an FP32-sized perturbation).
* ``cavity3d``: one rD3Q27 lid-driven cavity of the warm-start workload's
  kind, 32 x 32 x 16 nodes (dz = 0.5), Re 300, 1,000 steps from rest.

    python tests/golden/long_runs.py [name ...]      # default: every case
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE), HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import numpy as np  # noqa: E402

import oracle.rmrt as R  # noqa: E402
import workloads as W  # noqa: E402
from cases import Case  # noqa: E402
import store  # noqa: E402

SHAPE_2D = (512, 256, 1)
SPACING_2D = (1.0, 0.6, 1.0)
SHAPE_3D = (64, 64, 32)
SPACING_3D = (1.0, 1.0, 0.5)


def _case_2d(kind, f32_params=False):
    if kind == "nse":
        return Case("D2Q9", SHAPE_2D, SPACING_2D, kind="nse", nu=0.01, nu_bulk=0.02, s_free=1.1, rho0=1.0)
    r = (lambda v: float(np.float32(v))) if f32_params else float
    return Case("D2Q9", SHAPE_2D, SPACING_2D, kind=kind, diffusivity=r(0.005), adv=(r(0.05), r(0.02), 0.0),
                rho0=0.0, s_free=1.1)


def _case_3d(lattice, basis):
    return Case(lattice, SHAPE_3D, SPACING_3D, basis=basis, nu=0.005, nu_bulk=0.01, s_free=1.1, rho0=1.0)


# name -> (case, steps, snapshot steps, sub-lattice stride (x, y, z))
CASES = {
    "d2q9_nse_modes": (_case_2d("nse"), 10000, (100, 300, 1000, 3000), (8, 8, 1)),
    "d2q9_ncde_linear_hill": (_case_2d("ncde_linear"), 10000, (100, 300, 1000, 3000), (8, 8, 1)),
    "d2q9_ncde_quad_hill": (_case_2d("ncde_quad"), 10000, (100, 300, 1000, 3000), (8, 8, 1)),
    "d3q19_raw": (_case_3d("D3Q19", "raw"), 2000, (100, 300, 1000), (4, 4, 4)),
    "d3q19_central": (_case_3d("D3Q19", "central"), 2000, (100, 300, 1000), (4, 4, 4)),
    "d3q27_raw": (_case_3d("D3Q27", "raw"), 2000, (100, 300, 1000), (4, 4, 4)),
    "d3q27_central": (_case_3d("D3Q27", "central"), 2000, (100, 300, 1000), (4, 4, 4)),
    "d3q27_hermite": (_case_3d("D3Q27", "hermite"), 2000, (100, 300, 1000), (4, 4, 4)),
    "d3q27_central_hermite": (_case_3d("D3Q27", "central_hermite"), 2000, (100, 300, 1000), (4, 4, 4)),
    # conditioning of the quadratic hill: the same run from the initial
    # populations rounded to FP32 (a perturbation of the size FP32 storage
    # makes); how far it ends from the unperturbed run is what the discrete
    # problem itself does to an FP32 rounding
    "d2q9_ncde_quad_hill_f32init": (_case_2d("ncde_quad"), 10000, (100, 300, 1000, 3000), (8, 8, 1)),
    # the same with the state rounded to FP32 at step 1500, after the front
    # of the quadratic (Burgers) flux has steepened to the grid scale
    "d2q9_ncde_quad_hill_f32at1500": (_case_2d("ncde_quad"), 10000, (1500, 3000), (8, 8, 1)),
    # the same with the advection velocity and the diffusivity rounded to
    # FP32, the precision in which an FP32 implementation holds them
    "d2q9_ncde_quad_hill_f32params": (_case_2d("ncde_quad", f32_params=True), 10000, (1000, 3000), (8, 8, 1)),
    # the same with the populations rounded to FP32 after every step: what
    # storing them in FP32 (round to nearest) does to the run
    "d2q9_ncde_quad_hill_f32every": (_case_2d("ncde_quad"), 10000, (1000, 3000), (8, 8, 1)),
}
# perturbed runs: ("state", step at which the state is rounded to FP32) or
# ("params", 0) for constants rounded to FP32
PERTURBED = {"d2q9_ncde_quad_hill_f32init": ("state", 0), "d2q9_ncde_quad_hill_f32at1500": ("state", 1500),
             "d2q9_ncde_quad_hill_f32params": ("params", 0), "d2q9_ncde_quad_hill_f32every": ("every", 0)}
ROUNDED_AT = {k: v[1] for k, v in PERTURBED.items() if v[0] == "state"}


def initial_fields(case: Case):
    """Seeded initial (rho or phi, u) of a case, from ``workloads``."""
    nx, ny, nz = case.shape
    if case.kind.startswith("ncde"):
        phi = W.gaussian_hill((nz, ny, nx), case.spacing[:2], sigma0=40.0, peak=1.0)
        return phi, np.zeros((2, nz, ny, nx))
    if case.lattice == "D2Q9":
        cs2 = min(case.spacing[0], case.spacing[1]) ** 2 / 3
        return W.taylor_green_2d_modes(nx, ny, case.spacing[0], case.spacing[1], 1.0, cs2, seed=1)
    return W.taylor_green_3d(nx, ny, nz, case.spacing[0], case.spacing[1], case.spacing[2], 0.02, 1.0)


def sub(a, stride):
    """Every stride-th node of a field (..., nz, ny, nx)."""
    sx, sy, sz = stride
    return a[..., ::sz, ::sy, ::sx]


def run(name: str) -> str:
    case, steps, snaps, stride = CASES[name]
    lat, m, S = case.oracle_setup()
    rho, u = initial_fields(case)
    f = R.init_equilibrium(lat, m, S, rho, u)
    if ROUNDED_AT.get(name) == 0:
        f = f.astype(np.float32).astype(np.float64)
    arrays = {}
    t0 = time.time()
    done = 0
    every = PERTURBED.get(name, ("", 0))[0] == "every"
    for s in sorted(snaps) + [steps]:
        if every:
            for _ in range(s - done):
                f = R.step(lat, m, S, f, 1).astype(np.float32).astype(np.float64)
        else:
            f = R.step(lat, m, S, f, s - done)
        done = s
        if ROUNDED_AT.get(name) == s:
            f = f.astype(np.float32).astype(np.float64)
        r, v = R.fields(lat, m, f)
        if s == steps:
            arrays["rho"], arrays["u"] = r, v
        else:
            arrays[f"rho_sub_{s}"], arrays[f"u_sub_{s}"] = sub(r, stride), sub(v, stride)
        print(f"{name}: step {s} ({time.time() - t0:.0f} s)", flush=True)
    meta = {"name": name, "lattice": case.lattice, "shape": list(case.shape), "spacing": list(case.spacing),
            "kind": case.kind, "basis": case.basis, "rho0": case.rho0, "nu": case.nu, "nu_bulk": case.nu_bulk,
            "s_free": case.s_free, "diffusivity": case.diffusivity, "adv": list(case.adv), "steps": steps,
            "snapshots": list(snaps), "stride": list(stride), "cs2": lat.cs2,
            "rounded_to_f32_at_step": ROUNDED_AT.get(name), "rounded_to_f32_every_step": every,
            "writer": "tests/golden/long_runs.py (FP64 oracle only)", "oracle_seconds": round(time.time() - t0, 1)}
    return store.save(name, meta, arrays)


CAVITY_STEPS = 1000
CAVITY_CHECK = 100


def cavity_indices(domains):
    """Domain indices of a batch, smallest (by node count) first."""
    return sorted(range(len(domains)), key=lambda k: domains[k]["nx"] * domains[k]["ny"])


def run_cavities(count=8) -> str:
    """The smallest seeded config-4 cavities, each from rest for
    CAVITY_STEPS steps.  A domain whose state leaves the method's range
    (a non-finite value or max |u|^2 >= c_s^2 at one of the checks every
    CAVITY_CHECK steps) is recorded as unstable with that step; the first
    `count` that stay in range are stored for the parity comparison."""
    doms = W.cavity_domains(512, seed=4)
    arrays, kept, unstable = {}, [], {}
    t0 = time.time()
    for k in cavity_indices(doms):
        if len(kept) == count:
            break
        d = doms[k]
        lat = R.make_lattice("D2Q9", (d["dx"], d["dy"]), 1.0, d["cs2"] if d["cs2"] > 0 else None)
        S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, d["nu"], d["nu_bulk"], d["s_free"]))
        m = R.Model(R.NSE, rho0=1.0)
        f = R.init_equilibrium(lat, m, S, np.ones((1, d["ny"], d["nx"])), np.zeros((2, 1, d["ny"], d["nx"])))
        bad = None
        fp = None
        for s in range(CAVITY_CHECK, CAVITY_STEPS + 1, CAVITY_CHECK):
            f = R.step(lat, m, S, f, CAVITY_CHECK, walls=(0, 1), lid=(1, (d["lid_u"], 0.0), 1.0))
            rho, u = R.fields(lat, m, f)
            if not np.isfinite(f).all() or float((u * u).sum(axis=0).max()) >= lat.cs2:
                bad = s
                break
            if s == CAVITY_CHECK:
                # conditioning: the same run continued from this state rounded to FP32
                fp = f.astype(np.float32).astype(np.float64)
            else:
                fp = R.step(lat, m, S, fp, CAVITY_CHECK, walls=(0, 1), lid=(1, (d["lid_u"], 0.0), 1.0))
        if bad is not None:
            unstable[str(k)] = bad
            print(f"cavity {k}: {d['nx']} x {d['ny']} unstable by step {bad} ({time.time() - t0:.0f} s)", flush=True)
            continue
        arrays[f"rho_{k}"], arrays[f"u_{k}"] = rho, u
        arrays[f"rho_f32init_{k}"], arrays[f"u_f32init_{k}"] = R.fields(lat, m, fp)
        kept.append(k)
        print(f"cavity {k}: {d['nx']} x {d['ny']} ({time.time() - t0:.0f} s)", flush=True)
    meta = {"name": "cavities", "domains": [doms[k] for k in kept], "indices": kept, "steps": CAVITY_STEPS,
            "unstable": unstable, "seed": 4, "rho0": 1.0, "check_every": CAVITY_CHECK,
            "writer": "tests/golden/long_runs.py (FP64 oracle only)", "oracle_seconds": round(time.time() - t0, 1)}
    return store.save("cavities", meta, arrays)


# one rD3Q27 lid-driven cavity of the warm-start workload's kind (lid on the
# top z face moving +x at 0.05, dz = 0.5 dx, Re = U nx dx / nu), small
# enough for the oracle: 32 x 32 x 16 nodes, Re 300
CAVITY3D = dict(nx=32, ny=32, nz=16, dx=1.0, dy=1.0, dz=0.5, nu=0.05 * 32 / 300.0, nu_bulk=0.05 * 32 / 300.0,
                s_free=1.1, lid_u=0.05, cs2=0.0)


def run_cavity3d() -> str:
    d = CAVITY3D
    lat = R.make_lattice("D3Q27", (d["dx"], d["dy"], d["dz"]))
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, d["nu"], d["nu_bulk"], d["s_free"]))
    m = R.Model(R.NSE, rho0=1.0)
    shape = (d["nz"], d["ny"], d["nx"])
    f = R.init_equilibrium(lat, m, S, np.ones(shape), np.zeros((3,) + shape))
    t0 = time.time()
    f = R.step(lat, m, S, f, CAVITY_STEPS, walls=(0, 1, 2), lid=(2, (d["lid_u"], 0.0, 0.0), 1.0))
    rho, u = R.fields(lat, m, f)
    meta = {"name": "cavity3d", "domain": d, "lattice": "D3Q27", "steps": CAVITY_STEPS, "rho0": 1.0,
            "writer": "tests/golden/long_runs.py (FP64 oracle only)", "oracle_seconds": round(time.time() - t0, 1)}
    return store.save("cavity3d", meta, {"rho": rho, "u": u})


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES) + ["cavities", "cavity3d"]
    special = {"cavities": run_cavities, "cavity3d": run_cavity3d}
    for n in names:
        print(special[n]() if n in special else run(n), flush=True)
