"""Shared helpers of the parity tests: one physical configuration, run once
through the C ABI (CUDA path) and once through the oracle.

Both sides receive the same physical parameters and the same seeded inputs
(from ``workloads``); each derives its own weights, rates and equilibria.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import oracle.rmrt as R

KIND = {"nse": R.NSE, "nse_heluo": R.NSE_HELUO, "ncde_linear": R.NCDE_LINEAR, "ncde_quad": R.NCDE_QUAD,
        "ncde_simple_linear": R.NCDE_SIMPLE_LINEAR, "ncde_simple_quad": R.NCDE_SIMPLE_QUAD}


@dataclass
class Case:
    lattice: str = "D2Q9"
    shape: tuple = (37, 23, 1)            # nx, ny, nz
    spacing: tuple = (1.0, 0.6, 0.5)
    dt: float = 1.0
    cs2: float = 0.0                      # 0: default min c^2 / 3
    kind: str = "nse"
    basis: str = "raw"
    rho0: float = 1.0
    nu: float = 0.02
    nu_bulk: float = 0.05
    s_free: float = 1.1
    diffusivity: float = 0.01
    adv: tuple = (0.05, 0.02, -0.01)
    force: tuple = (0.0, 0.0, 0.0)
    source: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def d(self):
        return 2 if self.lattice in ("D2Q9", "D2Q5") else 3

    @property
    def field_shape(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def lat(self):
        return R.make_lattice(self.lattice, self.spacing, self.dt, self.cs2 if self.cs2 > 0 else None)

    def gpu_params(self):
        p = dict(cs2=self.cs2, rho0=self.rho0, nu=self.nu, nu_bulk=self.nu_bulk, s_free=self.s_free,
                 diffusivity=self.diffusivity, adv=self.adv, force=self.force, source=self.source)
        p.update(self.extra)
        return p

    def oracle_setup(self):
        lat = self.lat()
        if self.kind in ("nse", "nse_heluo"):
            r = R.rates_from_viscosity(lat, self.nu, self.nu_bulk, self.s_free)
        else:
            tau = self.diffusivity / (lat.cs2 * lat.dt) + 0.5
            d, s = lat.d, self.s_free
            r = R.Rates(s, np.full(d, 1.0 / tau), np.full(d, s), np.full(d, s), np.full((d, d), s), s)
        S = R.relaxation_matrix(lat, r)
        m = R.Model(KIND[self.kind], basis=self.basis, rho0=self.rho0, force=self.force[: lat.d],
                    source=self.source, adv=self.adv[: lat.d])
        return lat, m, S


_CACHE = {}


def oracle_run(case: Case, steps: int, fields=None, pops=None, key=None):
    """Oracle populations and (rho, u) after `steps` from fields or populations.

    With a `key` naming the seeded input, the result is cached for the
    session (the same oracle run serves every storage type)."""
    if key is not None:
        ck = (repr(case), steps, key)
        if ck not in _CACHE:
            _CACHE[ck] = oracle_run(case, steps, fields, pops)
        return _CACHE[ck]
    lat, m, S = case.oracle_setup()
    if pops is None:
        rho, u = fields
        f = R.init_equilibrium(lat, m, S, rho, u)
    else:
        f = pops.copy()
    f = R.step(lat, m, S, f, steps)
    rho, u = R.fields(lat, m, f)
    return f, rho, u


def gpu_solver(case: Case, storage: str, check_every: int = 0):
    from paper_2206_00366_gb300.rmrtlb import Solver
    p = case.gpu_params()
    p["check_every"] = check_every
    return Solver(case.lattice, case.shape, case.spacing, case.dt, p, case.kind, case.basis, storage)


def gpu_run(case: Case, storage: str, steps: int, fields=None, pops=None):
    import torch
    s = gpu_solver(case, storage)
    if pops is None:
        rho, u = fields
        s.init_equilibrium(np.ascontiguousarray(rho, dtype=np.float64),
                           np.ascontiguousarray(u, dtype=np.float64))
    else:
        s.set_populations(np.ascontiguousarray(pops, dtype=np.float64))
    s.step(steps)
    f = s.get_populations()
    rho, u = s.moments()
    torch.cuda.synchronize()
    return f, rho, u


def normwise(a, b):
    """max |a - b| / max |b| (per field)."""
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def component_scales(u_ref):
    """Denominator of each velocity component's normwise error: max |u_ref,c|,
    or max |u_ref| for a component below 1% of it (one that only the
    nonlinear terms feed, or none)."""
    umax = float(np.sqrt((u_ref * u_ref).sum(axis=0)).max())
    dens = []
    for c in range(u_ref.shape[0]):
        den = float(np.abs(u_ref[c]).max())
        dens.append(den if den >= 0.01 * umax else (umax if umax > 0 else 1.0))
    return np.array(dens)


def component_errors(u, u_ref):
    """max |u_c - u_ref,c| / component_scales(u_ref)_c for every component."""
    dens = component_scales(u_ref)
    return np.array([float(np.abs(u[c] - u_ref[c]).max()) for c in range(u_ref.shape[0])]) / dens


def normwise_u(u, u_ref):
    """Largest per-component normwise error of a velocity field (d, ...)."""
    return float(component_errors(u, u_ref).max())


def component_bounds(steps, q, c_max, f_max, rho_min, u_ref, gate, unit):
    """Per-component tolerance of a velocity comparison: the gate, or the
    accumulated rounding of a run in arithmetic of unit roundoff `unit`
    where that is larger.  A run holding full populations (up to f_max)
    passes every population through q multiply-adds per step and sums q
    populations times |c_j| <= c_max into the momentum, each rounding by at
    most `unit` of its size, so after n steps its velocity carries at most
    n q^2 unit c_max f_max / rho_min absolute (linear accumulation, the
    worst case)."""
    acc = steps * q * q * unit * c_max * f_max / rho_min
    return np.maximum(gate, acc / component_scales(u_ref))


def fp64_component_bounds(steps, q, c_max, f_max, rho_min, u_ref, gate=1e-12):
    """component_bounds of an FP64 comparison (unit 2^-53): the oracle's own
    accumulated rounding."""
    return component_bounds(steps, q, c_max, f_max, rho_min, u_ref, gate, 2.0 ** -53)


def of_max_u(u, u_ref):
    """Largest component error over max |u_ref| (the measure of the 16-bit
    storage gate: 2e-3 of max |u|)."""
    umax = float(np.sqrt((u_ref * u_ref).sum(axis=0)).max())
    return float(np.abs(u - u_ref).max() / (umax if umax > 0 else 1.0))
