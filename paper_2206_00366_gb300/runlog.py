"""JSON-lines record of a solver run.

One line for the configuration, one per periodic check, one summary:

    {"event": "config", ...the caller's configuration..., "nodes": N, "check_every": k}
    {"event": "check", "step": n, "mass": M, "momentum": [..], "kinetic_energy": E,
     "residual": r, "flags": f, "mass_drift": (M - M_first) / M_first,
     "steps": k, "wall_s": t, "mlups": N k / t / 1e6}
    {"event": "end", "steps": n, "checks": c, "stopped": "steps" | "residual" | "unstable",
     "wall_s": T, "mlups": ...}

Every figure of a check line is the library's own FP64 check (the sums of
rmrtlb_last_check: total mass and momentum, which the collision conserves,
Eq. 4-18-1; the residual ||u(t) - u(t - k)||_2 / ||u(t)||_2 against the
previous check).  The record only calls the solver's ``step`` and
``last_check``; the wall time of a line runs from before its steps to the
return of ``last_check``, which synchronises the solver's stream.
"""
from __future__ import annotations

import json
import time

FLAG_NAMES = {1: "nan_or_inf", 2: "density_not_positive", 4: "speed_at_or_above_cs", 8: "e3m12_saturated"}


def flag_names(flags: int) -> list:
    """The stability flags of a check word, by name."""
    return [name for bit, name in FLAG_NAMES.items() if int(flags) & bit]


def check_record(chk, first_mass=None) -> dict:
    """One check line from an rmrtlb_last_check vector (mass, momentum[3],
    kinetic energy, residual, step, flags).  The residual of the first
    check of a run is None (it has no previous snapshot)."""
    mass = float(chk[0])
    rec = {"event": "check", "step": int(chk[6]), "mass": mass, "momentum": [float(v) for v in chk[1:4]],
           "kinetic_energy": float(chk[4]), "residual": float(chk[5]) if chk[5] >= 0 else None,
           "flags": int(chk[7])}
    if rec["flags"]:
        rec["flag_names"] = flag_names(rec["flags"])
    if first_mass is not None and first_mass != 0.0:
        rec["mass_drift"] = (mass - first_mass) / first_mass
    return rec


def run_logged(solver, steps: int, path=None, config=None, stop_below=None, clock=time.perf_counter) -> list:
    """Advance `solver` by up to `steps` steps, one check interval at a
    time, and record every check.

    solver: a Solver (or anything with ``N``, ``params.check_every``,
    ``step(n)``, ``stats(allow_unstable)`` and
    ``last_check(allow_unstable)``) whose check interval k is positive and
    whose step counter is at a multiple of k (a fresh solver, or one
    stepped in multiples of k), so that every k steps end in a check;
    otherwise ValueError before any step.  The counter is read with one
    on-demand check (``stats``, which leaves the periodic check's residual
    snapshot alone).  The run stops at the first check past `steps`, at a check
    whose residual is below `stop_below`, or at a check that raised a
    stability flag.  path: a file the lines are appended to as they are
    made (None: no file).  Returns the records, the config line first and
    the end line last."""
    k = int(solver.params.check_every)
    if k <= 0:
        raise ValueError("run_logged needs a solver created with check_every > 0")
    if steps < 0:
        raise ValueError("steps must be >= 0")
    start = int(solver.stats(allow_unstable=True)[6])
    if start % k:
        raise ValueError(f"the solver's step counter {start} is not a multiple of its check interval {k}")
    records = []
    out = open(path, "a") if path is not None else None

    def emit(rec):
        records.append(rec)
        if out is not None:
            out.write(json.dumps(rec) + "\n")
            out.flush()

    try:
        emit({"event": "config", **(config or {}), "nodes": int(solver.N), "check_every": k})
        done, checks, first_mass, stopped, t_run = 0, 0, None, "steps", 0.0
        while done < steps:
            t0 = clock()
            solver.step(k)
            chk = solver.last_check(allow_unstable=True)
            wall = clock() - t0
            done += k
            checks += 1
            t_run += wall
            rec = check_record(chk, first_mass)
            if rec["step"] != start + done:
                raise RuntimeError(f"the last check is at step {rec['step']}, expected {start + done}")
            if first_mass is None:
                first_mass = rec["mass"]
                rec["mass_drift"] = 0.0
            rec.update(steps=k, wall_s=wall, mlups=solver.N * k / wall / 1e6 if wall > 0 else None)
            emit(rec)
            if rec["flags"]:
                stopped = "unstable"
                break
            if stop_below is not None and rec["residual"] is not None and rec["residual"] < stop_below:
                stopped = "residual"
                break
        emit({"event": "end", "steps": done, "checks": checks, "stopped": stopped, "wall_s": t_run,
              "mlups": solver.N * done / t_run / 1e6 if t_run > 0 else None})
    finally:
        if out is not None:
            out.close()
    return records
