"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module only draws random numbers and evaluates initial/analytic fields;
it holds none of the lattice Boltzmann arithmetic (no weights, equilibria,
moments or relaxation).  Both the CUDA path and the oracle consume what it
returns; each side turns macroscopic fields into populations with its own
code.

Field layout: scalars (nz, ny, nx), vectors (d, nz, ny, nx), x fastest, node
i on axis alpha at physical coordinate i * dx_alpha.  All arrays are float64.
"""
from __future__ import annotations

import numpy as np


def grid(shape, dx):
    """Physical node coordinates (X, Y, Z) for shape (nz, ny, nx)."""
    nz, ny, nx = shape
    z = np.arange(nz) * (dx[2] if len(dx) > 2 else 1.0)
    y = np.arange(ny) * dx[1]
    x = np.arange(nx) * dx[0]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def taylor_green_2d(nx, ny, dx, dy, u0, rho0, cs2, phase=(0.0, 0.0), mode=(1, 1)):
    """2-D Taylor-Green vortex on a periodic nx*dx by ny*dy box.

    u_x = -u0 cos(kx x) sin(ky y), u_y = u0 (kx/ky) sin(kx x) cos(ky y),
    rho = rho0 - rho0 u0^2/(4 cs2) [cos 2kx x + (kx/ky)^2 cos 2ky y],
    kx = 2 pi mx/(nx dx), ky = 2 pi my/(ny dy).  Velocity decays as
    exp(-nu (kx^2 + ky^2) t) under the incompressible Navier-Stokes equations.
    """
    X, Y, _ = grid((1, ny, nx), (dx, dy))
    kx = 2 * np.pi * mode[0] / (nx * dx)
    ky = 2 * np.pi * mode[1] / (ny * dy)
    ax, ay = kx * X + phase[0], ky * Y + phase[1]
    ux = -u0 * np.cos(ax) * np.sin(ay)
    uy = u0 * (kx / ky) * np.sin(ax) * np.cos(ay)
    rho = rho0 - rho0 * u0 * u0 / (4 * cs2) * (np.cos(2 * ax) + (kx / ky) ** 2 * np.cos(2 * ay))
    return rho, np.stack([ux, uy])


def taylor_green_2d_modes(nx, ny, dx, dy, rho0, cs2, seed, n_modes=4,
                          amp=(0.005, 0.02), max_mode=8):
    """Sum of n_modes Taylor-Green modes with seeded wavenumbers, amplitudes
    (uniform in amp) and phases; density carries only the linear background
    rho0 (the pressure of a mode sum is not separable)."""
    rng = np.random.default_rng(seed)
    u = np.zeros((2, 1, ny, nx))
    for _ in range(n_modes):
        mx, my = rng.integers(1, max_mode + 1, size=2)
        a = rng.uniform(*amp)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        _, um = taylor_green_2d(nx, ny, dx, dy, a, rho0, cs2, phase=ph, mode=(mx, my))
        u += um
    return np.full((1, ny, nx), float(rho0)), u


def taylor_green_3d(nx, ny, nz, dx, dy, dz, u0, rho0):
    """Classic 3-D Taylor-Green initial field on a periodic box.

    u = u0 (sin kx x cos ky y cos kz z, -(kx/ky) cos kx x sin ky y cos kz z, 0),
    k_alpha = 2 pi / L_alpha; divergence-free; density rho0.
    """
    X, Y, Z = grid((nz, ny, nx), (dx, dy, dz))
    kx, ky, kz = 2 * np.pi / (nx * dx), 2 * np.pi / (ny * dy), 2 * np.pi / (nz * dz)
    ux = u0 * np.sin(kx * X) * np.cos(ky * Y) * np.cos(kz * Z)
    uy = -u0 * (kx / ky) * np.cos(kx * X) * np.sin(ky * Y) * np.cos(kz * Z)
    uz = np.zeros_like(ux)
    return np.full((nz, ny, nx), float(rho0)), np.stack([ux, uy, uz])


def gaussian_hill(shape, dx, sigma0, peak=1.0, center=None, adv=(0.0, 0.0, 0.0), diff=0.0, t=0.0,
                  images=1):
    """Isotropic Gaussian hill advected at constant velocity and diffusing.

    phi(x, t) = peak * s0^2/(s0^2 + 2 D t) exp(-|x - x0 - u t|^2 / (2 (s0^2 + 2 D t)))
    in 2-D (exponent d/2 on the prefactor in d dimensions), summed over
    periodic images within +-images box lengths.  sigma0 in physical units.
    """
    nz, ny, nx = shape
    d = 2 if nz == 1 else 3
    L = [nx * dx[0], ny * dx[1], (nz * dx[2] if d == 3 else 1.0)]
    if center is None:
        center = [0.5 * L[0], 0.5 * L[1], 0.5 * L[2] if d == 3 else 0.0]
    X, Y, Z = grid(shape, list(dx) + [1.0] * (3 - len(dx)))
    s2 = sigma0 ** 2 + 2 * diff * t
    pref = (sigma0 ** 2 / s2) ** (d / 2)
    phi = np.zeros(shape)
    rng = range(-images, images + 1)
    for ix in rng:
        for iy in rng:
            for iz in (rng if d == 3 else [0]):
                rx = X - center[0] - adv[0] * t - ix * L[0]
                ry = Y - center[1] - adv[1] * t - iy * L[1]
                r2 = rx * rx + ry * ry
                if d == 3:
                    rz = Z - center[2] - adv[2] * t - iz * L[2]
                    r2 = r2 + rz * rz
                phi += np.exp(-r2 / (2 * s2))
    return peak * pref * phi


def burgers_cole_hopf(nx, dx, U, diff, t, a=2.0, b=1.0, mode=1):
    """Exact periodic solution of phi_t + U phi phi_x = D phi_xx.

    With w = U phi this is viscous Burgers; Cole-Hopf gives
    w = 2 D b k sin(k x) e^{-D k^2 t} / (a + b cos(k x) e^{-D k^2 t}),
    k = 2 pi mode / (nx dx), a > b > 0.  Returns phi on x_i = i dx.
    """
    x = np.arange(nx) * dx
    k = 2 * np.pi * mode / (nx * dx)
    E = np.exp(-diff * k * k * t)
    w = 2 * diff * b * k * np.sin(k * x) * E / (a + b * np.cos(k * x) * E)
    return w / U


def random_populations(q, shape, seed, level=1.0, amp=0.05, base=None):
    """Random positive populations (q, nz, ny, nx) for parity tests.

    Each direction gets a seeded base share of `level` (or the q given
    `base` values, e.g. a rest state) and every value a relative
    perturbation uniform in +-amp.  No equilibrium is implied: the collision
    step is defined for any populations.
    """
    rng = np.random.default_rng(seed)
    if base is None:
        base = rng.uniform(0.5, 1.5, size=q)
        base *= level / base.sum()
    else:
        base = np.asarray(base, dtype=np.float64).reshape(q)
    noise = rng.uniform(-amp, amp, size=(q,) + tuple(shape))
    return base.reshape((q,) + (1,) * len(shape)) * (1.0 + noise)


def random_fields(shape, d, seed, rho0=1.0, drho=0.01, umax=0.03):
    """Smooth-free random (rho, u) fields for parity tests."""
    rng = np.random.default_rng(seed)
    rho = rho0 + drho * rng.uniform(-1, 1, size=shape)
    u = umax * rng.uniform(-1, 1, size=(d,) + tuple(shape))
    return rho, u


def cavity_domains(n, seed, size=(32, 512), ratios=(0.25, 0.5, 1.0, 2.0, 4.0), re=(100.0, 1000.0),
                   lid=0.05, s_free=1.1):
    """Seeded lid-driven cavities: nx, ny uniform in `size`, dy/dx drawn from
    `ratios` with the smaller spacing 1, Reynolds number uniform in `re`
    (Re = lid * nx * dx / nu), bulk viscosity equal to nu.  Returns a list of
    dicts with the fields of rmrtlb_domain."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny = (int(v) for v in rng.integers(size[0], size[1] + 1, size=2))
        r = float(rng.choice(ratios))
        dx, dy = (1.0, r) if r >= 1 else (1.0 / r, 1.0)
        Re = float(rng.uniform(*re))
        nu = lid * nx * dx / Re
        out.append(dict(nx=nx, ny=ny, dx=dx, dy=dy, nu=nu, nu_bulk=nu, s_free=s_free, lid_u=lid, cs2=0.0))
    return out
