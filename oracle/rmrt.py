"""Plain FP64 oracle for the rectangular MRT lattice Boltzmann (RMRT-LB) step.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code, table or constant
generator with the CUDA library, and it imports nothing from that package.

Everything here follows Chai, Yuan & Shi, "Rectangular multiple-relaxation-time
lattice Boltzmann method for the Navier-Stokes and nonlinear
convection-diffusion equations" (arXiv 2206.00366), and is written in the
paper's order and notation:

* velocities and weights ............ Sec. III, Eqs. (3-1), (3-2), (3-3-5), (3-3-8)
* general REDF g^eq(A, B, M) ........ Eqs. (3-3), (3-4)
* NCDE f^eq, G, F ................... Eqs. (4-11), (4-14), (4-14-1)
* NSE  f^eq, G, F ................... Eqs. (NSEfeq), (NSEGeq), (NSEFeq), (4-26)
* He-Luo equilibrium ................ Sec. IV Remark IV
* relaxation rates from nu, nu_b .... Eq. (4-31)
* S_2 block ......................... Eqs. (4-27), (4-27-1); inverted numerically
* raw-moment matrix M ............... Eq. (5-2)
* collision operator ................ Eqs. (5-1), (5-1-2)
* forced moment-space step .......... Eqs. (2-3), (2-2-3), (2-4-1), (2-4-2)
* propagation ....................... Eq. (2-2b)
* non-equilibrium initialisation .... Eqs. (4-29), (4-35), (fne)
* local stress and strain rate ...... Eqs. (4-32), (4-33)

Matrices are built numerically (M from the monomial list over the velocity
set, M^-1 and the S_2 block by numerical inversion, m^eq = M f^eq from the
explicit REDF); nothing uses closed-form equilibrium moments.  The one place
where the paper is garbled or silent, the reading taken is stated in the
docstring of the function concerned.

Pins of the auxiliary distribution G (computed in
``equilibrium_and_sources``), which carries no mass or momentum and so
escapes the invariant pins: its force part u F + F u (Eq. M2GComput a) by
the reduction of a forced step to the textbook Guo-forced MRT step; its
source part c_s^2 Sbar I and the NCDE's M_1G (Eq. 4-11) by steady sourced
flows with closed forms that a planted omission of G misses.

Array conventions: a population field is an array of shape (q, nz, ny, nx)
(2-D lattices use nz = 1), x fastest; a node list is an array of shape (q, n).
Lattice units: dt is explicit, c_alpha = dx_alpha / dt.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import product

import numpy as np

LATTICES = ("D2Q9", "D3Q19", "D3Q27")
AXIS_LATTICES = ("D2Q5", "D3Q7")     # rDdQ(2d+1): rest and axis directions only (Remark I of Sec. III)


# --------------------------------------------------------------------------
# Sec. III: velocity sets
# --------------------------------------------------------------------------
def velocity_indices(name: str) -> np.ndarray:
    """Integer lattice directions e_j (c_j = e_j * c), shape (q, d).

    rD2Q9 follows the column order of Eq. (3-1).  rD3Q27 follows Eq. (3-2):
    j = 0, the six axis directions j = 1..6, the xy edges j = 7..10, the xz
    edges j = 11..14, the yz edges j = 15..18 and the corners j = 19..26.
    The printed xz block (Eq. 3-2b, j = 11..14) lists (c1,0,c3) and
    (-c1,0,-c3) twice each; it is read as (c1,0,c3), (-c1,0,c3),
    (-c1,0,-c3), (c1,0,-c3), the same sign pattern as the yz block.  rD3Q19
    is the rD3Q27 set without the corners (j >= 19), as Sec. III states.
    rD2Q5 and rD3Q7 (Remark I) are the rest and axis directions, the first
    5 of rD2Q9 and the first 7 of rD3Q27.
    """
    if name == "D2Q5":
        return velocity_indices("D2Q9")[:5]
    if name == "D3Q7":
        return velocity_indices("D3Q27")[:7]
    if name == "D2Q9":
        ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
        ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
        return np.array([ex, ey], dtype=np.int64).T
    if name in ("D3Q19", "D3Q27"):
        ex = [0, 1, 0, 0, -1, 0, 0,
              1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0,
              1, 1, 1, -1, -1, -1, -1, 1]
        ey = [0, 0, 1, 0, 0, -1, 0,
              1, 1, -1, -1, 0, 0, 0, 0, 1, -1, -1, 1,
              1, 1, -1, 1, -1, -1, 1, -1]
        ez = [0, 0, 0, 1, 0, 0, -1,
              0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1,
              1, -1, 1, 1, -1, 1, -1, -1]
        e = np.array([ex, ey, ez], dtype=np.int64).T
        return e[:19] if name == "D3Q19" else e
    raise ValueError(f"unknown lattice {name!r}")


def weights(name: str, c: np.ndarray, cs2: float) -> np.ndarray:
    """Weights omega_j from the velocity-moment constraints of Sec. III.

    rD2Q9: Eq. (3-3-5) with c_{s1} = c_{s2} = c_s.
    rD3Q27: Eq. (3-3-8) with c_{s alpha} = c_s.  omega_19 is free in
    (0, c_s^2 / (8 c_alpha^2)); it is fixed to c_s^6 / (8 c1^2 c2^2 c3^2),
    the value for which every weight factors into one-dimensional weights.
    rD3Q19: Eq. (3-3-8) with omega_19 = 0 (Sec. III, special case (1)).
    rD2Q5 (type I, omega_5 = 0) and rD3Q7: omega_alpha = c_s^2 / (2 c_alpha^2)
    for the two directions along axis alpha (Remark I of Sec. III).
    omega_0 = 1 - sum_{j>0} omega_j in every case (Eqs. 3-1, 3-2).
    """
    e = velocity_indices(name)
    q = e.shape[0]
    w = np.zeros(q)
    if name in AXIS_LATTICES:
        for j in range(1, q):
            al = int(np.flatnonzero(e[j])[0])
            w[j] = cs2 / (2.0 * c[al] * c[al])
    elif name == "D2Q9":
        c1, c2 = c
        w5 = cs2 * cs2 / (4.0 * c1 * c1 * c2 * c2)
        w1 = cs2 / (2.0 * c1 * c1) - 2.0 * w5
        w2 = cs2 / (2.0 * c2 * c2) - 2.0 * w5
        w[[1, 3]] = w1
        w[[2, 4]] = w2
        w[5:9] = w5
    else:
        c1, c2, c3 = c
        w19 = cs2 ** 3 / (8.0 * (c1 * c2 * c3) ** 2) if name == "D3Q27" else 0.0
        w7 = cs2 * cs2 / (4.0 * c1 * c1 * c2 * c2) - 2.0 * w19
        w11 = cs2 * cs2 / (4.0 * c1 * c1 * c3 * c3) - 2.0 * w19
        w15 = cs2 * cs2 / (4.0 * c2 * c2 * c3 * c3) - 2.0 * w19
        w1 = cs2 / (2.0 * c1 * c1) - 2.0 * (w7 + w11) - 4.0 * w19
        w2 = cs2 / (2.0 * c2 * c2) - 2.0 * (w7 + w15) - 4.0 * w19
        w3 = cs2 / (2.0 * c3 * c3) - 2.0 * (w11 + w15) - 4.0 * w19
        w[[1, 4]] = w1
        w[[2, 5]] = w2
        w[[3, 6]] = w3
        w[7:11] = w7
        w[11:15] = w11
        w[15:19] = w15
        if name == "D3Q27":
            w[19:27] = w19
    w[0] = 1.0 - w[1:].sum()
    return w


@dataclass
class Lattice:
    """A rectangular rDdQq lattice (Sec. III) in the paper's notation."""

    name: str
    dx: tuple            # spacings Delta x_alpha
    dt: float
    cs2: float           # c_s^2, the same along every axis (c_{s alpha} = c_s)
    d: int = field(init=False)
    q: int = field(init=False)
    e: np.ndarray = field(init=False)    # (q, d) integer directions
    c: np.ndarray = field(init=False)    # (d,) c_alpha = Delta x_alpha / Delta t
    cv: np.ndarray = field(init=False)   # (q, d) velocities c_j
    w: np.ndarray = field(init=False)    # (q,) weights

    def __post_init__(self):
        self.e = velocity_indices(self.name)
        self.q, self.d = self.e.shape
        self.dx = tuple(float(v) for v in self.dx[: self.d])
        self.c = np.array(self.dx) / self.dt
        self.cv = self.e * self.c[None, :]
        self.w = weights(self.name, self.c, self.cs2)


def make_lattice(name: str, dx, dt: float = 1.0, cs2: float | None = None) -> Lattice:
    """Build a lattice; c_s^2 defaults to min_alpha c_alpha^2 / 3 (rD3Q7:
    min_alpha c_alpha^2 / 4).

    The paper leaves c_s a free parameter subject to 0 < c_s^2 < c_alpha^2
    and omega_j >= 0 (Sec. III).  The default reduces to c^2/3 on the
    standard lattice; on rD3Q7, c^2/3 would make omega_0 = 0 there (Remark
    II: the rest velocity drops out), so its default is c^2/4, the usual
    D3Q7 choice (weights 1/4, 1/8).  A configuration with a negative weight,
    or with c_s^2 >= min c_alpha^2, is rejected.
    """
    d = 2 if name in ("D2Q9", "D2Q5") else 3
    c = np.array([float(v) for v in dx[:d]]) / dt
    if cs2 is None or cs2 <= 0:
        cs2 = float(np.min(c * c)) / (4.0 if name == "D3Q7" else 3.0)
    lat = Lattice(name, tuple(dx), dt, float(cs2))
    if not np.all(cs2 < c * c):
        raise ValueError("c_s^2 must be below every c_alpha^2")
    if np.any(lat.w < 0):
        raise ValueError(f"negative weight for {name} at c={c}, cs2={cs2}")
    return lat


# --------------------------------------------------------------------------
# Eq. (5-2): raw (natural) moment basis and the transformation matrix M
# --------------------------------------------------------------------------
def monomials(name: str) -> list:
    """Exponent tuples (m, n[, p]) of the raw moments, lowest order first.

    rD2Q9: the nine rows of Eq. (Md2q9), in that order
    (1, x, y, xx, yy, xy, xyy, xxy, xxyy).
    rD3Q27: all 27 exponents in {0,1,2}^3 of Eq. (5-2).
    rD3Q19: the paper prints no rD3Q19 basis; it is read as the 19 monomials
    of Eq. (5-2) that have at least one zero exponent (every other monomial
    vanishes on the rD3Q19 velocities).
    rD2Q5, rD3Q7: 1, the first powers and the squares of each axis (the
    raw moments that do not vanish identically on axis-only velocities).
    """
    if name == "D2Q9":
        return [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (1, 2), (2, 1), (2, 2)]
    if name == "D2Q5":
        return [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2)]
    if name == "D3Q7":
        return [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2)]
    allm = sorted(product(range(3), repeat=3), key=lambda a: (sum(a), [-v for v in a]))
    if name == "D3Q19":
        allm = [a for a in allm if min(a) == 0]
    return allm


def moment_order(name: str) -> np.ndarray:
    return np.array([sum(a) for a in monomials(name)])


def moment_matrix(lat: Lattice) -> np.ndarray:
    """M with rows c_{jx}^m c_{jy}^n c_{jz}^p over the velocity set (Eq. 5-2)."""
    mons = monomials(lat.name)
    M = np.ones((len(mons), lat.q))
    for k, a in enumerate(mons):
        for al in range(lat.d):
            M[k] *= lat.cv[:, al] ** a[al]
    return M


def central_moment_matrices(lat: Lattice, u: np.ndarray, hermite: bool = False) -> np.ndarray:
    """Per-node moment matrices Mbar(u) = N(u) M of Sec. V, shape (n, q, q).

    Row k of the monomial (m, n, p) is evaluated over the velocities j as
    prod_a P_k_a(c_ja - u_a): with P_k(xi) = xi^k the central-moment
    (cascaded) basis; with hermite, P_0 = 1, P_1 = xi, P_2 = xi^2 - c_s^2
    (the Hermite polynomials with the lattice's c_s^2), which gives the
    Hermite basis at u = 0 and the central-Hermite basis at the local u.
    Both are raw moments times a lower-triangular N (Eq. 5-1-1).  u (n, d).
    """
    mons = monomials(lat.name)
    n = u.shape[0]
    Mb = np.ones((n, len(mons), lat.q))
    for k, a in enumerate(mons):
        for al in range(lat.d):
            xi = lat.cv[None, :, al] - u[:, al, None]
            if hermite:
                Mb[:, k, :] *= (1.0, xi, xi * xi - lat.cs2)[a[al]] if a[al] else 1.0
            elif a[al]:
                Mb[:, k, :] *= xi ** a[al]
    return Mb


# --------------------------------------------------------------------------
# Eqs. (3-3), (3-4): the general rectangular EDF g^eq(A, B, M)
# --------------------------------------------------------------------------
def geq(lat: Lattice, A, B, Mt) -> np.ndarray:
    """g^eq_j(A, B, M) = omega_j (A + c~_j . B + Q~_j : M), shape (q, n).

    A: (n,), B: (n, d), Mt: (n, d, d) symmetric.  With Q_j = c_j c_j - Delta2,
    Q~_{j aa} = Q_{j aa} / (c_s^2 (c_a^2 - c_s^2)) and
    Q~_{j ab} = Q_{j ab} / (2 c_s^4) for a != b (Eq. 3-4, c_{s alpha} = c_s).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Mt = np.asarray(Mt, dtype=np.float64)
    cs2, c, cv = lat.cs2, lat.c, lat.cv
    g = A[None, :] + (cv @ B.T) / cs2
    for a in range(lat.d):
        for b in range(lat.d):
            if a == b:
                Q = cv[:, a] * cv[:, a] - cs2
                g += (Q / (cs2 * (c[a] * c[a] - cs2)))[:, None] * Mt[None, :, a, a]
            else:
                Q = cv[:, a] * cv[:, b]
                g += (Q / (2.0 * cs2 * cs2))[:, None] * Mt[None, :, a, b]
    return lat.w[:, None] * g


# --------------------------------------------------------------------------
# Relaxation: Eq. (4-31) rates, Eqs. (4-27)/(4-27-1) S_2 block, Eq. (5-1) S
# --------------------------------------------------------------------------
@dataclass
class Rates:
    """Relaxation rates of the block matrix S (Sec. V, Eq. 5-1)."""

    s0: float                 # zeroth order
    s1: np.ndarray            # (d,) first order (diagonal S_1)
    s_shear: np.ndarray       # (d,) s_{s alpha}
    s_bulk: np.ndarray        # (d,) s_{b alpha}
    s_off: np.ndarray         # (d, d) s_{alpha beta}, alpha != beta (symmetric)
    s_free: float             # every moment of order >= 3
    s2_diag_block: np.ndarray = None   # (d, d), filled by relaxation_matrix


def rates_from_viscosity(lat: Lattice, nu: float, nu_bulk: float, s_free: float,
                         s0: float | None = None, s1: float | None = None) -> Rates:
    """Rates that give kinematic viscosity nu and bulk viscosity nu_bulk.

    Eq. (4-31) with mu = rho nu and mu_b = rho nu_b:
      nu   = (1/s_ab - 1/2) c_s^2 dt                     (alpha != beta)
      nu   = (1/2)(1/s_sa - 1/2)(c_a^2 - c_s^2) dt
      nu_b = (1/d)(1/s_ba - 1/2)(c_a^2 - c_s^2) dt
    s_0 and S_1 do not enter the NSE; they default to s_free.
    """
    d, cs2, dt, c = lat.d, lat.cs2, lat.dt, lat.c
    s_ab = 1.0 / (nu / (cs2 * dt) + 0.5)
    s_s = 1.0 / (2.0 * nu / ((c * c - cs2) * dt) + 0.5)
    s_b = 1.0 / (d * nu_bulk / ((c * c - cs2) * dt) + 0.5)
    s_off = np.full((d, d), s_ab)
    np.fill_diagonal(s_off, 0.0)
    s0 = s_free if s0 is None else s0
    s1 = s_free if s1 is None else s1
    return Rates(s0, np.full(d, s1), s_s, s_b, s_off, s_free)


def nu_bulk_from_rate(lat: Lattice, s_e: float) -> float:
    """Bulk viscosity for a single bulk rate s_e given on the x axis.

    Reading of a bulk "rate s_e" in terms of Eq. (4-31b): nu_b is the value
    that rate gives on axis 1, nu_b = (1/d)(1/s_e - 1/2)(c_1^2 - c_s^2) dt;
    the per-axis s_{b alpha} then follow from nu_b.
    """
    return (1.0 / lat.d) * (1.0 / s_e - 0.5) * (lat.c[0] ** 2 - lat.cs2) * lat.dt


def s2_diag_block(lat: Lattice, r: Rates) -> np.ndarray:
    """The d x d block of S_2 acting on (m_xx, m_yy[, m_zz]).

    Built as the numerical inverse of S_2^(1) = diag(1/s_sa) + a b^T / d with
    a_a = (1/s_ba - 1/s_sa)(c_a^2 - c_s^2) and b_b = 1/(c_b^2 - c_s^2)
    (Eq. 4-27-1); Eq. (5-8-1) gives the same matrix in closed form.
    """
    c2 = lat.c * lat.c - lat.cs2
    a = (1.0 / r.s_bulk - 1.0 / r.s_shear) * c2
    b = 1.0 / c2
    S2inv = np.diag(1.0 / r.s_shear) + np.outer(a, b) / lat.d
    return np.linalg.inv(S2inv)


def relaxation_matrix(lat: Lattice, r: Rates) -> np.ndarray:
    """Dense S in the raw basis: block-diagonal (the special case after Eq. 5-8).

    Order 0: s_0; order 1: diag(S_1); order 2: the S_2 block of Eq. (5-8)
    (dense d x d on the diagonal second moments, s_ab on the mixed ones);
    every higher moment: s_free.
    """
    mons = monomials(lat.name)
    q = len(mons)
    S = np.zeros((q, q))
    blk = s2_diag_block(lat, r)
    diag2 = {}
    for k, a in enumerate(mons):
        o = sum(a)
        if o == 0:
            S[k, k] = r.s0
        elif o == 1:
            S[k, k] = r.s1[int(np.argmax(a))]
        elif o == 2 and max(a) == 2:
            diag2[int(np.argmax(a))] = k
        elif o == 2:
            al, be = [i for i in range(lat.d) if a[i] == 1]
            S[k, k] = r.s_off[al, be]
        else:
            S[k, k] = r.s_free
    for al, ka in diag2.items():
        for be, kb in diag2.items():
            S[ka, kb] = blk[al, be]
    return S


def s2_apply(lat: Lattice, S: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Apply the order-2 block of a raw-basis S to symmetric tensors X (n,d,d).

    Used for (I - S_2/2) in M_2G (Eq. 4-26): the second moments of X are
    laid out as a raw-moment vector, multiplied by S, and read back.
    """
    mons = monomials(lat.name)
    idx = {}
    for k, a in enumerate(mons):
        if sum(a) == 2:
            nz = [i for i in range(lat.d) for _ in range(a[i])]
            idx[(nz[0], nz[1])] = k
    n = X.shape[0]
    vec = np.zeros((len(mons), n))
    for (al, be), k in idx.items():
        vec[k] = X[:, al, be]
    out = S @ vec
    Y = np.zeros_like(X)
    for (al, be), k in idx.items():
        Y[:, al, be] = out[k]
        Y[:, be, al] = out[k]
    return Y


# --------------------------------------------------------------------------
# Model closures (Sec. IV)
# --------------------------------------------------------------------------
NSE, NSE_HELUO, NCDE_LINEAR, NCDE_QUAD = "nse", "nse_heluo", "ncde_linear", "ncde_quad"
# the simplified NCDE of Eq. (4-16): linear EDF, G from the time derivative of B
NCDE_SIMPLE_LINEAR, NCDE_SIMPLE_QUAD = "ncde_simple_linear", "ncde_simple_quad"
NCDE_SIMPLE = (NCDE_SIMPLE_LINEAR, NCDE_SIMPLE_QUAD)
NCDE_KINDS = (NCDE_LINEAR, NCDE_QUAD) + NCDE_SIMPLE
RAW, CENTRAL, HERMITE, CENTRAL_HERMITE = "raw", "central", "hermite", "central_hermite"


@dataclass
class Model:
    """What one collision needs besides the populations.

    kind: NSE (Eq. NSEfeq), NSE_HELUO (Remark IV of Sec. IV), NCDE_LINEAR or
    NCDE_QUAD (Eq. 4-14).  force / source: the NSE body force Fbar and source
    Sbar (Eq. NSE), or the NCDE source S (Eq. NCDE); each is a constant or a
    per-node array (force (d, n), source (n,)) on the node list being
    collided.  adv: the constant advection velocity of the NCDE.  rho0:
    reference density of the He-Luo equilibrium.
    """

    kind: str = NSE
    basis: str = RAW
    rho0: float = 1.0
    force: tuple = (0.0, 0.0, 0.0)
    source: float = 0.0
    adv: tuple = (0.0, 0.0, 0.0)


def force_of(m: Model, d: int, n: int) -> np.ndarray:
    """Body force as an (n, d) array."""
    F = np.asarray(m.force, dtype=np.float64)
    if F.ndim == 1:
        return np.broadcast_to(F[:d], (n, d)).copy()
    return F[:d].reshape(d, n).T.copy()


def source_of(m: Model, n: int) -> np.ndarray:
    """Source term as an (n,) array."""
    return np.broadcast_to(np.asarray(m.source, dtype=np.float64), (n,)).copy()


def ncde_flux(m: Model, phi: np.ndarray, d: int):
    """B(phi), C(phi) and B'(phi) for the two NCDE variants.

    The paper keeps B, C and D general (Eq. NCDE, Eq. 4-11).  Taken here with
    D = phi I, beta = 1 and C = int B' B' dphi (first case of Eq. 4-11):
      linear:     B = u phi,        C = u u phi,          B' = u
      quadratic:  B = u phi^2 / 2,  C = u u phi^3 / 3,    B' = u phi
    with u the constant advection velocity.  The simplified kinds of
    Eq. (4-16) take C = 0 with the same B.
    """
    u = np.asarray(m.adv[:d], dtype=np.float64)
    uu = np.outer(u, u)
    if m.kind in NCDE_SIMPLE:
        lin = m.kind == NCDE_SIMPLE_LINEAR
        B = (phi if lin else 0.5 * phi * phi)[:, None] * u[None, :]
        Bp = np.broadcast_to(u, (phi.size, d)).copy() if lin else phi[:, None] * u[None, :]
        return B, np.zeros((phi.size, d, d)), Bp
    if m.kind == NCDE_LINEAR:
        B = phi[:, None] * u[None, :]
        C = phi[:, None, None] * uu[None]
        Bp = np.broadcast_to(u, (phi.size, d)).copy()
    else:
        B = 0.5 * (phi * phi)[:, None] * u[None, :]
        C = (phi ** 3 / 3.0)[:, None, None] * uu[None]
        Bp = phi[:, None] * u[None, :]
    return B, C, Bp


def macroscopic(lat: Lattice, m: Model, fbar: np.ndarray):
    """Conserved fields from f-bar on a node list (q, n).

    NCDE, Eq. (2-4-1): phi = sum_j fbar_j + dt S / 2.
    NSE, Eq. (2-4-2): rho = sum_j fbar_j + dt Sbar / 2,
                      u = (sum_j c_j fbar_j + dt Fbar / 2) / rho.
    He-Luo (Remark IV of Sec. IV): u = (sum_j c_j fbar_j + dt Fbar/2) / rho0.
    Returns (density or phi (n,), velocity (n, d)); for the NCDE the
    velocity is the advection velocity.
    """
    dt, d = lat.dt, lat.d
    n = fbar.shape[1]
    rho = fbar.sum(axis=0) + 0.5 * dt * source_of(m, n)
    if m.kind in NCDE_KINDS:
        u = np.broadcast_to(np.asarray(m.adv[:d], float), (rho.size, d)).copy()
        return rho, u
    F = force_of(m, d, n)
    j = lat.cv.T @ fbar + 0.5 * dt * F.T
    den = m.rho0 if m.kind == NSE_HELUO else rho
    return rho, (j / den).T


def equilibrium_and_sources(lat: Lattice, m: Model, S: np.ndarray, rho, u, dBdt=None):
    """f^eq, G and F on a node list, each of shape (q, n).

    NSE (Eqs. NSEfeq, NSEGeq, NSEFeq):
      f^eq = g^eq(rho, rho u, rho u u)
      F    = g^eq(Sbar, Fbar, -c_s^2 Sbar I)
      G    = g^eq(0, 0, M_2G), M_2G = (I - S_2/2)(u Fbar + Fbar u + c_s^2 Sbar I)
             (Eq. M2GComput a).
    He-Luo: f^eq = g^eq(rho, rho0 u, rho0 u u) (Remark IV of Sec. IV).
    NCDE (Eqs. 4-14, 4-14-1): f^eq = g^eq(phi, B, C) (D = phi I, beta = 1),
      F = g^eq(S, 0, 0) = omega S, G = g^eq(0, M_1G, 0) with
      M_1G = (I - S_1/2) B' S (Eq. 4-11, first case).
    Simplified NCDE (Eq. 4-16): f^eq = g^eq(phi, B, 0), F = omega S,
      G = g^eq(0, (I - S_1/2) dB/dt, 0), dB/dt given per node (n, d).

    G is pinned by the Guo-forced MRT reduction (force part of M_2G), by
    steady sourced flows (source part of M_2G, M_1G of the NCDE) and, for
    the simplified NCDE, by the planted omission of dB/dt.
    """
    d, n, cs2 = lat.d, rho.size, lat.cs2
    I = np.eye(d)
    if m.kind in NCDE_SIMPLE:
        B, C, _ = ncde_flux(m, rho, d)
        feq = geq(lat, rho, B, C)
        Sn = source_of(m, n)
        F = geq(lat, Sn, np.zeros((n, d)), np.zeros((n, d, d)))
        s1 = np.array([S[k, k] for k, a in enumerate(monomials(lat.name)) if sum(a) == 1])
        dB = np.zeros((n, d)) if dBdt is None else dBdt
        G = geq(lat, np.zeros(n), (1.0 - 0.5 * s1)[None, :] * dB, np.zeros((n, d, d)))
        return feq, G, F
    if m.kind in (NCDE_LINEAR, NCDE_QUAD):
        B, C, Bp = ncde_flux(m, rho, d)
        feq = geq(lat, rho, B, C)
        Sn = source_of(m, n)
        F = geq(lat, Sn, np.zeros((n, d)), np.zeros((n, d, d)))
        s1 = np.array([S[k, k] for k, a in enumerate(monomials(lat.name)) if sum(a) == 1])
        M1G = (1.0 - 0.5 * s1)[None, :] * Bp * Sn[:, None]
        G = geq(lat, np.zeros(n), M1G, np.zeros((n, d, d)))
        return feq, G, F
    if m.kind == NSE_HELUO:
        feq = geq(lat, rho, m.rho0 * u, m.rho0 * np.einsum("na,nb->nab", u, u))
    else:
        feq = geq(lat, rho, rho[:, None] * u, rho[:, None, None] * np.einsum("na,nb->nab", u, u))
    Fb = force_of(m, d, n)
    Sb = source_of(m, n)
    F = geq(lat, Sb, Fb, -cs2 * Sb[:, None, None] * I[None])
    X = (np.einsum("na,nb->nab", u, Fb) + np.einsum("na,nb->nab", Fb, u)
         + cs2 * Sb[:, None, None] * I[None])
    M2G = X - 0.5 * s2_apply(lat, S, X)
    G = geq(lat, np.zeros(n), np.zeros((n, d)), M2G)
    return feq, G, F


# --------------------------------------------------------------------------
# Collision in moment space and propagation (Eqs. 2-2-3, 2-2b)
# --------------------------------------------------------------------------
def collide(lat: Lattice, m: Model, S: np.ndarray, fbar: np.ndarray, dBdt=None) -> np.ndarray:
    """Post-collision populations on a node list (q, n), Eq. (2-2-3).

    Raw basis:     m*  = mbar - S (mbar - m^eq) + dt (m_G + (I - S/2) m_F),
                   fbar* = M^-1 m*, with mbar = M fbar, m^eq = M f^eq, etc.
    Central basis: the same with M replaced per node by the central-moment
                   matrix Mbar(u) = N(u) M and S by Sbar (Eq. 5-1-2), so the
                   collision matrix is Lambda = Mbar^-1 Sbar Mbar; Mbar is
                   inverted numerically at every node.
    Hermite and central-Hermite bases: Mbar = N M with the Hermite rows of
                   central_moment_matrices at u = 0 or at the local u (the
                   other bases Sec. V names as special cases of Eq. 5-1-2).
    """
    dt = lat.dt
    rho, u = macroscopic(lat, m, fbar)
    feq, G, F = equilibrium_and_sources(lat, m, S, rho, u, dBdt)
    I = np.eye(S.shape[0])
    if m.basis == RAW:
        M = moment_matrix(lat)
        mb, meq, mG, mF = M @ fbar, M @ feq, M @ G, M @ F
        mstar = mb - S @ (mb - meq) + dt * (mG + (I - 0.5 * S) @ mF)
        return np.linalg.solve(M, mstar)
    shifted = m.basis in (CENTRAL, CENTRAL_HERMITE)
    Mb = central_moment_matrices(lat, u if shifted else np.zeros_like(u),
                                 hermite=m.basis in (HERMITE, CENTRAL_HERMITE))
    k = np.einsum("nkj,jn->kn", Mb, fbar)
    keq = np.einsum("nkj,jn->kn", Mb, feq)
    kG = np.einsum("nkj,jn->kn", Mb, G)
    kF = np.einsum("nkj,jn->kn", Mb, F)
    kstar = k - S @ (k - keq) + dt * (kG + (I - 0.5 * S) @ kF)
    return np.linalg.solve(Mb, kstar.T[:, :, None])[:, :, 0].T


def opposite(lat: Lattice) -> np.ndarray:
    """Index of -c_j for every j."""
    e = lat.e
    return np.array([int(np.where((e == -e[j]).all(axis=1))[0][0]) for j in range(lat.q)])


def stream(lat: Lattice, fstar: np.ndarray, walls: tuple = (), lid=None) -> np.ndarray:
    """Propagation f_j(x + c_j dt) = f*_j(x), Eq. (2-2b).

    Periodic on every axis, except that an axis listed in `walls` (0 = x,
    1 = y, 2 = z) is closed by walls half a spacing outside its first and
    last node (half-way bounce-back: a population that would leave through
    the wall returns to its node in the opposite direction).  The paper
    treats no boundaries; walls serve the Poiseuille, Couette and cavity
    checks.  `lid` = (axis, u_wall, rho_w) makes the wall beyond the last
    node of that axis move with velocity u_wall: a population j reflected
    there gains 2 omega_j rho_w (c_j . u_wall) / c_s^2, the linear term of
    the REDF (Eq. 3-3).  Walls are applied axis by axis in increasing order,
    so a corner population that crosses the lid gets the lid term.
    """
    out = np.empty_like(fstar)
    for j in range(lat.q):
        sh = [0, 0, 0]
        for al in range(lat.d):
            sh[2 - al] = int(lat.e[j, al])
        out[j] = np.roll(fstar[j], shift=sh, axis=(0, 1, 2))
    if walls:
        opp = opposite(lat)
        for al in sorted(walls):
            ax = 2 - al
            n = fstar.shape[1 + ax]
            for j in range(lat.q):
                ej = int(lat.e[j, al])
                if ej == 0:
                    continue
                first = [slice(None)] * 3
                first[ax] = 0 if ej > 0 else n - 1
                # populations arriving at the first (last) node from outside
                val = fstar[opp[j]][tuple(first)]
                if lid is not None and lid[0] == al and ej < 0:
                    uw = np.asarray(lid[1], dtype=np.float64)[: lat.d]
                    val = val + 2.0 * lat.w[j] * lid[2] * float(lat.cv[j] @ uw) / lat.cs2
                out[j][tuple(first)] = val
    return out


def step(lat: Lattice, m: Model, S: np.ndarray, fbar: np.ndarray, nsteps: int = 1,
         walls: tuple = (), lid=None, state: dict | None = None) -> np.ndarray:
    """nsteps of collide-and-stream on a field (q, nz, ny, nx).

    The simplified NCDE kinds (Eq. 4-16) need B at the previous step: it is
    kept in `state["B"]` (node list (n, d)) across calls when a dict is
    passed; with no previous value dB/dt is taken as zero (the first step
    after initialisation), dB/dt = (B(t) - B(t - dt)) / dt afterwards.
    """
    shape = fbar.shape
    f = fbar
    state = {} if state is None else state
    for _ in range(nsteps):
        fl = f.reshape(lat.q, -1)
        dB = None
        if m.kind in NCDE_SIMPLE:
            phi, _ = macroscopic(lat, m, fl)
            B, _, _ = ncde_flux(m, phi, lat.d)
            prev = state.get("B")
            dB = np.zeros_like(B) if prev is None else (B - prev) / lat.dt
            state["B"] = B
        fs = collide(lat, m, S, fl, dB).reshape(shape)
        f = stream(lat, fs, walls, lid)
    return f


def fields(lat: Lattice, m: Model, fbar: np.ndarray):
    """(rho or phi, u) of a population field; rho (nz,ny,nx), u (d,nz,ny,nx)."""
    shp = fbar.shape[1:]
    rho, u = macroscopic(lat, m, fbar.reshape(lat.q, -1))
    return rho.reshape(shp), u.T.reshape((lat.d,) + shp)


def init_equilibrium(lat: Lattice, m: Model, S: np.ndarray, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """f-bar = f^eq(rho, u) on a field; rho (nz,ny,nx), u (d,nz,ny,nx).

    The initial state carries no non-equilibrium part (Eq. fne is not added).
    For the NCDE, rho is phi and u is ignored (the advection velocity is used).
    """
    shp = rho.shape
    r = rho.reshape(-1).astype(np.float64)
    uu = u.reshape(lat.d, -1).T.astype(np.float64)
    feq, _, _ = equilibrium_and_sources(lat, m, S, r, uu)
    return feq.reshape((lat.q,) + shp)


def local_stress(lat: Lattice, m: Model, r: Rates, fbar: np.ndarray):
    """Local viscous stress and strain rate of the NSE, Eqs. (4-32), (4-33).

    With X = sum_k c_k c_k f_k^ne + (dt/2)(u Fbar + Fbar u + c_s^2 Sbar I),
    the stress K_mu (grad u + grad u^T) = -(I - S_2/2) X and the strain rate
    (grad u + grad u^T)/2 = -(K_mu^-1/2)(I - S_2/2) X, every product taken
    entry by entry, S_2 the matrix of entries s_sa (diagonal) and s_ab,
    K_mu of Eq. (4-29a) with the local density.  f^ne = f - f^eq with
    f = fbar + dt F/2 (Eq. 2-3); the second moment of F = g^eq(Sbar, Fbar,
    -c_s^2 Sbar I) vanishes (Eq. 3-5), so sum c c f^ne = sum c c (fbar - f^eq).
    fbar (q, nz, ny, nx); returns (stress, strain), each (d, d, nz, ny, nx).
    """
    d, cs2, dt, c = lat.d, lat.cs2, lat.dt, lat.c
    shp = fbar.shape[1:]
    fl = fbar.reshape(lat.q, -1)
    n = fl.shape[1]
    if m.kind not in (NSE, NSE_HELUO):
        raise ValueError("the local stress is defined for the NSE")
    rho, u = macroscopic(lat, m, fl)
    fc = m.rho0 * np.ones(n) if m.kind == NSE_HELUO else rho
    feq = geq(lat, rho, fc[:, None] * u, fc[:, None, None] * np.einsum("na,nb->nab", u, u))
    m2 = np.einsum("ja,jb,jn->abn", lat.cv, lat.cv, fl - feq)
    F = force_of(m, d, n)
    Sb = source_of(m, n)
    X = m2 + 0.5 * dt * (np.einsum("na,nb->abn", u, F) + np.einsum("na,nb->abn", F, u))
    X += 0.5 * dt * cs2 * Sb[None, None, :] * np.eye(d)[:, :, None]
    stress = np.zeros((d, d, n))
    strain = np.zeros((d, d, n))
    for a in range(d):
        for b in range(d):
            if a == b:
                s = r.s_shear[a]
                K = 0.5 * (1.0 / s - 0.5) * rho * (c[a] * c[a] - cs2) * dt
            else:
                s = r.s_off[a, b]
                K = (1.0 / s - 0.5) * rho * cs2 * dt
            stress[a, b] = -(1.0 - 0.5 * s) * X[a, b]
            strain[a, b] = stress[a, b] / (2.0 * K)
    return stress.reshape((d, d) + shp), strain.reshape((d, d) + shp)


def velocity_gradient(lat: Lattice, u: np.ndarray) -> np.ndarray:
    """g[a, b] = d u_b / d x_a on a field u (d, nz, ny, nx); shape (d, d, nz, ny, nx).

    The paper gives no difference stencil (it derives the local stress of
    Eqs. 4-32/4-33 precisely to avoid one).  Reading taken for the
    initialisation of Eq. (fne): second-order central differences inside the
    domain, first-order one-sided differences at the first and last node of
    an axis, zero along an axis with a single node; spacing dx_a = c_a dt.
    """
    d = lat.d
    g = np.zeros((d, d) + u.shape[1:])
    for a in range(d):
        ax = 2 - a                # array axis of x_a in (nz, ny, nx)
        n = u.shape[1 + ax]
        if n < 2:
            continue
        h = lat.dx[a]
        for b in range(d):
            ub = u[b]
            gb = np.empty_like(ub)
            sl = lambda i: tuple(slice(None) if k != ax else i for k in range(3))
            gb[sl(slice(1, n - 1))] = (ub[sl(slice(2, n))] - ub[sl(slice(0, n - 2))]) / (2.0 * h)
            gb[sl(0)] = (ub[sl(1)] - ub[sl(0)]) / h
            gb[sl(n - 1)] = (ub[sl(n - 1)] - ub[sl(n - 2)]) / h
            g[a, b] = gb
    return g


def noneq_second_moment(lat: Lattice, r: Rates, rho: np.ndarray, grad: np.ndarray) -> np.ndarray:
    """m_2^ne = sum_k c_k c_k f_k^ne of Eq. (4-35) without forcing or source.

    m_2^ne = -(I - S_2/2)^-1 K_mu (grad u + grad u^T), the products taken
    entry by entry, with S_2 the matrix of entries s_sa (diagonal) and s_ab
    (off-diagonal) named below Eq. (4-32), and the viscosity tensor of
    Eq. (4-29a): K_mu,aa = (1/2)(1/s_sa - 1/2) rho (c_a^2 - c_s^2) dt,
    K_mu,ab = (1/s_ab - 1/2) rho c_s^2 dt.  rho (n,), grad (d, d, n);
    returns (n, d, d).
    """
    d, cs2, dt, c = lat.d, lat.cs2, lat.dt, lat.c
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    out = np.zeros((rho.size, d, d))
    for a in range(d):
        for b in range(d):
            if a == b:
                s = r.s_shear[a]
                K = 0.5 * (1.0 / s - 0.5) * rho * (c[a] * c[a] - cs2) * dt
            else:
                s = r.s_off[a, b]
                K = (1.0 / s - 0.5) * rho * cs2 * dt
            strain = grad[a, b].reshape(-1) + grad[b, a].reshape(-1)
            out[:, a, b] = -K * strain / (1.0 - 0.5 * s)
    return out


def init_noneq(lat: Lattice, m: Model, S: np.ndarray, r: Rates, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """f-bar = f^eq(rho, u) + f^ne, f^ne = g^eq(0, 0, m_2^ne) (Eq. fne), with
    m_2^ne from Eq. (4-35) and the velocity gradient of velocity_gradient.
    NSE only; rho (nz,ny,nx), u (d,nz,ny,nx)."""
    shp = rho.shape
    feq = init_equilibrium(lat, m, S, rho, u)
    m2 = noneq_second_moment(lat, r, rho, velocity_gradient(lat, u))
    n = rho.size
    fne = geq(lat, np.zeros(n), np.zeros((n, lat.d)), m2)
    return feq + fne.reshape((lat.q,) + shp)


def collide_stream_at(lat: Lattice, m: Model, S: np.ndarray, fbar: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """One step's result at selected nodes of a periodic field.

    nodes: (n, 3) integer (z, y, x).  Returns (q, n): fbar_j(x, t+dt) =
    f*_j(x - e_j), the post-collision value at the upstream node.  Used to
    check full-size runs without stepping the whole field.
    """
    nz, ny, nx = fbar.shape[1:]
    out = np.empty((lat.q, nodes.shape[0]))
    for j in range(lat.q):
        ez = int(lat.e[j, 2]) if lat.d == 3 else 0
        ey, ex = int(lat.e[j, 1]), int(lat.e[j, 0])
        z = (nodes[:, 0] - ez) % nz
        y = (nodes[:, 1] - ey) % ny
        x = (nodes[:, 2] - ex) % nx
        up = fbar[:, z, y, x]
        out[j] = collide(lat, m, S, up)[j]
    return out
