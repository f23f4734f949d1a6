"""Pins for the FP64 oracle: what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Eqs. Md2q9, meqd2q9, meqd2q9-HL, Md2q9-1..3, meqd2q9-1, 5-9,
5-10, 5-8-1), exact textbook special cases (standard D2Q9/D3Q19/D3Q27 weights,
BGK and Lallemand-Luo MRT steps), invariants (Eqs. 3-3-1..3-3-11, 3-5, 3-9,
4-18-1) and closed-form flow solutions (Taylor-Green, shear and sound waves,
Poiseuille, advected Gaussian hill, Cole-Hopf Burgers).
"""
import numpy as np
import pytest

import oracle.rmrt as R
import workloads as W

RNG = np.random.default_rng(1234)


def rand_lattice(name, rng):
    d = 2 if name == "D2Q9" else 3
    dx = rng.uniform(0.5, 1.5, size=3)
    c = dx[:d]
    cs2 = float(np.min(c * c)) / 3.0 * rng.uniform(0.6, 1.0)
    return R.make_lattice(name, tuple(dx), 1.0, cs2)


# ---------------------------------------------------------------- lattices
@pytest.mark.parametrize("name,expect", [
    ("D2Q9", {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}),
    ("D3Q19", {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}),
    ("D3Q27", {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}),
])
def test_standard_weights(name, expect):
    """On the standard lattice with c_s^2 = c^2/3 the weights are the classic
    ones (Sec. V: the popular models are the special case)."""
    lat = R.make_lattice(name, (1.0, 1.0, 1.0), 1.0, 1.0 / 3.0)
    speed2 = (lat.e ** 2).sum(axis=1)
    for s2, w in expect.items():
        np.testing.assert_allclose(lat.w[speed2 == s2], w, rtol=0, atol=5e-15)


@pytest.mark.parametrize("name", R.LATTICES)
def test_velocity_set_structure(name):
    e = R.velocity_indices(name)
    q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[name]
    assert e.shape[0] == q
    assert len({tuple(v) for v in e}) == q                       # distinct
    assert {tuple(-v) for v in e} == {tuple(v) for v in e}        # symmetric
    if name == "D3Q19":
        assert (e == 0).any(axis=1).all()                         # no corners
    if name != "D2Q9":
        assert (e[:19] == R.velocity_indices("D3Q19")).all()


@pytest.mark.parametrize("name", R.LATTICES)
def test_velocity_moments(name):
    """Eqs. (3-3-1), (3-3-2), (3-3-11): Delta0 = 1, odd moments 0,
    Delta2 = c_s^2 I, Delta4_aaaa = c_a^2 c_s^2, Delta4_aabb = c_s^4, else 0."""
    for _ in range(5):
        lat = rand_lattice(name, RNG)
        w, cv, cs2, d = lat.w, lat.cv, lat.cs2, lat.d
        assert (w >= 0).all()
        assert abs(w.sum() - 1) < 1e-15
        np.testing.assert_allclose(np.einsum("j,ja->a", w, cv), 0, atol=1e-15)
        D2 = np.einsum("j,ja,jb->ab", w, cv, cv)
        np.testing.assert_allclose(D2, cs2 * np.eye(d), atol=1e-15)
        np.testing.assert_allclose(np.einsum("j,ja,jb,jc->abc", w, cv, cv, cv), 0, atol=1e-15)
        D4 = np.einsum("j,ja,jb,jc,jd->abcd", w, cv, cv, cv, cv)
        for a in range(d):
            for b in range(d):
                for c in range(d):
                    for e in range(d):
                        idx = sorted([a, b, c, e])
                        if idx[0] == idx[3]:
                            want = lat.c[a] ** 2 * cs2
                        elif idx[0] == idx[1] and idx[2] == idx[3]:
                            want = cs2 * cs2
                        else:
                            want = 0.0
                        assert abs(D4[a, b, c, e] - want) < 1e-14


def test_no_rd3q15_rd3q13():
    """Eqs. (3-3-9), (3-3-10): dropping the edge (rD3Q15) or axis+corner
    (rD3Q13) velocities forces c_1 = c_2 = c_3.  On a rectangular lattice the
    rD3Q27 weight solution therefore keeps the edge and axis weights
    nonzero for every admissible omega_19."""
    lat = R.make_lattice("D3Q27", (1.0, 0.8, 0.6))
    c2 = lat.c ** 2
    cs2 = lat.cs2
    for w19 in np.linspace(0, cs2 / (8 * c2.max()), 5):
        w7 = cs2 ** 2 / (4 * c2[0] * c2[1]) - 2 * w19
        w11 = cs2 ** 2 / (4 * c2[0] * c2[2]) - 2 * w19
        w15 = cs2 ** 2 / (4 * c2[1] * c2[2]) - 2 * w19
        # rD3Q15 needs w7 = w11 = w15 = 0 at once: impossible with unequal c
        assert not (abs(w7) < 1e-14 and abs(w11) < 1e-14 and abs(w15) < 1e-14)


# ---------------------------------------------------------------- REDF
@pytest.mark.parametrize("name", R.LATTICES)
def test_redf_moments(name):
    """Eqs. (3-5), (3-9): the REDF moments up to third order."""
    lat = rand_lattice(name, RNG)
    d, n = lat.d, 7
    A = RNG.uniform(0.5, 1.5, n)
    B = RNG.normal(size=(n, d))
    Mt = RNG.normal(size=(n, d, d))
    Mt = Mt + Mt.transpose(0, 2, 1)
    g = R.geq(lat, A, B, Mt)
    cv, cs2 = lat.cv, lat.cs2
    np.testing.assert_allclose(g.sum(0), A, rtol=1e-13)
    np.testing.assert_allclose(np.einsum("ja,jn->na", cv, g), B, atol=1e-13)
    np.testing.assert_allclose(np.einsum("ja,jb,jn->nab", cv, cv, g),
                               A[:, None, None] * cs2 * np.eye(d) + Mt, atol=1e-13)
    third = np.einsum("ja,jb,jc,jn->nabc", cv, cv, cv, g)
    I = np.eye(d)
    want = cs2 * (np.einsum("ab,nc->nabc", I, B) + np.einsum("ac,nb->nabc", I, B)
                  + np.einsum("bc,na->nabc", I, B))
    for a in range(d):   # delta4_aaaa = c_s^2 (c_a^2 - 3 c_s^2), B~ = B / c_s^2
        want[:, a, a, a] += cs2 * (lat.c[a] ** 2 - 3 * cs2) * B[:, a] / cs2
    np.testing.assert_allclose(third, want, atol=1e-12)


# ---------------------------------------------------------------- rD2Q9 printed forms
MTILDE_D2Q9 = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 1, 0, 1, 0, 1, 1, 1, 1],
    [0, 0, 1, 0, 1, 1, 1, 1, 1],
    [0, 0, 0, 0, 0, 1, -1, 1, -1],
    [0, 0, 0, 0, 0, 1, -1, -1, 1],
    [0, 0, 0, 0, 0, 1, 1, -1, -1],
    [0, 0, 0, 0, 0, 1, 1, 1, 1]], dtype=float)


def test_d2q9_M_equals_D_Mtilde():
    """Eq. (Md2q9): M = D M~ with the printed integer M~ and
    D = diag(1, c1, c2, c1^2, c2^2, c1c2, c1c2^2, c1^2c2, c1^2c2^2)."""
    lat = R.make_lattice("D2Q9", (1.3, 0.7))
    c1, c2 = lat.c
    D = np.diag([1, c1, c2, c1 ** 2, c2 ** 2, c1 * c2, c1 * c2 ** 2, c1 ** 2 * c2, c1 ** 2 * c2 ** 2])
    np.testing.assert_allclose(R.moment_matrix(lat), D @ MTILDE_D2Q9, rtol=1e-15)


def test_d2q9_meq_printed():
    """Eqs. (meqd2q9) and (meqd2q9-HL): M f^eq in closed form."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    cs2 = lat.cs2
    rho = np.array([1.02, 0.97])
    u = np.array([[0.03, -0.02], [-0.05, 0.01]])
    M = R.moment_matrix(lat)
    S = np.eye(9)
    feq, _, _ = R.equilibrium_and_sources(lat, R.Model(R.NSE), S, rho, u)
    ux, uy = u[:, 0], u[:, 1]
    want = rho * np.array([np.ones(2), ux, uy, cs2 + ux ** 2, cs2 + uy ** 2, ux * uy,
                           cs2 * ux, cs2 * uy, cs2 * (ux ** 2 + uy ** 2 + cs2)])
    np.testing.assert_allclose(M @ feq, want, atol=1e-15)
    r0 = 1.0
    feq, _, _ = R.equilibrium_and_sources(lat, R.Model(R.NSE_HELUO, rho0=r0), S, rho, u)
    want = np.array([rho, r0 * ux, r0 * uy, cs2 * rho + r0 * ux ** 2, cs2 * rho + r0 * uy ** 2,
                     r0 * ux * uy, cs2 * r0 * ux, cs2 * r0 * uy,
                     cs2 * (r0 * (ux ** 2 + uy ** 2) + cs2 * rho)])
    np.testing.assert_allclose(M @ feq, want, atol=1e-15)


def test_bhll_relation():
    """Eqs. (Md2q9-1..3), (meqd2q9-1), (5-9), (5-10): the Bouzidi et al.
    orthogonal matrix is N_BHLL M_a, and N_BHLL M f^eq is the printed
    equilibrium with C_1..C_3."""
    for a in (0.5, 0.8, 1.0, 1.7):
        lat = R.make_lattice("D2Q9", (1.0, a), 1.0, 0.9 * min(1.0, a * a) / 3.0)
        r1, r2, r3, r4, r5, r6 = 1 + a * a, 1 - 2 * a * a, -2 + a * a, -1 + a * a, 2 + a * a, -1 - 2 * a * a
        Mb = np.array([
            [1, 1, 1, 1, 1, 1, 1, 1, 1],
            [0, 1, 0, -1, 0, 1, -1, -1, 1],
            [0, 0, a, 0, -a, a, a, -a, -a],
            [-2 * r1, r2, r3, r2, r3, r1, r1, r1, r1],
            [-2 * r4, r5, r6, r5, r6, r4, r4, r4, r4],
            [0, 0, 0, 0, 0, a, -a, a, -a],
            [0, -2, 0, 2, 0, 1, -1, -1, 1],
            [0, 0, -2 * a, 0, 2 * a, a, a, -a, -a],
            [4, -2, -2, -2, -2, 1, 1, 1, 1]], dtype=float)
        a2 = a * a
        N = np.zeros((9, 9))
        N[0, 0] = N[1, 1] = N[2, 2] = N[5, 5] = 1
        N[3, [0, 3, 4]] = [-2 * a2 - 2, 3, 3]
        N[4, [0, 3, 4]] = [-2 * a2 + 2, 3 * a2, -3 / a2]
        N[6, [1, 6]] = [-2, 3 / a2]
        N[7, [2, 7]] = [-2, 3]
        N[8, [0, 3, 4, 8]] = [4, -6, -6 / a2, 9 / a2]
        M = R.moment_matrix(lat)
        np.testing.assert_allclose(N @ M, Mb, atol=1e-13)
        rho = np.array([1.01])
        u = np.array([[0.04, -0.03]])
        feq, _, _ = R.equilibrium_and_sources(lat, R.Model(), np.eye(9), rho, u)
        cs2 = lat.cs2
        uu, vv = u[0, 0], u[0, 1]
        C1 = 2 * (3 * cs2 - 2 * a2) / a2
        C2 = 2 * (3 * cs2 - 2)
        C3 = (9 * cs2 ** 2 + 9 * cs2 * uu ** 2 + 9 * cs2 * vv ** 2 - 6 * cs2 - 6 * vv ** 2) / a2 \
            - (6 * uu ** 2 + 6 * cs2 - 4)
        e_eq = 3 * (uu ** 2 + vv ** 2) + 2 * (3 * cs2 - r1)
        pxx = r4 * (3 * r1 * cs2 - 2 * a2) / a2 + 3 * (a2 * uu ** 2 - vv ** 2 / a2)
        want = rho[0] * np.array([1, uu, vv, e_eq, pxx, uu * vv, C1 * uu / 2, C2 * vv / 2, C3])
        np.testing.assert_allclose((Mb @ feq)[:, 0], want, atol=1e-13)
        assert abs(C1 - (C2 + 4 * (1 - a2)) / a2) < 1e-13


def test_sherman_morrison_block():
    """Eq. (5-8-1): the numerically inverted S_2^(1) (Eq. 4-27-1) equals
    A - A abar b^T A / (1 + b^T A abar), A = diag(s_s), abar = a/d."""
    for name in R.LATTICES:
        lat = rand_lattice(name, RNG)
        r = R.rates_from_viscosity(lat, 0.013, 0.07, 1.1)
        c2 = lat.c ** 2 - lat.cs2
        a = (1 / r.s_bulk - 1 / r.s_shear) * c2
        b = 1 / c2
        A = np.diag(r.s_shear)
        ab = a / lat.d
        sm = A - (A @ np.outer(ab, b) @ A) / (1 + b @ A @ ab)
        np.testing.assert_allclose(R.s2_diag_block(lat, r), sm, rtol=1e-13)


def test_viscosity_relations():
    """Eq. (4-31) inverted: the rates reproduce nu and nu_b."""
    lat = R.make_lattice("D3Q19", (1.0, 0.8, 0.5))
    nu, nub = 0.011, 0.05
    r = R.rates_from_viscosity(lat, nu, nub, 1.1)
    cs2, c2, d = lat.cs2, lat.c ** 2, lat.d
    np.testing.assert_allclose((1 / r.s_off[0, 1] - 0.5) * cs2, nu, rtol=1e-14)
    np.testing.assert_allclose(0.5 * (1 / r.s_shear - 0.5) * (c2 - cs2), nu, rtol=1e-14)
    np.testing.assert_allclose((1 / d) * (1 / r.s_bulk - 0.5) * (c2 - cs2), nub, rtol=1e-14)


# ---------------------------------------------------------------- standard reductions
def bgk_feq_standard(e, w, rho, u):
    """Textbook second-order equilibrium with c_s^2 = 1/3 on a unit lattice."""
    cu = e @ u.T
    usq = (u * u).sum(axis=1)
    return w[:, None] * rho[None, :] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq[None, :])


@pytest.mark.parametrize("name", R.LATTICES)
@pytest.mark.parametrize("basis", [R.RAW, R.CENTRAL])
def test_reduces_to_bgk(name, basis):
    """Standard lattice, c_s^2 = 1/3, every rate s: the collision is the
    textbook BGK step f* = f - s (f - f^eq) (Sec. V: the popular models are
    special cases; with S = s I the basis does not matter, Eq. 5-1-2)."""
    lat = R.make_lattice(name, (1, 1, 1), 1.0, 1.0 / 3.0)
    s = 1.37
    r = R.Rates(s, np.full(lat.d, s), np.full(lat.d, s), np.full(lat.d, s),
                np.full((lat.d, lat.d), s), s)
    S = R.relaxation_matrix(lat, r)
    np.testing.assert_allclose(S, s * np.eye(lat.q), atol=1e-14)
    f = W.random_populations(lat.q, (40,), seed=3)
    rho = f.sum(0)
    u = (lat.cv.T @ f / rho).T
    want = f - s * (f - bgk_feq_standard(lat.e.astype(float), lat.w, rho, u))
    got = R.collide(lat, R.Model(R.NSE, basis=basis), S, f)
    np.testing.assert_allclose(got, want, atol=2e-15)


def test_reduces_to_lallemand_luo_mrt():
    """Standard D2Q9 with c_s^2 = 1/3: with S = N^-1 Sbar N (Eq. 5-1-2), N
    taking raw moments to the Lallemand-Luo orthogonal moments, one oracle
    collision equals the textbook Lallemand-Luo MRT collision."""
    lat = R.make_lattice("D2Q9", (1, 1), 1.0, 1.0 / 3.0)
    MLL = np.array([
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=float)
    s_e, s_eps, s_q, s_nu = 1.2, 1.4, 1.15, 1.8
    Sbar = np.diag([0.9, s_e, s_eps, 0.9, s_q, 0.9, s_q, s_nu, s_nu])
    f = W.random_populations(9, (50,), seed=5)
    rho = f.sum(0)
    jx, jy = MLL[3] @ f, MLL[5] @ f
    u2 = (jx ** 2 + jy ** 2) / rho ** 2
    meq = np.array([rho, -2 * rho + 3 * rho * u2, rho - 3 * rho * u2, jx, -jx, jy, -jy,
                    (jx ** 2 - jy ** 2) / rho, jx * jy / rho])
    want = f - np.linalg.solve(MLL, Sbar @ (MLL @ f - meq))
    N = MLL @ np.linalg.inv(R.moment_matrix(lat))
    S = np.linalg.solve(N, Sbar @ N)
    got = R.collide(lat, R.Model(), S, f)
    np.testing.assert_allclose(got, want, atol=2e-15)


def test_forced_step_reduces_to_guo_forced_mrt():
    """Standard D2Q9 (c_s^2 = 1/3), body force, no source: through third
    order every raw moment after one oracle collision equals the textbook
    Lallemand-Luo MRT step with Guo's forcing (Guo, Zheng & Shi, Phys. Rev.
    E 65, 046308 (2002), in moment space: m* = m - Sbar (m - m^eq) +
    dt (I - Sbar/2) M F~, F~_i = w_i [(e_i - u)/c_s^2 + (e_i.u) e_i/c_s^4].F,
    u = (j + dt F/2)/rho).  The second-order moments carry the force only
    through the auxiliary distribution G (M_2G of Eq. M2GComput a), so a
    dropped G, a wrong (I - S_2/2) factor or a transposed u F term fails
    here.  Only the fourth-order moment xxyy, which does not enter the NSE,
    is built differently by the two schemes."""
    lat = R.make_lattice("D2Q9", (1, 1), 1.0, 1.0 / 3.0)
    MLL = np.array([
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=float)
    Sbar = np.diag([0.9, 1.2, 1.4, 0.9, 1.15, 0.9, 1.15, 1.8, 1.8])
    f = W.random_populations(9, (50,), seed=6)
    F = np.array([2e-3, -1.5e-3])
    cs2 = 1.0 / 3.0
    ex, ey = lat.e[:, 0].astype(float), lat.e[:, 1].astype(float)
    rho = f.sum(0)
    ux = (ex @ f + 0.5 * F[0]) / rho
    uy = (ey @ f + 0.5 * F[1]) / rho
    u2 = ux ** 2 + uy ** 2
    meq = np.array([rho, -2 * rho + 3 * rho * u2, rho - 3 * rho * u2, rho * ux, -rho * ux, rho * uy, -rho * uy,
                    rho * (ux ** 2 - uy ** 2), rho * ux * uy])
    eu = ex[:, None] * ux[None] + ey[:, None] * uy[None]
    eF = ex * F[0] + ey * F[1]
    uF = ux * F[0] + uy * F[1]
    Ft = lat.w[:, None] * ((eF[:, None] - uF[None]) / cs2 + eu * eF[:, None] / cs2 ** 2)
    mll = MLL @ f
    want = np.linalg.solve(MLL, mll - Sbar @ (mll - meq) + (np.eye(9) - 0.5 * Sbar) @ (MLL @ Ft))
    N = MLL @ np.linalg.inv(R.moment_matrix(lat))
    S = np.linalg.solve(N, Sbar @ N)
    got = R.collide(lat, R.Model(force=(F[0], F[1], 0.0)), S, f)
    M = R.moment_matrix(lat)
    low = [k for k, a in enumerate(R.monomials("D2Q9")) if sum(a) <= 3]
    np.testing.assert_allclose((M @ got)[low], (M @ want)[low], atol=2e-15)
    # what G adds to the second-order moments, u F + F u, is ten orders of
    # magnitude above the tolerance (the pin has teeth)
    assert min(np.abs(2 * ux * F[0]).max(), np.abs(2 * uy * F[1]).max(),
               np.abs(ux * F[1] + uy * F[0]).max()) > 1e-5


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("name", R.LATTICES)
@pytest.mark.parametrize("basis", [R.RAW, R.CENTRAL, R.HERMITE, R.CENTRAL_HERMITE])
def test_collision_invariants(name, basis):
    """Eq. (4-18-1): mass and momentum are collision invariants; with
    forcing the increments are exactly dt Sbar and dt Fbar (Eq. 2-4-2)."""
    lat = rand_lattice(name, RNG)
    r = R.rates_from_viscosity(lat, 0.02, 0.05, 1.1)
    S = R.relaxation_matrix(lat, r)
    f = W.random_populations(lat.q, (30,), seed=7)
    for force, src in [((0, 0, 0), 0.0), ((1e-4, -2e-4, 3e-4), 2e-5)]:
        m = R.Model(R.NSE, basis=basis, force=force, source=src)
        fs = R.collide(lat, m, S, f)
        np.testing.assert_allclose(fs.sum(0), f.sum(0) + src, rtol=0, atol=5e-15)
        np.testing.assert_allclose(lat.cv.T @ fs, lat.cv.T @ f + np.array(force[:lat.d])[:, None],
                                   rtol=0, atol=5e-15)
    for kind in (R.NCDE_LINEAR, R.NCDE_QUAD):
        m = R.Model(kind, basis=basis, adv=(0.05, 0.02, -0.01), source=3e-5)
        S1 = R.relaxation_matrix(lat, R.Rates(1.0, np.full(lat.d, 1.6), np.full(lat.d, 1.1),
                                              np.full(lat.d, 1.1), np.full((lat.d, lat.d), 1.1), 1.1))
        fs = R.collide(lat, m, S1, f)
        np.testing.assert_allclose(fs.sum(0), f.sum(0) + 3e-5, rtol=0, atol=5e-15)


def test_s0_s1_irrelevant_for_nse():
    """The unforced NSE result does not depend on s_0 and S_1 (their moments
    are conserved, Eq. 4-18-1)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    f = W.random_populations(9, (20,), seed=9)
    outs = []
    for s01 in (0.7, 1.3, 1.9):
        r = R.rates_from_viscosity(lat, 0.02, 0.04, 1.1, s0=s01, s1=s01)
        outs.append(R.collide(lat, R.Model(), R.relaxation_matrix(lat, r), f))
    np.testing.assert_allclose(outs[0], outs[1], atol=1e-16)
    np.testing.assert_allclose(outs[0], outs[2], atol=1e-16)


@pytest.mark.parametrize("name", R.LATTICES)
def test_central_basis_structure(name):
    """Eqs. (5-1-1), (5-1-2): Mbar(u) = N(u) M with N unit lower-triangular
    in moment order, so S = N^-1 Sbar N is block-lower-triangular with the
    diagonal blocks of Sbar.  The central moments of f^eq have zero first
    order and c_s^2 rho I second order for any u."""
    lat = rand_lattice(name, RNG)
    u = np.array([[0.04, -0.03, 0.02][: lat.d]])
    M = R.moment_matrix(lat)
    N = R.central_moment_matrices(lat, u)[0] @ np.linalg.inv(M)
    order = R.moment_order(lat.name)
    for k in range(lat.q):
        for l in range(lat.q):
            if order[l] > order[k] or (order[l] == order[k] and l != k):
                assert abs(N[k, l]) < 1e-12
        assert abs(N[k, k] - 1) < 1e-12
    r = R.rates_from_viscosity(lat, 0.02, 0.04, 1.1)
    Sbar = R.relaxation_matrix(lat, r)
    S = np.linalg.solve(N, Sbar @ N)
    for k in range(lat.q):
        for l in range(lat.q):
            if order[l] > order[k]:
                assert abs(S[k, l]) < 1e-12
            if order[l] == order[k]:
                assert abs(S[k, l] - Sbar[k, l]) < 1e-12
    rho = np.array([1.03])
    feq, _, _ = R.equilibrium_and_sources(lat, R.Model(), Sbar, rho, u)
    cc = lat.cv - u[0][None, :]
    np.testing.assert_allclose(cc.T @ feq[:, 0], 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("ja,jb,j->ab", cc, cc, feq[:, 0]),
                               lat.cs2 * rho[0] * np.eye(lat.d), atol=1e-15)


def test_central_equals_raw_at_rest_and_unit_rates():
    """At u = 0, N = I so central and raw coincide; with every rate 1 both
    give f^eq."""
    lat = R.make_lattice("D3Q27", (1.0, 0.9, 0.6))
    f = W.random_populations(lat.q, (12,), seed=11)
    # remove the momentum so that u = 0 at every node
    rho = f.sum(0)
    u = (lat.cv.T @ f) / rho
    f0 = f - R.geq(lat, np.zeros(12), (rho * u).T, np.zeros((12, 3, 3)))
    r = R.rates_from_viscosity(lat, 0.02, 0.04, 1.1)
    S = R.relaxation_matrix(lat, r)
    a = R.collide(lat, R.Model(basis=R.RAW), S, f0)
    b = R.collide(lat, R.Model(basis=R.CENTRAL), S, f0)
    np.testing.assert_allclose(a, b, atol=1e-15)
    one = R.relaxation_matrix(lat, R.Rates(1, np.ones(3), np.ones(3), np.ones(3), np.ones((3, 3)), 1))
    a = R.collide(lat, R.Model(basis=R.RAW), one, f)
    b = R.collide(lat, R.Model(basis=R.CENTRAL), one, f)
    rho, u = R.macroscopic(lat, R.Model(), f)
    feq, _, _ = R.equilibrium_and_sources(lat, R.Model(), one, rho, u)
    np.testing.assert_allclose(a, feq, atol=1e-15)
    np.testing.assert_allclose(b, feq, atol=1e-15)


@pytest.mark.parametrize("name,dx", [("D2Q9", (1.0, 0.6)), ("D3Q27", (1.0, 0.7, 0.5))])
def test_hermite_basis_orthogonal(name, dx):
    """On the tensor-product lattices the Hermite polynomials P_0 = 1,
    P_1 = xi, P_2 = xi^2 - c_s^2 of each axis are orthogonal under the 1-D
    weights (1 - c_s^2/c^2, c_s^2/(2c^2), c_s^2/(2c^2)), so the Hermite
    basis rows are orthogonal under omega_j: sum_j omega_j H_k H_l = 0,
    k != l, with H_k H_k summing to the product over axes of 1, c_s^2 and
    c_s^2 (c_a^2 - c_s^2) (2 c_s^4 on the standard lattice)."""
    lat = R.make_lattice(name, dx)
    H = R.central_moment_matrices(lat, np.zeros((1, lat.d)), hermite=True)[0]
    G = H @ np.diag(lat.w) @ H.T
    mons = R.monomials(lat.name)
    want = np.array([np.prod([(1.0, lat.cs2, lat.cs2 * (lat.c[al] ** 2 - lat.cs2))[a[al]] for al in range(lat.d)])
                     for a in mons])
    np.testing.assert_allclose(G, np.diag(want), atol=1e-14)


@pytest.mark.parametrize("name", R.LATTICES)
@pytest.mark.parametrize("basis", [R.HERMITE, R.CENTRAL_HERMITE])
def test_hermite_bases_structure_and_limits(name, basis):
    """Eq. (5-1-1) for the Hermite bases: Mbar = N M with N unit
    lower-triangular in moment order; with every non-conserved rate equal
    the collision is BGK and independent of the basis; the Hermite basis at
    u = 0 equals the central-Hermite basis."""
    lat = rand_lattice(name, RNG)
    u = np.array([[0.04, -0.03, 0.02][: lat.d]])
    M = R.moment_matrix(lat)
    Mb = R.central_moment_matrices(lat, u if basis == R.CENTRAL_HERMITE else 0 * u, hermite=True)[0]
    N = Mb @ np.linalg.inv(M)
    order = R.moment_order(lat.name)
    for k in range(lat.q):
        for l in range(lat.q):
            if order[l] > order[k] or (order[l] == order[k] and l != k):
                assert abs(N[k, l]) < 1e-12
        assert abs(N[k, k] - 1) < 1e-12
    f = W.random_populations(lat.q, (10,), seed=12)
    s = 1.3
    bgk = R.relaxation_matrix(lat, R.Rates(s, np.full(lat.d, s), np.full(lat.d, s), np.full(lat.d, s),
                                           np.full((lat.d, lat.d), s), s))
    a = R.collide(lat, R.Model(basis=R.RAW), bgk, f)
    b = R.collide(lat, R.Model(basis=basis), bgk, f)
    np.testing.assert_allclose(a, b, atol=1e-14)
    rho = f.sum(0)
    mom = (lat.cv.T @ f) / rho
    f0 = f - R.geq(lat, np.zeros(10), (rho * mom).T, np.zeros((10, lat.d, lat.d)))
    r = R.rates_from_viscosity(lat, 0.02, 0.04, 1.1)
    S = R.relaxation_matrix(lat, r)
    np.testing.assert_allclose(R.collide(lat, R.Model(basis=R.HERMITE), S, f0),
                               R.collide(lat, R.Model(basis=R.CENTRAL_HERMITE), S, f0), atol=1e-15)


def test_hermite_basis_differs_from_raw_only_through_high_orders():
    """Hermite moments of order <= 2 of a non-equilibrium part with no mass
    or momentum are its raw moments, so the viscosity is unchanged: with
    s_free equal to the second-order rates where they coincide (standard
    lattice, nu_bulk chosen so all second-order rates agree), Hermite and
    raw collisions coincide; with a different s_free they differ."""
    lat = R.make_lattice("D2Q9", (1.0, 1.0), cs2=1.0 / 3.0)
    f = W.random_populations(9, (10,), seed=13)
    s_nu = 1.0 / (0.02 / (lat.cs2) + 0.5)
    nu_b = (1.0 / s_nu - 0.5) * (1.0 - lat.cs2) / 2.0    # makes s_b = s_s = s_nu on the standard lattice
    for s_free, same in ((s_nu, True), (1.1, False)):
        r = R.rates_from_viscosity(lat, 0.02, nu_b, s_free)
        S = R.relaxation_matrix(lat, r)
        a = R.collide(lat, R.Model(basis=R.RAW), S, f)
        b = R.collide(lat, R.Model(basis=R.HERMITE), S, f)
        assert (np.abs(a - b).max() < 1e-14) == same


def test_streaming_direction():
    """Eq. (2-2b): a population at x moves to x + c_j dt (one node along e_j)."""
    for name in R.LATTICES:
        lat = R.make_lattice(name, (1.0, 0.7, 0.5))
        shp = (5, 6, 7) if lat.d == 3 else (1, 6, 7)
        for j in range(lat.q):
            f = np.zeros((lat.q,) + shp)
            z, y, x = (2 if lat.d == 3 else 0), 3, 4
            f[j, z, y, x] = 1.0
            g = R.stream(lat, f)
            ez = int(lat.e[j, 2]) if lat.d == 3 else 0
            assert g[j, (z + ez) % shp[0], (y + lat.e[j, 1]) % shp[1], (x + lat.e[j, 0]) % shp[2]] == 1.0
            assert g.sum() == 1.0


def test_f_form_equivalence():
    """Eq. (2-1) with the implicit scheme for D_j F_j and Eq. (2-3) in the
    transformed variable fbar = f - dt F/2 give the same f (Sec. II)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    r = R.rates_from_viscosity(lat, 0.03, 0.05, 1.2)
    S = R.relaxation_matrix(lat, r)
    shp = (1, 8, 10)
    n = int(np.prod(shp))
    rng = np.random.default_rng(2)
    force = 1e-4 * rng.normal(size=(2, n))
    src = 1e-5 * rng.normal(size=n)
    m = R.Model(R.NSE, force=force, source=src)
    fbar = W.random_populations(9, shp, seed=4)
    # F_j does not depend on u (Eq. NSEFeq), so it is known at t + dt
    Fj = R.geq(lat, src, force.T, -lat.cs2 * src[:, None, None] * np.eye(2)[None])
    f = fbar + 0.5 * Fj.reshape(fbar.shape)
    M = R.moment_matrix(lat)
    Lam = np.linalg.solve(M, S @ M)
    for _ in range(3):
        fb_next = R.step(lat, m, S, fbar, 1)
        # f-form: f(x+c, t+1) = f - Lam f^ne + G + F + (F(x+c) - F(x))/2
        fl = f.reshape(9, -1)
        rho = fl.sum(0)
        u = ((lat.cv.T @ fl) / rho).T
        feq, G, F = R.equilibrium_and_sources(lat, m, S, rho, u)
        post = fl - Lam @ (fl - feq) + G + F - 0.5 * F
        f = R.stream(lat, post.reshape(fbar.shape)) + 0.5 * F.reshape(fbar.shape)
        fbar = fb_next
        np.testing.assert_allclose(fbar + 0.5 * Fj.reshape(fbar.shape), f, atol=1e-15)


# ---------------------------------------------------------------- flows
def mode_amp(field, basis):
    return (field * basis).sum() / (basis * basis).sum()


def test_taylor_green_decay_rectangular():
    """rD2Q9, 64 x 32 with dx = 1, dy = 0.5, c_s^2 = 1/12, nu = 0.01, bulk
    rate 1.2 on x, free rates 1.1, 2000 steps: the kinetic energy decays as
    exp(-2 nu k^2 t), k^2 = kx^2 + ky^2 (rate within 1%).  Eq. (4-31)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    nu = 0.01
    r = R.rates_from_viscosity(lat, nu, R.nu_bulk_from_rate(lat, 1.2), 1.1)
    S = R.relaxation_matrix(lat, r)
    m = R.Model()
    rho, u = W.taylor_green_2d(64, 32, 1.0, 0.5, 0.01, 1.0, lat.cs2)
    f = R.init_equilibrium(lat, m, S, rho, u)
    f = R.step(lat, m, S, f, 200)
    E0 = (R.fields(lat, m, f)[1] ** 2).sum()
    f = R.step(lat, m, S, f, 1800)
    E1 = (R.fields(lat, m, f)[1] ** 2).sum()
    k2 = (2 * np.pi / 64) ** 2 + (2 * np.pi / 16) ** 2
    rate = -np.log(E1 / E0) / 1800
    assert abs(rate / (2 * nu * k2) - 1) < 0.01


def shear_wave_rate(lat, S, nx, ny, kvec_idx, steps=600):
    """Decay rate of a divergence-free plane shear wave."""
    kx = 2 * np.pi * kvec_idx[0] / (nx * lat.dx[0])
    ky = 2 * np.pi * kvec_idx[1] / (ny * lat.dx[1])
    X, Y, _ = W.grid((1, ny, nx), lat.dx)
    kk = np.hypot(kx, ky)
    ph = kx * X + ky * Y
    amp = 1e-3
    u = np.stack([-ky / kk * amp * np.sin(ph), kx / kk * amp * np.sin(ph)])
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones((1, ny, nx)), u)
    basis = np.sin(ph)
    pol = (-ky / kk, kx / kk)

    def amp_of(f):
        uu = R.fields(lat, m, f)[1]
        return mode_amp(pol[0] * uu[0] + pol[1] * uu[1], basis)
    f = R.step(lat, m, S, f, 100)
    a0 = amp_of(f)
    f = R.step(lat, m, S, f, steps)
    a1 = amp_of(f)
    return -np.log(a1 / a0) / steps / (kk * kk)


def test_shear_wave_isotropy():
    """On a rectangular lattice (dx = 1, dy = 0.6) shear waves along x, along
    y and along the physical diagonal decay with the same nu (Eqs. 4-27,
    4-31); the diagonal one involves the dense S_2 block."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    nu = 0.02
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, 0.03, 1.1))
    for nx, ny, kk in [(32, 2, (1, 0)), (2, 48, (0, 1)), (30, 50, (1, 1))]:
        assert abs(shear_wave_rate(lat, S, nx, ny, kk) / nu - 1) < 0.01


def test_shear_wave_detects_single_rate_s2():
    """Planted mistake: relaxing the normal stresses at the off-diagonal rate
    (a single viscous rate, Remark II of Sec. IV) makes the diagonal shear
    wave decay at the wrong rate, so the isotropy pin does see the S_2
    block."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    nu = 0.02
    r = R.rates_from_viscosity(lat, nu, 0.03, 1.1)
    r.s_shear = np.full(2, r.s_off[0, 1])
    r.s_bulk = np.full(2, r.s_off[0, 1])
    S = R.relaxation_matrix(lat, r)
    assert abs(shear_wave_rate(lat, S, 30, 50, (1, 1)) / nu - 1) > 0.05


def test_sound_wave_speed_and_bulk_attenuation():
    """A plane sound wave along x propagates at c_s and its energy decays at
    k^2 [2 nu (1 - 1/d) + nu_b] (Eqs. 4-24-3, 4-31b; linear acoustics)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    nu, nub = 0.01, 0.04
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, nub, 1.1))
    nx, ny = 64, 2
    k = 2 * np.pi / (nx * lat.dx[0])
    X, _, _ = W.grid((1, ny, nx), lat.dx)
    amp = 1e-4
    u = np.stack([amp * np.sin(k * X), np.zeros_like(X)])
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones((1, ny, nx)), u)
    cs = np.sqrt(lat.cs2)
    period = 2 * np.pi / (cs * k)
    nsteps = int(round(4 * period))
    E, A = [], []
    for t in range(nsteps + 1):
        rho, uu = R.fields(lat, m, f)
        a = mode_amp(uu[0], np.sin(k * X))
        b = mode_amp(rho - 1, np.cos(k * X))
        E.append(a * a + lat.cs2 * b * b)
        A.append(a)
        f = R.step(lat, m, S, f, 1)
    t = np.arange(nsteps + 1)
    slope = np.polyfit(t, np.log(E), 1)[0]
    nuL = 2 * nu * (1 - 1 / 2) + nub
    assert abs(-slope / (nuL * k * k) - 1) < 0.03
    A = np.array(A)
    zc = np.where(np.diff(np.sign(A)) != 0)[0]
    half = np.mean(np.diff(zc))
    assert abs(2 * half / period - 1) < 0.02


# ---------------------------------------------------------------- 3-D S_2 block and bulk viscosity
SPACING_3D = (1.0, 0.8, 0.5)


def shear_wave_rate_3d(lat, S, shape, kidx, pol, steps=300):
    """Decay rate / k^2 of a plane shear wave u = pol A sin(k . x) on a
    periodic (nx, ny, nz) box, k_a = 2 pi kidx_a / (n_a dx_a); pol is
    perpendicular to k (a divergence-free wave)."""
    nx, ny, nz = shape
    X, Y, Z = W.grid((nz, ny, nx), lat.dx)
    k = np.array([2 * np.pi * kidx[a] / (shape[a] * lat.dx[a]) for a in range(3)])
    pol = np.asarray(pol, dtype=np.float64)
    assert abs(pol @ k) < 1e-12
    ph = k[0] * X + k[1] * Y + k[2] * Z
    amp = 1e-3
    u = np.stack([pol[a] * amp * np.sin(ph) for a in range(3)])
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones((nz, ny, nx)), u)
    basis = np.sin(ph)

    def amp_of(f):
        uu = R.fields(lat, m, f)[1]
        return mode_amp(sum(pol[a] * uu[a] for a in range(3)), basis)
    f = R.step(lat, m, S, f, 100)
    a0 = amp_of(f)
    f = R.step(lat, m, S, f, steps)
    a1 = amp_of(f)
    return -np.log(a1 / a0) / steps / (k @ k)


def xz_diagonal_wave():
    """A shear wave along the physical diagonal of the xz plane (24 nodes at
    dx = 1 and 48 at dz = 0.5 per wavelength; the second-order truncation
    error of the decay rate is then about 0.6%), polarised in that plane:
    its stress has normal components on x and z, so it runs through the
    dense S_2 block."""
    k = np.array([2 * np.pi / 24, 0.0, 2 * np.pi / 24])
    return (24, 2, 48), (1, 0, 1), (-k[2] / np.hypot(k[0], k[2]), 0.0, k[0] / np.hypot(k[0], k[2]))


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
def test_shear_wave_isotropy_3d(name):
    """rD3Q19 and rD3Q27 with dx = 1, dy = 0.8, dz = 0.5: shear waves along z
    (x-polarised), along the xz diagonal (polarised in the xz plane and
    along y) all decay at the one nu of Eq. (4-31) within 1%."""
    lat = R.make_lattice(name, SPACING_3D)
    nu = 0.01
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, 0.03, 1.1))
    shape, kidx, pol = xz_diagonal_wave()
    for shp, kk, pp in [((2, 2, 48), (0, 0, 1), (1.0, 0.0, 0.0)), (shape, kidx, pol), (shape, kidx, (0.0, 1.0, 0.0))]:
        assert abs(shear_wave_rate_3d(lat, S, shp, kk, pp) / nu - 1) < 0.01, (shp, pp)


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
def test_shear_wave_3d_detects_single_rate_s2(name):
    """Planted mistake: normal stresses relaxed at the off-diagonal rate (one
    viscous rate for every second moment) leave the z-axis wave untouched
    but make the xz-diagonal wave decay at a wrong rate."""
    lat = R.make_lattice(name, SPACING_3D)
    nu = 0.01
    r = R.rates_from_viscosity(lat, nu, 0.03, 1.1)
    r.s_shear = np.full(3, r.s_off[0, 1])
    r.s_bulk = np.full(3, r.s_off[0, 1])
    S = R.relaxation_matrix(lat, r)
    shape, kidx, pol = xz_diagonal_wave()
    assert abs(shear_wave_rate_3d(lat, S, shape, kidx, pol) / nu - 1) > 0.2


def sound_wave_3d(lat, S, axis, n=64, periods=4):
    """Energy decay rate / k^2 and period / (2 pi / (c_s k)) of a plane sound
    wave along one axis of a 3-D box (two nodes on the other axes)."""
    shape = [2, 2, 2]
    shape[axis] = n
    nx, ny, nz = shape
    X = W.grid((nz, ny, nx), lat.dx)[axis]
    k = 2 * np.pi / (n * lat.dx[axis])
    amp = 1e-4
    u = np.zeros((3, nz, ny, nx))
    u[axis] = amp * np.sin(k * X)
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones((nz, ny, nx)), u)
    period = 2 * np.pi / (np.sqrt(lat.cs2) * k)
    nsteps = int(round(periods * period))
    E, A = [], []
    for _ in range(nsteps + 1):
        rho, uu = R.fields(lat, m, f)
        a = mode_amp(uu[axis], np.sin(k * X))
        b = mode_amp(rho - 1, np.cos(k * X))
        E.append(a * a + lat.cs2 * b * b)
        A.append(a)
        f = R.step(lat, m, S, f, 1)
    slope = np.polyfit(np.arange(nsteps + 1), np.log(E), 1)[0]
    A = np.array(A)
    zc = np.where(np.diff(np.sign(A)) != 0)[0]
    return -slope / (k * k), 2 * np.mean(np.diff(zc)) / period


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
def test_sound_wave_3d_bulk_attenuation(name):
    """Plane sound waves along x and along z (dz = 0.5) propagate at c_s and
    their energy decays at k^2 [2 nu (1 - 1/d) + nu_b] with d = 3 (Eqs.
    4-24-3, 4-31b): pins nu_b and the z-axis entries of the S_2 block."""
    lat = R.make_lattice(name, SPACING_3D)
    nu, nub = 0.01, 0.04
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, nub, 1.1))
    nuL = 2 * nu * (1 - 1 / 3) + nub
    for axis in (0, 2):
        g, per = sound_wave_3d(lat, S, axis)
        assert abs(g / nuL - 1) < 0.015, axis
        assert abs(per - 1) < 0.01, axis


def _s2_block_with(d_in_rank_one=None, z_axis_c2_from=None):
    """A copy of the oracle's S_2 block with one planted change: the rank-one
    term divided by `d_in_rank_one` instead of d, or a_z built with the
    (c^2 - c_s^2) of another axis."""
    def block(lat, r):
        c2 = lat.c * lat.c - lat.cs2
        a = (1.0 / r.s_bulk - 1.0 / r.s_shear) * c2
        if z_axis_c2_from is not None:
            a = a.copy()
            a[2] = (1.0 / r.s_bulk[2] - 1.0 / r.s_shear[2]) * c2[z_axis_c2_from]
        d = lat.d if d_in_rank_one is None else d_in_rank_one
        return np.linalg.inv(np.diag(1.0 / r.s_shear) + np.outer(a, 1.0 / c2) / d)
    return block


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27"])
def test_3d_pins_detect_planted_s2_mistakes(name, monkeypatch):
    """The 3-D pins see a wrong 1/d in Eq. (4-27-1) (the sound attenuation is
    30% off) and a z-axis a_z built with c_x (the z sound wave decays several
    times too fast and the xz-diagonal shear wave more than 2% off, beyond
    the 1% of the isotropy pin)."""
    lat = R.make_lattice(name, SPACING_3D)
    nu, nub = 0.01, 0.04
    nuL = 2 * nu * (1 - 1 / 3) + nub
    monkeypatch.setattr(R, "s2_diag_block", _s2_block_with(d_in_rank_one=2))
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, nub, 1.1))
    assert abs(sound_wave_3d(lat, S, 0)[0] / nuL - 1) > 0.2
    monkeypatch.setattr(R, "s2_diag_block", _s2_block_with(z_axis_c2_from=0))
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, nub, 1.1))
    assert abs(sound_wave_3d(lat, S, 2)[0] / nuL - 1) > 0.5
    shape, kidx, pol = xz_diagonal_wave()
    assert abs(shear_wave_rate_3d(lat, S, shape, kidx, pol) / nu - 1) > 0.015


def test_poiseuille_profile():
    """Force-driven channel between resting walls (y axis, half-way
    bounce-back): the steady profile is u = F/(2 rho nu) (y+dy/2)(H-y-dy/2)
    to within 1% on the rectangular lattice (forcing per Eq. 2-3)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    nu = 0.05
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, 0.05, 1.1))
    ny, nx = 24, 2
    H = ny * lat.dx[1]
    F = 1e-6
    m = R.Model(force=(F, 0.0))
    f = R.init_equilibrium(lat, m, S, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    f = R.step(lat, m, S, f, 4000, walls=(1,))
    ux = R.fields(lat, m, f)[1][0][0, :, 0]
    y = (np.arange(ny) + 0.5) * lat.dx[1]
    want = F / (2 * nu) * y * (H - y)
    assert np.max(np.abs(ux - want)) / want.max() < 0.01


def hill_error(n_scale, kind=R.NCDE_LINEAR, lattice="D2Q9"):
    """Relative L2 error of the advected-diffusing Gaussian hill at t = T."""
    nx, ny = 32 * n_scale, 40 * n_scale
    L = (32.0, 24.0)
    dx = (L[0] / nx, L[1] / ny)
    dt = 1.0 / (n_scale * n_scale)
    lat = R.make_lattice(lattice, dx, dt)
    D = 0.05
    tau = D / (lat.cs2 * dt) + 0.5
    s1 = 1 / tau
    rr = R.Rates(1.0, np.full(2, s1), np.full(2, 1.1), np.full(2, 1.1), np.full((2, 2), 1.1), 1.1)
    S = R.relaxation_matrix(lat, rr)
    adv = (0.05, 0.02)
    m = R.Model(kind, adv=adv)
    sig = 3.0
    phi0 = W.gaussian_hill((1, ny, nx), dx, sig, peak=1.0, adv=adv, diff=D, t=0.0)
    f = R.init_equilibrium(lat, m, S, phi0, np.zeros((2, 1, ny, nx)))
    T = 40.0
    f = R.step(lat, m, S, f, int(round(T / dt)))
    phi = R.fields(lat, m, f)[0]
    ref = W.gaussian_hill((1, ny, nx), dx, sig, peak=1.0, adv=adv, diff=D, t=T)
    return np.sqrt(((phi - ref) ** 2).sum() / (ref ** 2).sum())


def test_gaussian_hill_second_order():
    """Linear NCDE (B = u phi, D = phi I, Eqs. 4-10, 4-14): the advected,
    diffusing Gaussian hill matches its closed form, and the error falls
    at second order under diffusive refinement (dx/2, dt/4)."""
    e1, e2 = hill_error(1), hill_error(2)
    assert e1 < 1e-2
    assert np.log2(e1 / e2) > 1.8


def burgers_error(n_scale):
    nx, ny = 48 * n_scale, 2
    dx = (1.0 / n_scale, 0.6)
    dt = 1.0 / (n_scale * n_scale)
    lat = R.make_lattice("D2Q9", dx, dt, cs2=0.1 * n_scale * n_scale)
    D = 0.08
    tau = D / (lat.cs2 * dt) + 0.5
    rr = R.Rates(1.0, np.full(2, 1 / tau), np.full(2, 1.1), np.full(2, 1.1), np.full((2, 2), 1.1), 1.1)
    S = R.relaxation_matrix(lat, rr)
    U = 0.2
    m = R.Model(R.NCDE_QUAD, adv=(U, 0.0))
    phi0 = W.burgers_cole_hopf(nx, dx[0], U, D, 0.0)
    phi0 = np.broadcast_to(phi0[None, None, :], (1, ny, nx)).copy()
    f = R.init_equilibrium(lat, m, S, phi0, np.zeros((2, 1, ny, nx)))
    T = 150.0
    f = R.step(lat, m, S, f, int(round(T / dt)))
    phi = R.fields(lat, m, f)[0][0, 0]
    ref = W.burgers_cole_hopf(nx, dx[0], U, D, T)
    return np.sqrt(((phi - ref) ** 2).sum() / (ref ** 2).sum())


def test_burgers_cole_hopf_second_order():
    """Quadratic NCDE (B = u phi^2/2, C = u u phi^3/3, D = phi I) along x is
    viscous Burgers for w = U phi; the oracle follows the exact Cole-Hopf
    solution and converges at second order."""
    e1, e2 = burgers_error(1), burgers_error(2)
    assert e1 < 2e-2
    assert np.log2(e1 / e2) > 1.8


@pytest.mark.slow
def test_taylor_green_second_order():
    """The decayed Taylor-Green field converges at second order under
    diffusive refinement on the rectangular lattice."""
    errs = []
    for s in (1, 2):
        nx, ny = 16 * s, 16 * s
        dx = (1.0 / s, 0.5 / s)
        dt = 1.0 / (s * s)
        lat = R.make_lattice("D2Q9", dx, dt)
        nu = 0.02
        S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, 0.02, 1.1))
        m = R.Model()
        u0 = 0.01 / s
        rho, u = W.taylor_green_2d(nx, ny, dx[0], dx[1], u0, 1.0, lat.cs2)
        f = R.init_equilibrium(lat, m, S, rho, u)
        T = 300.0
        f = R.step(lat, m, S, f, int(round(T / dt)))
        uu = R.fields(lat, m, f)[1]
        k2 = (2 * np.pi / 16) ** 2 + (2 * np.pi / 8) ** 2
        _, ue = W.taylor_green_2d(nx, ny, dx[0], dx[1], u0 * np.exp(-nu * k2 * T), 1.0, lat.cs2)
        errs.append(np.sqrt(((uu - ue) ** 2).sum() / (ue ** 2).sum()))
    assert np.log2(errs[0] / errs[1]) > 1.7


def test_couette_moving_lid():
    """Resting bottom wall, lid moving at U on top (half-way bounce-back with
    the REDF linear term), x periodic: the steady profile is the exact line
    u(y) = U (y + dy/2) / H on the rectangular lattice."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    nu, U = 0.1, 0.02
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, 0.1, 1.1))
    ny, nx = 16, 2
    H = ny * lat.dx[1]
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    f = R.step(lat, m, S, f, 8000, walls=(1,), lid=(1, (U, 0.0), 1.0))
    rho, u = R.fields(lat, m, f)
    y = (np.arange(ny) + 0.5) * lat.dx[1]
    np.testing.assert_allclose(u[0][0, :, 0], U * y / H, rtol=0, atol=1e-6 * U)
    np.testing.assert_allclose(u[1], 0, atol=1e-12)


def test_cavity_walls_conserve_mass():
    """All four walls closed, lid moving: bounce-back conserves mass exactly
    (every population that would leave returns to its node)."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, 0.05, 0.05, 1.1))
    m = R.Model()
    f = W.random_populations(9, (1, 12, 10), seed=6)
    m0 = f.sum()
    f = R.step(lat, m, S, f, 50, walls=(0, 1), lid=(1, (0.05, 0.0), 1.0))
    assert abs(f.sum() - m0) < 1e-12 * m0


def _cavity_leaves_range(d, steps, check=100):
    """Step one seeded cavity from rest in the oracle; the first check step at
    which its state leaves the method's range (a non-finite value or
    max |u|^2 >= c_s^2), else None."""
    lat = R.make_lattice("D2Q9", (d["dx"], d["dy"]), 1.0, d["cs2"] if d["cs2"] > 0 else None)
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, d["nu"], d["nu_bulk"], d["s_free"]))
    m = R.Model(R.NSE, rho0=1.0)
    f = R.init_equilibrium(lat, m, S, np.ones((1, d["ny"], d["nx"])), np.zeros((2, 1, d["ny"], d["nx"])))
    for s in range(check, steps + 1, check):
        with np.errstate(all="ignore"):
            f = R.step(lat, m, S, f, check, walls=(0, 1), lid=(1, (d["lid_u"], 0.0), 1.0))
            u = R.fields(lat, m, f)[1]
            if not np.isfinite(f).all() or float((u * u).sum(axis=0).max()) >= lat.cs2:
                return s
    return None


def test_underresolved_batched_cavity_is_unstable_in_the_method():
    """Cavity 460 of the 512 seeded cavities of the batched workload (seed 4:
    46 x 33 nodes, dy/dx = 2, Re 943, lid 0.05) leaves the method's range
    within 600 steps from rest in the FP64 oracle itself, so a batch that
    retires it as unstable reports the method, not the kernels; cavity 410
    (84 x 33, dy/dx = 4, Re 272) stays in range for 1000 steps."""
    doms = W.cavity_domains(512, seed=4)
    d = doms[460]
    assert (d["nx"], d["ny"], d["dy"] / d["dx"]) == (46, 33, 2.0)
    assert _cavity_leaves_range(d, 600) is not None
    assert _cavity_leaves_range(doms[410], 1000) is None


# ---------------------------------------------------------------- Eqs. (4-35), (fne)
@pytest.mark.parametrize("name,dx", [("D2Q9", (1.0, 0.5)), ("D3Q27", (1.0, 0.5, 0.8))])
def test_velocity_gradient_exact_for_linear_fields(name, dx):
    """Central and one-sided differences are exact on a linear field, so the
    stencil returns the generating matrix at every node, walls included."""
    lat = R.make_lattice(name, dx)
    d = lat.d
    shape = (1, 6, 7) if d == 2 else (5, 6, 7)
    G = np.random.default_rng(3).normal(size=(d, d))
    X = W.grid(shape, lat.dx)
    u = np.zeros((d,) + shape)
    for b in range(d):
        for a in range(d):
            u[b] += G[a, b] * X[a]
    g = R.velocity_gradient(lat, u)
    for a in range(d):
        for b in range(d):
            np.testing.assert_allclose(g[a, b], G[a, b], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,dx", [("D2Q9", (1.0, 0.5)), ("D3Q19", (1.0, 1.0, 0.5)), ("D3Q27", (1.0, 0.5, 0.8))])
def test_noneq_moment_matches_couette_steady_state(name, dx):
    """The shear component of Eq. (4-35) equals the non-equilibrium second
    moment sum c_x c_y (f - f^eq) that the method itself settles to in
    steady Couette flow (lid on y = H, exact gradient U / H)."""
    lat = R.make_lattice(name, dx)
    d = lat.d
    nu, U = 0.1, 0.02
    r = R.rates_from_viscosity(lat, nu, 0.1, 1.1)
    S = R.relaxation_matrix(lat, r)
    shape = (1, 16, 2) if d == 2 else (2, 16, 2)
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones(shape), np.zeros((d,) + shape))
    f = R.step(lat, m, S, f, 6000, walls=(1,), lid=(1, (U,) + (0.0,) * (d - 1), 1.0))
    rho, u = R.fields(lat, m, f)
    fne = (f - R.init_equilibrium(lat, m, S, rho, u)).reshape(lat.q, -1)
    m2 = np.einsum("ja,jb,jn->nab", lat.cv, lat.cv, fne)
    g = np.zeros((d, d, rho.size))
    g[1, 0] = U / (shape[1] * lat.dx[1])
    pred = R.noneq_second_moment(lat, r, rho.reshape(-1), g)
    np.testing.assert_allclose(m2[:, 0, 1], pred[:, 0, 1], rtol=1e-3)
    np.testing.assert_allclose(m2[:, 1, 0], pred[:, 1, 0], rtol=1e-3)


@pytest.mark.parametrize("name,dx", [("D2Q9", (1.0, 0.5)), ("D3Q27", (1.0, 0.5, 0.8))])
def test_noneq_moment_matches_taylor_green(name, dx):
    """Diagonal and shear components of Eq. (4-35) against the measured
    non-equilibrium moments of a decaying Taylor-Green vortex (bulk viscosity
    different from the shear viscosity; the flow is divergence-free), within
    the central-difference error (k dx)^2 / 6."""
    lat = R.make_lattice(name, dx)
    d = lat.d
    r = R.rates_from_viscosity(lat, 0.02, 0.05, 1.1)
    S = R.relaxation_matrix(lat, r)
    m = R.Model()
    n = 32
    rho0, u2 = W.taylor_green_2d(n, n, lat.dx[0], lat.dx[1], 1e-4, 1.0, lat.cs2)
    if d == 3:
        rho0 = np.repeat(rho0, 2, axis=0)
        u = np.zeros((3,) + rho0.shape)
        u[:2] = np.repeat(u2, 2, axis=1)
    else:
        u = u2
    f = R.step(lat, m, S, R.init_noneq(lat, m, S, r, rho0, u), 100)
    rho, uu = R.fields(lat, m, f)
    fne = (f - R.init_equilibrium(lat, m, S, rho, uu)).reshape(lat.q, -1)
    m2 = np.einsum("ja,jb,jn->nab", lat.cv, lat.cv, fne)
    g = np.zeros((d, d, rho.size))
    for a in range(2):
        for b in range(2):
            g[a, b] = ((np.roll(uu[b], -1, axis=2 - a) - np.roll(uu[b], 1, axis=2 - a)) / (2 * lat.dx[a])).ravel()
    pred = R.noneq_second_moment(lat, r, rho.reshape(-1), g)
    for a, b in [(0, 0), (1, 1), (0, 1)]:
        err = np.abs(m2[:, a, b] - pred[:, a, b]).max() / np.abs(pred[:, a, b]).max()
        assert err < 0.015, (a, b, err)


def test_noneq_start_removes_initial_transient():
    """Starting Couette flow from f^eq + f^ne (Eq. fne) of its exact profile
    leaves the interior nearly unchanged after one step; starting from f^eq
    alone does not."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    r = R.rates_from_viscosity(lat, 0.1, 0.1, 1.1)
    S = R.relaxation_matrix(lat, r)
    m = R.Model()
    U, ny = 0.02, 16
    y = (np.arange(ny) + 0.5) * lat.dx[1]
    u = np.zeros((2, 1, ny, 2))
    u[0] = (U * y / (ny * lat.dx[1]))[None, :, None]
    rho = np.ones((1, ny, 2))
    change = []
    for f0 in (R.init_equilibrium(lat, m, S, rho, u), R.init_noneq(lat, m, S, r, rho, u)):
        f1 = R.step(lat, m, S, f0, 1, walls=(1,), lid=(1, (U, 0.0), 1.0))
        change.append(np.abs(f1 - f0)[:, :, 2:-2].max())
    assert change[1] < 0.1 * change[0]


# ---------------------------------------------------------------- Eqs. (4-32), (4-33)
@pytest.mark.parametrize("name,dx", [("D2Q9", (1.0, 0.5)), ("D3Q19", (1.0, 1.0, 0.5)), ("D3Q27", (1.0, 0.5, 0.8))])
def test_local_stress_couette(name, dx):
    """Steady Couette flow (lid U on y = H): the local strain rate of
    Eq. (4-33) is U / (2H) at every node and the stress of Eq. (4-32) is
    rho nu U / H, with no normal components."""
    lat = R.make_lattice(name, dx)
    d = lat.d
    nu, U = 0.1, 0.02
    r = R.rates_from_viscosity(lat, nu, 0.1, 1.1)
    S = R.relaxation_matrix(lat, r)
    shape = (1, 16, 2) if d == 2 else (2, 16, 2)
    m = R.Model()
    f = R.init_equilibrium(lat, m, S, np.ones(shape), np.zeros((d,) + shape))
    f = R.step(lat, m, S, f, 6000, walls=(1,), lid=(1, (U,) + (0.0,) * (d - 1), 1.0))
    rho, _ = R.fields(lat, m, f)
    stress, strain = R.local_stress(lat, m, r, f)
    H = shape[1] * lat.dx[1]
    np.testing.assert_allclose(strain[0, 1], U / (2 * H), rtol=1e-5)
    np.testing.assert_allclose(strain[1, 0], U / (2 * H), rtol=1e-5)
    np.testing.assert_allclose(stress[0, 1], rho * nu * U / H, rtol=1e-5)
    assert np.abs(strain[0, 0]).max() < 1e-2 * U / H


def test_local_stress_taylor_green():
    """Decaying Taylor-Green vortex on the rectangular rD2Q9 lattice: the
    local strain rate equals the analytic velocity gradients of the decayed
    vortex (normal and shear components) within 1%."""
    lat = R.make_lattice("D2Q9", (1.0, 0.5))
    r = R.rates_from_viscosity(lat, 0.02, 0.05, 1.1)
    S = R.relaxation_matrix(lat, r)
    m = R.Model()
    n, u0 = 32, 1e-3
    rho0, uinit = W.taylor_green_2d(n, n, 1.0, 0.5, u0, 1.0, lat.cs2)
    f = R.step(lat, m, S, R.init_noneq(lat, m, S, r, rho0, uinit), 100)
    _, u = R.fields(lat, m, f)
    _, strain = R.local_stress(lat, m, r, f)
    kx, ky = 2 * np.pi / n, 2 * np.pi / (n * 0.5)
    X, Y, _ = W.grid((1, n, n), (1.0, 0.5))
    a = np.abs(u[0]).max()               # decayed amplitude
    gxx = a * kx * np.sin(kx * X) * np.sin(ky * Y)
    gxy = 0.5 * a * (kx * kx / ky - ky) * np.cos(kx * X) * np.cos(ky * Y)
    assert np.abs(strain[0, 0] - gxx).max() < 0.01 * np.abs(gxx).max()
    assert np.abs(strain[1, 1] + gxx).max() < 0.01 * np.abs(gxx).max()
    assert np.abs(strain[0, 1] - gxy).max() < 0.01 * np.abs(gxy).max()


# ---------------------------------------------------------------- rD2Q5 / rD3Q7, Eq. (4-16)
@pytest.mark.parametrize("name,dx", [("D2Q5", (1.0, 1.0)), ("D2Q5", (1.0, 0.6)), ("D3Q7", (1.0, 1.0, 1.0)),
                                     ("D3Q7", (1.0, 0.8, 0.5))])
def test_axis_lattice_weights(name, dx):
    """Remark I of Sec. III: omega_alpha = c_s^2 / (2 c_alpha^2); the standard
    D2Q5 (c_s^2 = 1/3: 1/3, 1/6) and D3Q7 (c_s^2 = 1/4: 1/4, 1/8) weights;
    sum omega = 1, first moments 0 and second moments c_s^2 I, so the
    linear EDF g^eq(phi, B, 0) has moments (phi, B, c_s^2 phi I)."""
    lat = R.make_lattice(name, dx)
    if dx == (1.0,) * lat.d:
        want = [1 / 3, 1 / 6] if name == "D2Q5" else [1 / 4, 1 / 8]
        np.testing.assert_allclose(lat.w, [want[0]] + [want[1]] * (lat.q - 1), rtol=1e-15)
    assert abs(lat.w.sum() - 1) < 1e-15
    np.testing.assert_allclose(lat.cv.T @ lat.w, 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("j,ja,jb->ab", lat.w, lat.cv, lat.cv), lat.cs2 * np.eye(lat.d), atol=1e-15)
    phi = np.array([0.7, 1.3])
    B = np.array([[0.01, -0.02, 0.03][: lat.d], [0.0, 0.05, -0.01][: lat.d]])
    g = R.geq(lat, phi, B, np.zeros((2, lat.d, lat.d)))
    M = R.moment_matrix(lat)
    mom = M @ g
    mons = R.monomials(name)
    for k, a in enumerate(mons):
        o = sum(a)
        if o == 0:
            want = phi
        elif o == 1:
            want = B[:, int(np.argmax(a))]
        else:
            want = lat.cs2 * phi
        np.testing.assert_allclose(mom[k], want, atol=1e-15)


def test_simple_ncde_bgk_reduction():
    """Standard D2Q5, no advection, every rate 1/tau: the simplified NCDE
    collision (Eq. 4-16) is the textbook BGK diffusion step
    f* = f - (f - omega phi) / tau."""
    lat = R.make_lattice("D2Q5", (1.0, 1.0))
    tau = 0.8
    s = 1 / tau
    S = R.relaxation_matrix(lat, R.Rates(s, np.full(2, s), np.full(2, s), np.full(2, s), np.full((2, 2), s), s))
    f = W.random_populations(5, (20,), seed=21)
    m = R.Model(R.NCDE_SIMPLE_LINEAR, adv=(0.0, 0.0))
    phi = f.sum(0)
    want = f - (f - lat.w[:, None] * phi[None, :]) / tau
    np.testing.assert_allclose(R.collide(lat, m, S, f), want, atol=1e-15)


@pytest.mark.parametrize("name,dx", [("D2Q5", (1.0, 0.6)), ("D3Q7", (1.0, 0.8, 0.5)), ("D2Q9", (1.0, 0.6))])
@pytest.mark.parametrize("kind", [R.NCDE_SIMPLE_LINEAR, R.NCDE_SIMPLE_QUAD])
def test_simple_ncde_conserves_phi(name, dx, kind):
    """phi is a collision invariant up to the source (Eq. 4-18-1 for the
    NCDE: sum f* = sum f + dt S) whatever dB/dt is; on a periodic grid the
    total is conserved over steps without a source."""
    lat = R.make_lattice(name, dx)
    r = R.Rates(1.0, np.full(lat.d, 1.4), np.full(lat.d, 1.1), np.full(lat.d, 1.1),
                np.full((lat.d, lat.d), 1.1), 1.1)
    S = R.relaxation_matrix(lat, r)
    f = W.random_populations(lat.q, (25,), seed=22)
    m = R.Model(kind, adv=(0.05, 0.02, -0.01), source=2e-5)
    dB = np.random.default_rng(3).normal(scale=1e-3, size=(25, lat.d))
    np.testing.assert_allclose(R.collide(lat, m, S, f, dB).sum(0), f.sum(0) + 2e-5, atol=5e-15)
    m = R.Model(kind, adv=(0.05, 0.02, -0.01))
    shp = (4, 5, 6) if lat.d == 3 else (1, 5, 6)
    g = W.random_populations(lat.q, shp, seed=23)
    g2 = R.step(lat, m, S, g, 10)
    assert abs(g2.sum() - g.sum()) < 1e-12 * g.sum()


def simple_hill_error(n_scale, lattice, adv, with_dB=True):
    nx, ny = 32 * n_scale, 40 * n_scale
    L = (32.0, 24.0)
    dx = (L[0] / nx, L[1] / ny)
    dt = 1.0 / (n_scale * n_scale)
    lat = R.make_lattice(lattice, dx, dt)
    D = 0.05
    tau = D / (lat.cs2 * dt) + 0.5
    rr = R.Rates(1.0, np.full(2, 1 / tau), np.full(2, 1.1), np.full(2, 1.1), np.full((2, 2), 1.1), 1.1)
    S = R.relaxation_matrix(lat, rr)
    m = R.Model(R.NCDE_SIMPLE_LINEAR, adv=adv)
    phi0 = W.gaussian_hill((1, ny, nx), dx, 3.0, peak=1.0, adv=adv, diff=D, t=0.0)
    f = R.init_equilibrium(lat, m, S, phi0, np.zeros((2, 1, ny, nx)))
    n = int(round(40.0 / dt))
    if with_dB:
        f = R.step(lat, m, S, f, n)
    else:                       # a planted mistake: dB/dt dropped (fresh state every step)
        for _ in range(n):
            f = R.step(lat, m, S, f, 1)
    phi = R.fields(lat, m, f)[0]
    ref = W.gaussian_hill((1, ny, nx), dx, 3.0, peak=1.0, adv=adv, diff=D, t=40.0)
    return np.sqrt(((phi - ref) ** 2).sum() / (ref ** 2).sum())


def test_simple_ncde_hill_second_order_on_rd2q5():
    """The simplified NCDE (Eq. 4-16) on the rectangular rD2Q5 lattice
    follows the closed-form advected, diffusing Gaussian hill at second
    order under diffusive refinement."""
    e1 = simple_hill_error(1, "D2Q5", (0.05, 0.02))
    e2 = simple_hill_error(2, "D2Q5", (0.05, 0.02))
    assert e1 < 1e-2
    assert np.log2(e1 / e2) > 1.8


def test_simple_ncde_needs_the_dBdt_term():
    """With faster advection the G = (I - S_1/2) dB/dt term of Eq. (4-16)
    carries the correction: dropping it makes the hill error several times
    larger."""
    e = simple_hill_error(1, "D2Q5", (0.2, 0.1))
    e_no = simple_hill_error(1, "D2Q5", (0.2, 0.1), with_dB=False)
    assert e < 0.02 and e < 0.4 * e_no, (e, e_no)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q27"])
def test_sampled_step_equals_the_full_step(name):
    """collide_stream_at (the oracle at selected nodes, for full-size
    checks) equals one full periodic step at every node of a small field."""
    dx = (1.0, 0.7, 0.55)
    lat = R.make_lattice(name, dx[: 2 if name == "D2Q9" else 3])
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, 0.03, 0.05, 1.1))
    m = R.Model(R.NSE, force=(1e-4, -2e-4, 1e-4), source=2e-5)
    shape = (1, 5, 6) if name == "D2Q9" else (3, 4, 5)
    f = W.random_populations(lat.q, shape, seed=9)
    full = R.step(lat, m, S, f, 1)
    nodes = np.array([(z, y, x) for z in range(shape[0]) for y in range(shape[1]) for x in range(shape[2])])
    got = R.collide_stream_at(lat, m, S, f, nodes)
    np.testing.assert_allclose(got, full.reshape(lat.q, -1), rtol=0, atol=1e-15)


# ---------------------------------------------------------------- the auxiliary distribution G with a source
def _collide_without_G(lat, m, S, fl):
    """A planted mistake: the oracle's raw-basis collision with G dropped."""
    rho, u = R.macroscopic(lat, m, fl)
    feq, _, F = R.equilibrium_and_sources(lat, m, S, rho, u)
    M, I = R.moment_matrix(lat), np.eye(lat.q)
    mb, meq, mF = M @ fl, M @ feq, M @ F
    return np.linalg.solve(M, mb - S @ (mb - meq) + lat.dt * (I - 0.5 * S) @ mF)


def _steady_sourced(model, S, lat, nx, ny, steps, with_G):
    f = R.init_equilibrium(lat, model, S, np.ones((1, ny, nx)), np.zeros((2, 1, ny, nx)))
    for _ in range(steps):
        fl = f.reshape(lat.q, -1)
        fs = R.collide(lat, model, S, fl) if with_G else _collide_without_G(lat, model, S, fl)
        f = R.stream(lat, fs.reshape(f.shape))
    return R.fields(lat, model, f)


@pytest.mark.parametrize("kind,S0,bound", [(R.NCDE_LINEAR, 1e-3, 2e-3), (R.NCDE_QUAD, 1e-4, 3e-3)])
def test_sourced_ncde_steady_state_needs_G(kind, S0, bound):
    """phi_t + u phi_x = D phi_xx + S0 sin(kx) on the rectangular rD2Q9
    lattice (dx = 1, dy = 0.7), periodic, u = 0.2 along x: the steady state
    is phi = 1 + A sin(kx) + B cos(kx), A = S0 D / (u^2 + D^2 k^2),
    B = -u A / (D k) (for the quadratic kind B = u phi^2/2 at small
    amplitude, where the same linear solution holds to O(A)).  The oracle
    reaches it within `bound`; dropping G = g^eq(0, M_1G, 0) of Eq. (4-11),
    M_1G = (I - S_1/2) B' S, makes the error many times larger."""
    lat = R.make_lattice("D2Q9", (1.0, 0.7), 1.0)
    nx, ny, u, D = 32, 2, 0.2, 0.05
    tau = D / (lat.cs2 * lat.dt) + 0.5
    rr = R.Rates(1.0, np.full(2, 1 / tau), np.full(2, 1.1), np.full(2, 1.1), np.full((2, 2), 1.1), 1.1)
    S = R.relaxation_matrix(lat, rr)
    x = np.arange(nx, dtype=float)
    k = 2 * np.pi / nx
    src = np.broadcast_to(S0 * np.sin(k * x), (ny, nx)).reshape(-1).copy()
    model = R.Model(kind, adv=(u, 0.0, 0.0), source=src)
    A = S0 * D / (u * u + D * D * k * k)
    exact = 1.0 + A * np.sin(k * x) - u * A / (D * k) * np.cos(k * x)
    err = []
    for with_G in (True, False):
        phi = _steady_sourced(model, S, lat, nx, ny, 4000, with_G)[0][0, 0]
        err.append(np.abs(phi - exact).max() / np.abs(exact - 1.0).max())
    assert err[0] < bound and err[0] < 0.2 * err[1], err


def test_nse_mass_source_steady_state_needs_G():
    """NSE with a mass source Sbar = S0 sin(kx) on rD2Q9 (dx = 1, dy = 0.7),
    periodic, small S0: continuity gives u = -S0 cos(kx) / (k rho0) and the
    normal viscous stress, with the longitudinal viscosity nu_L = 2 nu
    (1 - 1/d) + nu_b of the sound-attenuation pin, balances the pressure:
    rho = rho0 + nu_L S0 sin(kx) / c_s^2.  The oracle matches both within
    1 %; dropping G (its M_2G = (I - S_2/2) c_s^2 Sbar I here, Eq.
    M2GComput a) leaves u unchanged but makes the density error about 20 %."""
    lat = R.make_lattice("D2Q9", (1.0, 0.7), 1.0)
    nx, ny, nu, nub, S0 = 32, 2, 0.05, 0.05, 1e-5
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, nu, nub, 1.1))
    x = np.arange(nx, dtype=float)
    k = 2 * np.pi / nx
    src = np.broadcast_to(S0 * np.sin(k * x), (ny, nx)).reshape(-1).copy()
    model = R.Model(R.NSE, source=src)
    nuL = 2 * (1 - 1 / 2) * nu + nub
    rho_ex = 1.0 + nuL * S0 * np.sin(k * x) / lat.cs2
    u_ex = -S0 * np.cos(k * x) / k
    res = []
    for with_G in (True, False):
        rho, u = _steady_sourced(model, S, lat, nx, ny, 4000, with_G)
        res.append((np.abs(rho[0, 0] - rho_ex).max() / np.abs(rho_ex - 1).max(),
                    np.abs(u[0, 0, 0] - u_ex).max() / np.abs(u_ex).max()))
    (er, eu), (er_no, _) = res
    assert er < 1e-2 and eu < 1e-2 and er < 0.1 * er_no, res


# ---------------------------------------------------------------- brute force in exact arithmetic
def _exact_step(name, c, cs2, nu, nub, sfree, shape, seed):
    """One unforced NSE collide-and-stream step in sympy rationals, written
    from the printed formulas: weights (Eqs. 3-3-5 / 3-3-8 with the tensor
    omega_19), f^eq (Eq. NSEfeq), rates (Eq. 4-31), the S_2 block as the
    exact inverse of Eq. (4-27-1), m* = m - S (m - m^eq), f* = M^-1 m*,
    periodic pull streaming.  Returns (f0, f1) as float arrays."""
    sp = pytest.importorskip("sympy")
    R_ = sp.Rational
    d = len(c)
    e = R.velocity_indices(name)
    q = e.shape[0]
    cv = [[R_(int(e[j, a])) * c[a] for a in range(d)] for j in range(q)]
    # weights
    w = [R_(0)] * q
    for j in range(1, q):
        nz = [a for a in range(d) if e[j, a] != 0]
        if name == "D2Q9":
            w5 = cs2 ** 2 / (4 * c[0] ** 2 * c[1] ** 2)
            w[j] = w5 if len(nz) == 2 else cs2 / (2 * c[nz[0]] ** 2) - 2 * w5
        else:
            w19 = cs2 ** 3 / (8 * c[0] ** 2 * c[1] ** 2 * c[2] ** 2) if name == "D3Q27" else R_(0)
            edge = {}
            for (a, b) in ((0, 1), (0, 2), (1, 2)):
                edge[(a, b)] = cs2 ** 2 / (4 * c[a] ** 2 * c[b] ** 2) - 2 * w19
            if len(nz) == 3:
                w[j] = w19
            elif len(nz) == 2:
                w[j] = edge[tuple(nz)]
            else:
                a = nz[0]
                w[j] = cs2 / (2 * c[a] ** 2) - 2 * sum(v for k, v in edge.items() if a in k) - 4 * w19
    w[0] = 1 - sum(w[1:])
    # rates and S
    s_ab = 1 / (nu / cs2 + R_(1, 2))
    ss = [1 / (2 * nu / (c[a] ** 2 - cs2) + R_(1, 2)) for a in range(d)]
    sb = [1 / (d * nub / (c[a] ** 2 - cs2) + R_(1, 2)) for a in range(d)]
    av = [(1 / sb[a] - 1 / ss[a]) * (c[a] ** 2 - cs2) for a in range(d)]
    bv = [1 / (c[a] ** 2 - cs2) for a in range(d)]
    S2inv = sp.Matrix(d, d, lambda i, k: (1 / ss[i] if i == k else 0) + av[i] * bv[k] / d)
    S2 = S2inv.inv()
    mons = R.monomials(name)
    M = sp.Matrix(q, q, lambda k, j: sp.prod([cv[j][a] ** mons[k][a] for a in range(d)]))
    S = sp.zeros(q, q)
    diag2 = {}
    for k, a in enumerate(mons):
        o = sum(a)
        if o == 2 and max(a) == 2:
            diag2[a.index(2)] = k
        elif o == 2:
            S[k, k] = s_ab
        else:
            S[k, k] = sfree
    for al, ka in diag2.items():
        for be, kb in diag2.items():
            S[ka, kb] = S2[al, be]
    Minv = M.inv()
    rng = np.random.default_rng(seed)
    nodes = int(np.prod(shape))
    f0 = [[w[j] * (1 + R_(int(rng.integers(-50, 51)), 1000)) for _ in range(nodes)] for j in range(q)]
    fstar = [[None] * nodes for _ in range(q)]
    for n in range(nodes):
        f = sp.Matrix([f0[j][n] for j in range(q)])
        rho = sum(f)
        u = [sum(cv[j][a] * f[j] for j in range(q)) / rho for a in range(d)]
        feq = []
        for j in range(q):
            t = 1 + sum(cv[j][a] * u[a] for a in range(d)) / cs2
            t += sum(u[a] ** 2 * (cv[j][a] ** 2 - cs2) / (cs2 * (c[a] ** 2 - cs2)) for a in range(d))
            t += sum(u[a] * u[b] * cv[j][a] * cv[j][b] / (2 * cs2 ** 2) for a in range(d) for b in range(d) if a != b)
            feq.append(w[j] * rho * t)
        m = M * f
        mstar = m - S * (m - M * sp.Matrix(feq))
        fs = Minv * mstar
        for j in range(q):
            fstar[j][n] = fs[j]
    # periodic pull streaming on (nz, ny, nx)
    nzs, nys, nxs = shape
    f1 = [[None] * nodes for _ in range(q)]
    for j in range(q):
        ex = int(e[j, 0]); ey = int(e[j, 1]); ez = int(e[j, 2]) if d == 3 else 0
        for z in range(nzs):
            for y in range(nys):
                for x in range(nxs):
                    src = (((z - ez) % nzs) * nys + (y - ey) % nys) * nxs + (x - ex) % nxs
                    f1[j][(z * nys + y) * nxs + x] = fstar[j][src]
    to = lambda F: np.array([[float(v) for v in row] for row in F]).reshape((q,) + shape)
    return to(f0), to(f1)


@pytest.mark.parametrize("name,c,shape", [("D2Q9", (1, (1, 2)), (1, 2, 3)), ("D3Q19", (1, 1, (1, 2)), (2, 2, 3)),
                                          ("D3Q27", (1, (3, 4), (1, 2)), (2, 2, 3))])
def test_oracle_matches_exact_rational_step(name, c, shape):
    """Brute force: the oracle's FP64 step equals one step computed in exact
    rational arithmetic from the printed formulas (to 1e-14)."""
    sp = pytest.importorskip("sympy")
    cr = [sp.Rational(*v) if isinstance(v, tuple) else sp.Rational(v) for v in c]
    cs2 = min(v * v for v in cr) / 3
    nu, nub, sfree = sp.Rational(1, 50), sp.Rational(1, 20), sp.Rational(11, 10)
    f0, f1 = _exact_step(name, cr, cs2, nu, nub, sfree, shape, seed=5)
    lat = R.make_lattice(name, tuple(float(v) for v in cr))
    r = R.rates_from_viscosity(lat, float(nu), float(nub), float(sfree))
    S = R.relaxation_matrix(lat, r)
    got = R.step(lat, R.Model(), S, f0, 1)
    np.testing.assert_allclose(got, f1, rtol=0, atol=1e-14)
