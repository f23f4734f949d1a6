"""Slab decomposition on one GPU: several slabs of one periodic grid driven
from one process (slab.LocalSlabs: the library's rmrtlb_halo_pack and
rmrtlb_halo_unpack with device copies between the slabs' buffers) give the
single grid's run bit for bit, every storage (the 16-bit stochastic rounding
draws its random bits by global node index), and the FP64 run matches the
oracle.  The ring exchange between processes is covered on CPU
(test_slab_host.py)."""
import numpy as np
import pytest

import oracle.rmrt as R
import workloads as W
from cases import Case, normwise, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_2206_00366_gb300 import build
    build.build()


CASES = [("D2Q9", (72, 30, 1), (1.0, 0.6, 1.0), 3, "nse", "raw"),
         ("D2Q9", (36, 17, 1), (1.0, 0.6, 1.0), 2, "ncde_quad", "raw"),
         ("D3Q19", (16, 12, 10), (1.0, 0.8, 0.5), 2, "nse", "central"),
         ("D3Q27", (16, 12, 9), (1.0, 0.8, 0.5), 3, "nse", "raw"),
         ("D3Q27", (13, 7, 5), (1.0, 0.8, 0.5), 2, "nse", "central_hermite"),
         ("D2Q5", (18, 12, 1), (1.0, 0.6, 1.0), 3, "ncde_simple_linear", "raw")]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "e3m12"])
@pytest.mark.parametrize("lattice,shape,spacing,parts,kind,basis", CASES)
def test_slabs_equal_the_single_grid(lattice, shape, spacing, parts, kind, basis, storage):
    from paper_2206_00366_gb300.rmrtlb import Solver
    from paper_2206_00366_gb300.slab import LocalSlabs
    if lattice == "D2Q5" and storage == "f16":
        pytest.skip("covered by the other storages")
    params = dict(nu=0.02, nu_bulk=0.03, s_free=1.1, rho0=1.0 if kind == "nse" else 0.0, diffusivity=0.02,
                  adv=(0.05, -0.03, 0.02), check_every=5)
    nx, ny, nz = shape
    d = 2 if lattice.startswith("D2") else 3
    rho, u = W.random_fields((nz, ny, nx), d, seed=21, umax=0.03)
    if kind != "nse":
        rho = rho - 0.9                                   # phi of order 0.1 around phi0 = 0
    whole = Solver(lattice, shape, spacing, 1.0, params, kind, basis, storage)
    whole.init_equilibrium(rho, u)
    whole.step(12)
    slabs = LocalSlabs(parts, lattice, shape, spacing, 1.0, params, kind, basis, storage)
    slabs.init_equilibrium(rho, u)
    slabs.step(12)
    np.testing.assert_array_equal(slabs.populations(), whole.get_populations())
    r1, u1 = slabs.moments()
    r0, u0 = whole.moments()
    np.testing.assert_array_equal(r1, r0)
    # the reduced check of the slabs equals the whole grid's (sums in another order)
    g = slabs.check()
    w = whole.last_check()
    assert abs(g[0] - w[0]) <= 1e-12 * abs(w[0])
    np.testing.assert_allclose(g[1:5], w[1:5], rtol=1e-9, atol=1e-13 * abs(w[0]))
    assert abs(g[5] - w[5]) <= 1e-9 * abs(w[5])
    assert int(g[7]) == int(w[7]) == 0


def test_slabs_match_the_oracle_fp64():
    from paper_2206_00366_gb300.slab import LocalSlabs
    case = Case("D3Q19", (10, 8, 7), (1.0, 0.8, 0.5), basis="central", nu=0.02, nu_bulk=0.03)
    rho, u = W.random_fields(case.field_shape, 3, seed=4, umax=0.03)
    _, ro, uo = oracle_run(case, 9, fields=(rho, u))
    slabs = LocalSlabs(3, "D3Q19", case.shape, case.spacing, 1.0, case.gpu_params(), "nse", "central", "f64")
    slabs.init_equilibrium(rho, u)
    slabs.step(9)
    rg, ug = slabs.moments()
    assert normwise(rg, ro) <= 1e-12
    assert normwise(ug, uo) <= 1e-12


def test_halo_rejects_host_buffers():
    import torch

    from paper_2206_00366_gb300 import rmrtlb as B
    s = B.Solver("D2Q9", (8, 6, 1), (1.0, 1.0, 1.0), 1.0, dict(nu=0.02, nu_bulk=0.03, s_free=1.1, rho0=1.0))
    n = B.rmrtlb_halo_bytes(s.h)
    assert n == 3 * 8 * 4                                  # three crossing directions, one row of 8, FP32
    dev = torch.empty(n, dtype=torch.uint8, device="cuda")
    host = np.zeros(n, dtype=np.uint8)
    with pytest.raises(B.RmrtlbError):
        B.rmrtlb_halo_pack(s.h, host.ctypes.data, dev.data_ptr())
    with pytest.raises(B.RmrtlbError):
        B.rmrtlb_halo_unpack(s.h, dev.data_ptr(), host.ctypes.data)


SPLIT_CASES = [("D2Q9", (40, 12, 1), "nse", "raw"), ("D2Q9", (36, 4, 1), "nse", "raw"),
               ("D3Q19", (16, 8, 9), "nse", "central"), ("D3Q27", (12, 6, 7), "nse", "raw"),
               ("D2Q5", (18, 12, 1), "ncde_simple_linear", "raw"), ("D3Q7", (10, 6, 8), "ncde_simple_linear", "raw")]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "e3m12"])
@pytest.mark.parametrize("lattice,shape,kind,basis", SPLIT_CASES)
def test_interior_and_boundary_parts_equal_the_step(lattice, shape, kind, basis, storage):
    """rmrtlb_step_interior (planes 2 .. n - 3 of the slab axis) followed by
    rmrtlb_step_boundary, or by rmrtlb_step, is bitwise rmrtlb_step, periodic
    check included; with fewer than five planes the interior part steps
    nothing; a second interior part before the step is completed is
    refused."""
    from paper_2206_00366_gb300 import rmrtlb as B
    from paper_2206_00366_gb300.rmrtlb import Solver
    params = dict(nu=0.02, nu_bulk=0.03, s_free=1.1, rho0=1.0 if kind == "nse" else 0.0, diffusivity=0.02,
                  adv=(0.05, -0.03, 0.02), check_every=3)
    nx, ny, nz = shape
    d = 2 if lattice.startswith("D2") else 3
    rho, u = W.random_fields((nz, ny, nx), d, seed=23, umax=0.03)
    if kind != "nse":
        rho = rho - 0.9
    sp = (1.0, 0.6, 1.0) if d == 2 else (1.0, 0.8, 0.5)
    whole = Solver(lattice, shape, sp, 1.0, params, kind, basis, storage)
    whole.init_equilibrium(rho, u)
    whole.step(7)
    split = Solver(lattice, shape, sp, 1.0, params, kind, basis, storage)
    split.init_equilibrium(rho, u)
    for k in range(7):
        B.rmrtlb_step_interior(split.h)
        if k % 2:
            B.rmrtlb_step_boundary(split.h)
        else:
            split.step(1)
    np.testing.assert_array_equal(split.get_populations(), whole.get_populations())
    np.testing.assert_array_equal(split.last_check(), whole.last_check())
    planes = ny if d == 2 else nz
    B.rmrtlb_step_interior(split.h)
    if planes >= 5:
        with pytest.raises(B.RmrtlbError) as ei:
            B.rmrtlb_step_interior(split.h)
        assert ei.value.status == B.EINVAL
    else:
        B.rmrtlb_step_interior(split.h)                  # nothing stepped, nothing pending
    B.rmrtlb_step_boundary(split.h)
    whole.step(1)
    np.testing.assert_array_equal(split.get_populations(), whole.get_populations())


class _FakeRing:
    """A stand-in for the process group of slab.start_exchange and
    finish_exchange, for several Slab objects in one process on one GPU:
    each rank's n-th posting joins round n, and the first wait on a round
    whose ranks have all posted delivers every rank's buffers to its
    neighbours (device copies), as the ring exchange would."""

    def __init__(self, world):
        self.world, self.rounds, self.count = world, {}, [0] * world

    def start(self, send_up, send_down, recv_from_below, recv_from_above, rank, world, group=None):
        n = self.count[rank]
        self.count[rank] += 1
        self.rounds.setdefault(n, {"posted": {}, "done": False})["posted"][rank] = (
            send_up, send_down, recv_from_below, recv_from_above)
        return [(self, n)]

    @staticmethod
    def finish(reqs):
        import torch
        for ring, n in reqs:
            r = ring.rounds[n]
            if r["done"]:
                continue
            assert len(r["posted"]) == ring.world, "a rank waited before every rank posted"
            torch.cuda.synchronize()
            for k, (_, _, below, above) in r["posted"].items():
                below.copy_(r["posted"][(k - 1) % ring.world][0])
                above.copy_(r["posted"][(k + 1) % ring.world][1])
            torch.cuda.synchronize()
            r["done"] = True


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("lattice,shape,spacing,kind,basis,storage", [
    ("D2Q9", (48, 30, 1), (1.0, 0.6, 1.0), "nse", "raw", "f32"),
    ("D3Q27", (16, 12, 15), (1.0, 0.8, 0.5), "nse", "central", "f16")])
def test_slab_ranks_with_the_exchange_in_flight(monkeypatch, lattice, shape, spacing, kind, basis, storage, world):
    """Slab objects of every rank of a ring driven in turn, one step per call,
    so that each step's exchange is still in flight when the next call
    starts (it lands after that call's interior part): after the last
    finish() the slabs hold the single grid's run bit for bit, and their
    reduced check equals the grid's."""
    from paper_2206_00366_gb300 import slab as SL
    from paper_2206_00366_gb300.rmrtlb import Solver
    ring = _FakeRing(world)
    monkeypatch.setattr(SL, "start_exchange", ring.start)
    monkeypatch.setattr(SL, "finish_exchange", _FakeRing.finish)
    params = dict(nu=0.02, nu_bulk=0.03, s_free=1.1, rho0=1.0, check_every=4)
    nx, ny, nz = shape
    d = 2 if lattice == "D2Q9" else 3
    rho, u = W.random_fields((nz, ny, nx), d, seed=17, umax=0.03)
    whole = Solver(lattice, shape, spacing, 1.0, params, kind, basis, storage)
    whole.init_equilibrium(rho, u)
    whole.step(9)
    slabs = [SL.Slab(lattice, shape, spacing, 1.0, params, kind, basis, storage, rank=r, world=world)
             for r in range(world)]
    for s in slabs:
        s.init_equilibrium(rho, u)
    for _ in range(9):
        for s in slabs:
            s.step(1)
    for s in slabs:
        s.finish()
    ax = SL.field_axis(d) + 1
    got = np.concatenate([s.solver.get_populations() for s in slabs], axis=ax)
    np.testing.assert_array_equal(got, whole.get_populations())
    g = SL.global_check([B_sums(s) for s in slabs])
    w = whole.last_check()
    assert abs(g[0] - w[0]) <= 1e-12 * abs(w[0])
    assert abs(g[5] - w[5]) <= 1e-9 * abs(w[5])


def B_sums(s):
    from paper_2206_00366_gb300 import rmrtlb as B
    return B.rmrtlb_check_sums(s.solver.h)
