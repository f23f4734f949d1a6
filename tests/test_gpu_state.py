"""Checkpoint and resume (rmrtlb_save_state / rmrtlb_load_state): a run
stopped after n1 steps, saved, loaded into a fresh solver with the same
parameters and continued for n2 steps gives bitwise the populations and the
periodic check of the uninterrupted n1 + n2 run — every storage (the 16-bit
stochastic rounding draws its bits from the restored step counter), a
central basis, forcing, and the simplified NCDE with its B(t - dt)
history; blobs in host and in device memory; a blob from a solver with
other parameters, a truncated blob and a corrupted one are rejected and
leave the solver as it was, as is one saved at another node offset (the
random bits of the rounding would differ)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    from paper_2206_00366_gb300 import build
    build.build()


CASES = [("D2Q9", (40, 24, 1), "nse", "raw", False), ("D3Q19", (16, 12, 10), "nse", "central", True),
         ("D3Q27", (16, 10, 8), "nse", "central_hermite", False), ("D2Q5", (30, 20, 1), "ncde_simple_linear", "raw",
                                                                    True), ("D2Q9", (36, 20, 1), "ncde_quad", "raw",
                                                                            True)]


def make(lattice, shape, kind, basis, storage, forced, nu=0.02):
    from paper_2206_00366_gb300.rmrtlb import Solver
    params = dict(nu=nu, nu_bulk=0.03, s_free=1.1, rho0=1.0 if kind.startswith("nse") else 0.0,
                  diffusivity=0.02, adv=(0.04, -0.02, 0.01), check_every=5)
    if forced:
        params.update(force=(1e-5, -2e-5, 3e-6), source=1e-6)
    sp = (1.0, 0.7, 1.0) if shape[2] == 1 else (1.0, 0.7, 0.5)
    return Solver(lattice, shape, sp, 1.0, params, kind, basis, storage)


def fields(lattice, shape, kind):
    nx, ny, nz = shape
    rho, u = W.random_fields((nz, ny, nx), 2 if nz == 1 else 3, seed=31, umax=0.03)
    if not kind.startswith("nse"):
        rho = rho - 0.9
    return rho, u


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "e3m12"])
@pytest.mark.parametrize("lattice,shape,kind,basis,forced", CASES)
def test_resume_is_bitwise_identical(lattice, shape, kind, basis, forced, storage):
    import torch
    if lattice == "D2Q5" and storage == "bf16":
        pytest.skip("covered by the other storages")
    rho, u = fields(lattice, shape, kind)
    n1, n2 = 13, 11                     # a check at steps 5, 10 before the save, 15, 20 after
    a = make(lattice, shape, kind, basis, storage, forced)
    a.init_equilibrium(rho, u)
    a.step(n1 + n2)
    fa, ca = a.get_populations(), a.last_check()
    b = make(lattice, shape, kind, basis, storage, forced)
    b.init_equilibrium(rho, u)
    b.step(n1)
    blob = b.save_state()
    dev = b.save_state(torch.empty(blob.size, dtype=torch.uint8, device="cuda"))
    np.testing.assert_array_equal(dev.cpu().numpy(), blob)
    del b
    for src in (blob, dev):
        c = make(lattice, shape, kind, basis, storage, forced)
        c.init_equilibrium(rho * 0 + (1.0 if kind.startswith("nse") else 0.0), u * 0)   # another state, overwritten
        c.load_state(src)
        c.step(n2)
        np.testing.assert_array_equal(c.get_populations(), fa)
        np.testing.assert_array_equal(c.last_check(), ca)


def test_load_rejects_foreign_truncated_and_corrupted_blobs():
    from paper_2206_00366_gb300 import rmrtlb as B
    lattice, shape, kind, basis, forced = CASES[0]
    rho, u = fields(lattice, shape, kind)
    a = make(lattice, shape, kind, basis, "f32", forced)
    a.init_equilibrium(rho, u)
    a.step(7)
    blob = a.save_state()
    before = a.get_populations()
    other = make(lattice, shape, kind, basis, "f32", forced, nu=0.021)       # another viscosity
    other_storage = make(lattice, shape, kind, basis, "f64", forced)
    from paper_2206_00366_gb300.rmrtlb import Solver
    other_offset = Solver(lattice, shape, (1.0, 0.7, 1.0), 1.0,
                          dict(nu=0.02, nu_bulk=0.03, s_free=1.1, rho0=1.0, diffusivity=0.02,
                               adv=(0.04, -0.02, 0.01), check_every=5, node_offset=4096), kind, basis, "f32")
    bad = blob.copy()
    bad[0] ^= 0xFF
    for target, b in ((other, blob), (other_storage, blob), (other_offset, blob), (a, blob[: blob.size // 2].copy()),
                      (a, bad)):
        with pytest.raises(B.RmrtlbError) as ei:
            target.load_state(b)
        assert ei.value.status == B.EINVAL
    np.testing.assert_array_equal(a.get_populations(), before)
    a.load_state(blob)
    np.testing.assert_array_equal(a.get_populations(), before)
