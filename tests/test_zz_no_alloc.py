"""The allocation-free totals entry point against the solver's own check
and against plain FP64 sums of the same populations.

rmrtlb_population_totals_noalloc serves callers that cannot allocate device
memory (their memory belongs to another allocator, or an allocation would
synchronise the device in the middle of their stream work): it keeps its
reduction scratch in a fixed array inside the library.  This test calls it
through the C ABI twice in a row on device populations and checks both
results against rmrtlb_stats of the same state and against numpy FP64 sums
of the populations copied to the host, at the FP64 tolerance of the parity
tests.  It lives in its own file so that it is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice,shape", [("D2Q9", (70, 41, 1)), ("D3Q27", (24, 20, 18))])
def test_noalloc_totals_match_stats(lattice, shape):
    import torch

    from paper_2206_00366_gb300 import build
    build.build()
    from paper_2206_00366_gb300 import rmrtlb as B
    import workloads as W

    assert torch.cuda.is_available()
    spacing = (1.0, 0.6, 0.5)
    nx, ny, nz = shape
    s = B.Solver(lattice, shape, spacing, 1.0, dict(nu=0.01, nu_bulk=0.03, s_free=1.1, rho0=1.0), "nse", "raw",
                 "f64")
    if lattice == "D2Q9":
        rho, u = W.taylor_green_2d_modes(nx, ny, spacing[0], spacing[1], 1.0, 0.12, seed=3)
    else:
        rho, u = W.taylor_green_3d(nx, ny, nz, *spacing, 0.02, 1.0)
    s.init_equilibrium(rho, u)
    stream = s.stream.cuda_stream
    f = torch.empty((s.q,) + rho.shape, dtype=torch.float64, device="cuda")
    out_dev = torch.full((5,), np.nan, dtype=torch.float64, device="cuda")
    results = []
    for call in range(2):
        s.step(7)
        want = s.stats()                                   # existing entry point (workspace scratch)
        s.get_populations(f)
        host_out = (ctypes.c_double * 5)()
        B.rmrtlb_population_totals_noalloc(B.LATTICE_NAMES[lattice], nx, ny, nz, *spacing, 1.0,
                                           f.data_ptr(), ctypes.addressof(host_out), stream)
        B.rmrtlb_population_totals_noalloc(B.LATTICE_NAMES[lattice], nx, ny, nz, *spacing, 1.0,
                                           f.data_ptr(), out_dev.data_ptr(), stream)
        torch.cuda.synchronize()
        got_h = np.array(host_out[:])
        got_d = out_dev.cpu().numpy()
        np.testing.assert_array_equal(got_h, got_d)
        assert abs(got_h[0] - want[0]) <= 1e-12 * abs(want[0])
        # the net momentum of these flows is ~0: scale by mass * (bound on |u| = 0.1)
        assert np.abs(got_h[1:4] - want[1:4]).max() <= 1e-12 * abs(want[0]) * 0.1
        assert abs(got_h[4] - want[4]) <= 1e-12 * abs(want[4])
        # independent of the library: plain FP64 sums of the same populations on the host
        fh = f.cpu().numpy().reshape(s.q, -1)
        e = B.rmrtlb_lattice_info(B.LATTICE_NAMES[lattice])[2] * np.array(spacing)   # c_j = e_j dx / dt, dt = 1
        rho_n = fh.sum(0)
        j_n = e.T @ fh
        ref = np.array([rho_n.sum(), *j_n.sum(1), (0.5 * (j_n * j_n).sum(0) / rho_n).sum()])
        assert abs(got_h[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.abs(got_h[1:4] - ref[1:4]).max() <= 1e-12 * abs(ref[0]) * 0.1
        assert abs(got_h[4] - ref[4]) <= 1e-12 * abs(ref[4])
        results.append(got_h)
    assert not np.array_equal(results[0][4], results[1][4])   # the state moved on between the calls


def test_noalloc_rejects_oversize_and_host_input():
    import torch

    from paper_2206_00366_gb300 import build
    build.build()
    from paper_2206_00366_gb300 import rmrtlb as B
    f = torch.zeros(9 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RmrtlbError) as ei:
        B.rmrtlb_population_totals_noalloc(B.D2Q9, 16384, 4097, 1, 1.0, 1.0, 1.0, 1.0, f.data_ptr(),
                                           out.data_ptr(), 0)
    assert ei.value.status == B.ETOOBIG
    host = np.zeros(9 * 4)
    with pytest.raises(B.RmrtlbError) as ei:
        B.rmrtlb_population_totals_noalloc(B.D2Q9, 2, 2, 1, 1.0, 1.0, 1.0, 1.0, host.ctypes.data,
                                           out.data_ptr(), 0)
    assert ei.value.status == B.EINVAL
    with pytest.raises(B.RmrtlbError) as ei:                 # axis-only lattices are not accepted
        B.rmrtlb_population_totals_noalloc(B.D2Q5, 2, 2, 1, 1.0, 1.0, 1.0, 1.0, f.data_ptr(), out.data_ptr(), 0)
    assert ei.value.status == B.EINVAL


@pytest.mark.skipif("__import__('torch').cuda.device_count() < 2")
def test_noalloc_rejects_memory_of_another_gpu():
    """Populations on a GPU other than the current one are refused before
    any launch (checked on the host from the pointer's attributes)."""
    import torch

    from paper_2206_00366_gb300 import build
    build.build()
    from paper_2206_00366_gb300 import rmrtlb as B
    f1 = torch.zeros(9 * 4, dtype=torch.float64, device="cuda:1")
    out0 = torch.zeros(5, dtype=torch.float64, device="cuda:0")
    torch.cuda.set_device(0)
    with pytest.raises(B.RmrtlbError) as ei:
        B.rmrtlb_population_totals_noalloc(B.D2Q9, 2, 2, 1, 1.0, 1.0, 1.0, 1.0, f1.data_ptr(), out0.data_ptr(), 0)
    assert ei.value.status == B.EINVAL
