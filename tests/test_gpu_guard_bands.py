"""Write-once canaries around every buffer the library writes: the solver and
batch workspaces and the convolution outputs sit inside a larger device
allocation whose guard bands hold a byte pattern; after initialisation,
steps (with periodic checks), read-back and the auxiliary outputs, the guard
bands must be unchanged.  This catches an out-of-bounds store of any kernel
(the one-, two- and four-nodes-per-thread step kernels, the check and stress
kernels, the batch kernels, the tensor-core convolutions) without a
sanitizer and without faulting a GPU: the stray write lands in memory this
test owns."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 1 << 20          # bytes on each side (a multiple of 256: the interior stays aligned)
CANARY = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_2206_00366_gb300 import build
    build.build()


def guarded(nbytes):
    """(backing tensor, device pointer of the interior) with canary bands."""
    import torch
    t = torch.full((2 * GUARD + nbytes,), CANARY, dtype=torch.uint8, device="cuda")
    return t, t.data_ptr() + GUARD


def assert_bands(t, nbytes):
    import torch
    torch.cuda.synchronize()
    lo = t[:GUARD].cpu().numpy()
    hi = t[GUARD + nbytes:].cpu().numpy()
    assert (lo == CANARY).all(), f"write below the buffer at offset {np.flatnonzero(lo != CANARY)[-1] - GUARD}"
    assert (hi == CANARY).all(), f"write past the buffer at offset {np.flatnonzero(hi != CANARY)[0]}"


SOLVER_CASES = [
    ("D2Q9", (37, 23, 1)), ("D2Q9", (70, 23, 1)), ("D2Q9", (72, 23, 1)), ("D2Q9", (4, 3, 1)),
    ("D3Q19", (13, 11, 7)), ("D3Q19", (16, 11, 7)), ("D3Q27", (14, 11, 7)), ("D3Q27", (16, 11, 7)),
]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("lattice,shape", SOLVER_CASES)
def test_solver_writes_stay_in_its_buffers(lattice, shape, basis, storage):
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    lat, st = B.LATTICE_NAMES[lattice], B.STORAGE_NAMES[storage]
    nx, ny, nz = shape
    q, d, _ = B.rmrtlb_lattice_info(lat)
    n = nx * ny * nz
    nbytes = B.rmrtlb_workspace_bytes(lat, nx, ny, nz, st)
    ws, wp = guarded(nbytes)
    p = B.make_params(nu=0.02, nu_bulk=0.03, s_free=1.1, check_every=2, force=(1e-5, -2e-5, 1e-5))
    h = B.rmrtlb_create(lat, nx, ny, nz, 1.0, 0.7, 0.55, 1.0, p, 0, basis, st, wp, nbytes,
                        torch.cuda.current_stream().cuda_stream)
    try:
        rho, u = W.random_fields((nz, ny, nx), d, seed=3, umax=0.03)
        # device outputs, each guarded too
        rho_t, rho_p = guarded(n * 8)
        u_t, u_p = guarded(d * n * 8)
        f_t, f_p = guarded(q * n * 8)
        ns = d * (d + 1) // 2
        s_t, s_p = guarded(ns * n * 8)
        r_t, r_p = guarded(ns * n * 8)
        B.rmrtlb_init_equilibrium(h, rho.ctypes.data, u.ctypes.data)
        B.rmrtlb_step(h, 5)
        B.rmrtlb_stats(h)
        B.rmrtlb_moments(h, rho_p, u_p)
        B.rmrtlb_get_populations(h, f_p)
        B.rmrtlb_stress(h, s_p, r_p)
        B.rmrtlb_set_populations(h, f_p)
        B.rmrtlb_step(h, 1)
        torch.cuda.synchronize()
        for t, nb in [(ws, nbytes), (rho_t, n * 8), (u_t, d * n * 8), (f_t, q * n * 8), (s_t, ns * n * 8),
                      (r_t, ns * n * 8)]:
            assert_bands(t, nb)
    finally:
        B.rmrtlb_destroy(h)


@pytest.mark.parametrize("per_thread", [1, 2])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q27"])
def test_batch_writes_stay_in_its_workspace(lattice, per_thread):
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    lat = B.LATTICE_NAMES[lattice]
    if lattice == "D2Q9":
        doms = W.cavity_domains(12, seed=9, size=(8, 40))
    else:
        doms = [dict(nx=9, ny=6, nz=5, dx=1.0, dy=1.0, dz=0.5, nu=0.05, nu_bulk=0.05, s_free=1.1, lid_u=0.05),
                dict(nx=4, ny=7, nz=3, dx=1.0, dy=2.0, dz=1.0, nu=0.1, nu_bulk=0.1, s_free=1.0, lid_u=0.03)]
    doms = [dict(B._DOMAIN_DEFAULTS, **dd) for dd in doms]
    st = B.STORAGE_NAMES["f32"]
    nbytes = B.rmrtlb_batch_workspace_bytes(lat, doms, st)
    ws, wp = guarded(nbytes)
    stream = torch.cuda.Stream()
    h = B.rmrtlb_batch_create(lat, 0, doms, st, 1.0, 4, 1e-9, wp, nbytes, stream.cuda_stream)
    try:
        B.rmrtlb_batch_set_launch(h, 32, 2, per_thread)
        B.rmrtlb_batch_step(h, 9)
        B.rmrtlb_batch_status(h, len(doms))
        dd = doms[0]
        nn = dd["nx"] * dd["ny"] * dd["nz"]
        q, d, _ = B.rmrtlb_lattice_info(lat)
        f_t, f_p = guarded(q * nn * 8)
        B.rmrtlb_batch_get_populations(h, 0, f_p)
        rho_t, rho_p = guarded(nn * 8)
        u_t, u_p = guarded(d * nn * 8)
        B.rmrtlb_batch_fields(h, 0, rho_p, u_p)
        B.rmrtlb_batch_set_populations(h, 0, f_p)
        B.rmrtlb_batch_run(h, 16)
        torch.cuda.synchronize()
        for t, nb in [(ws, nbytes), (f_t, q * nn * 8), (rho_t, nn * 8), (u_t, d * nn * 8)]:
            assert_bands(t, nb)
    finally:
        B.rmrtlb_batch_destroy(h)


@pytest.mark.parametrize("cin,cout", [(8, 32), (32, 32), (32, 4)])
def test_convolution_writes_stay_in_their_outputs(cin, cout):
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = 1, 5, 6, 13                     # 390 voxels: a ragged last tile
    v = n * d * h * w
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.normal(size=(v, cin)), dtype=torch.bfloat16, device="cuda")
    wt = torch.tensor(rng.normal(scale=0.2, size=(27, cin, cout)), dtype=torch.bfloat16, device="cuda")
    bias = torch.zeros(cout, dtype=torch.float32, device="cuda")
    z_t, z_p = guarded(v * cout * 4)
    a_t, a_p = guarded(v * cout * 2)
    B.rmrtlb_conv3d_forward(n, d, h, w, cin, cout, x.data_ptr(), wt.data_ptr(), bias.data_ptr(), 1, z_p, a_p)
    B.rmrtlb_cnn_check()
    assert_bands(z_t, v * cout * 4)
    assert_bands(a_t, v * cout * 2)
    if cin == 32:
        dy = torch.tensor(rng.normal(size=(v, cout)), dtype=torch.float32, device="cuda")
        dx_t, dx_p = guarded(v * cin * 4)
        B.rmrtlb_conv3d_backward_data(n, d, h, w, cin, cout, dy.data_ptr(), wt.data_ptr(), 0, dx_p)
        B.rmrtlb_cnn_check()
        assert_bands(dx_t, v * cin * 4)
    # the copy-fed kernels (a plane that holds 16 x 8 boxes), output and dy scratch guarded
    n2, d2, h2, w2 = 1, 3, 9, 20
    v2 = n2 * d2 * h2 * w2
    x2 = torch.tensor(rng.normal(size=(v2, cin)), dtype=torch.bfloat16, device="cuda")
    z2_t, z2_p = guarded(v2 * cout * 4)
    a2_t, a2_p = guarded(v2 * cout * 2)
    B.rmrtlb_conv3d_forward(n2, d2, h2, w2, cin, cout, x2.data_ptr(), wt.data_ptr(), bias.data_ptr(), 1, z2_p, a2_p)
    B.rmrtlb_cnn_check()
    assert_bands(z2_t, v2 * cout * 4)
    assert_bands(a2_t, v2 * cout * 2)
    if cin == 32:
        dy2 = torch.tensor(rng.normal(size=(v2, cout)), dtype=torch.float32, device="cuda")
        sd = B.rmrtlb_conv3d_backward_data_scratch(n2, d2, h2, w2, cin, cout)
        sd_t, sd_p = guarded(max(sd, 16))
        dx2_t, dx2_p = guarded(v2 * cin * 4)
        B.rmrtlb_conv3d_backward_data(n2, d2, h2, w2, cin, cout, dy2.data_ptr(), wt.data_ptr(), 0, dx2_p, sd_p, sd)
        B.rmrtlb_cnn_check()
        assert_bands(sd_t, max(sd, 16))
        assert_bands(dx2_t, v2 * cin * 4)
    # the copy-fed weight gradient: partials, bias partials and dy's BF16 copy inside the scratch
    dy2 = torch.tensor(rng.normal(size=(v2, cout)), dtype=torch.float32, device="cuda")
    sw = B.rmrtlb_conv3d_backward_weight_scratch(n2, d2, h2, w2, cin, cout)
    sw_t, sw_p = guarded(sw)
    dw2_t, dw2_p = guarded(27 * cin * cout * 4)
    db2_t, db2_p = guarded(cout * 4)
    B.rmrtlb_conv3d_backward_weight(n2, d2, h2, w2, cin, cout, x2.data_ptr(), dy2.data_ptr(), dw2_p, db2_p,
                                    sw_p, sw)
    B.rmrtlb_cnn_check()
    for t, nb in [(sw_t, sw), (dw2_t, 27 * cin * cout * 4), (db2_t, cout * 4)]:
        assert_bands(t, nb)
    dy = torch.tensor(rng.normal(size=(v, cout)), dtype=torch.float32, device="cuda")
    sb = B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout)
    sc_t, sc_p = guarded(sb)
    dw_t, dw_p = guarded(27 * cin * cout * 4)
    db_t, db_p = guarded(cout * 4)
    B.rmrtlb_conv3d_backward_weight(n, d, h, w, cin, cout, x.data_ptr(), dy.data_ptr(), dw_p, db_p, sc_p, sb)
    B.rmrtlb_cnn_check()
    for t, nb in [(sc_t, sb), (dw_t, 27 * cin * cout * 4), (db_t, cout * 4)]:
        assert_bands(t, nb)
