"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every declared symbol, and its host parameter derivation
(weights of Sec. III, rates of Eq. 4-31, the S_2 block of Eq. 5-8-1, the
NCDE S_1 of Eq. 4-10) agrees with the oracle.  rmrtlb_create touches no GPU,
so a placeholder workspace address is enough here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle.rmrt as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2206_00366_gb300 import build
    build.build()
    from paper_2206_00366_gb300 import rmrtlb
    return rmrtlb


def test_header_symbols_exported(B):
    inc = os.path.join(ROOT, "include")
    hdr = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    declared = set(re.findall(r"^\s*(?:const char\*|int|size_t)\s+(rmrtlb_\w+)\s*\(", hdr, re.M))
    assert declared == set(B.exported_symbols())
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_lattice_info_matches_paper_order(B):
    for name, code in B.LATTICE_NAMES.items():
        q, d, e = B.rmrtlb_lattice_info(code)
        eo = R.velocity_indices(name)
        assert (q, d) == eo.shape
        assert (e[:, :d] == eo).all()
        if d == 2:
            assert (e[:, 2] == 0).all()
    with pytest.raises(B.RmrtlbError):
        B.rmrtlb_lattice_info(7)


def test_strerror(B):
    for st in (0, -1, -2, -3, -4, -99):
        assert isinstance(B.rmrtlb_strerror(st), str) and B.rmrtlb_strerror(st)


def test_workspace_bytes(B):
    n = B.rmrtlb_workspace_bytes(B.D3Q19, 256, 256, 128, B.ST_F32)
    assert n >= 2 * 19 * 256 * 256 * 128 * 4
    assert B.rmrtlb_workspace_bytes(B.D3Q19, 256, 256, 128, B.ST_F16) < n
    for bad in [(B.D2Q9, 0, 4, 1), (B.D2Q9, 4, 4, 2), (B.D3Q27, 4, -1, 4), (5, 4, 4, 4)]:
        with pytest.raises(B.RmrtlbError):
            B.rmrtlb_workspace_bytes(*bad, B.ST_F32)


def create(B, lat, shape, spacing, kind=0, **kw):
    p = B.make_params(**kw)
    nbytes = B.rmrtlb_workspace_bytes(lat, *shape, B.ST_F32)
    return B.rmrtlb_create(lat, *shape, *spacing, 1.0, p, kind, 0, B.ST_F32, 256, nbytes, 0)


@pytest.mark.parametrize("name", R.LATTICES)
def test_constants_match_oracle(B, name):
    spacing = (1.0, 0.7, 0.5)
    shape = (8, 8, 1 if name == "D2Q9" else 8)
    nu, nub, sf = 0.013, 0.06, 1.15
    h = create(B, B.LATTICE_NAMES[name], shape, spacing, nu=nu, nu_bulk=nub, s_free=sf, rho0=1.0)
    c = B.rmrtlb_get_constants(h)
    B.rmrtlb_destroy(h)
    lat = R.make_lattice(name, spacing)
    r = R.rates_from_viscosity(lat, nu, nub, sf)
    d = lat.d
    assert abs(c[0] - lat.cs2) < 1e-15
    np.testing.assert_allclose(c[1:1 + d], lat.c, rtol=1e-15)
    np.testing.assert_allclose(c[4:4 + lat.q], lat.w, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(c[35:44].reshape(3, 3)[:d, :d], R.s2_diag_block(lat, r), rtol=1e-12)
    np.testing.assert_allclose(c[44], r.s_off[0, 1], rtol=1e-14)
    assert c[47] == sf


def test_ncde_constants(B):
    lat = R.make_lattice("D2Q9", (1.0, 0.6))
    D = 0.005
    h = create(B, B.D2Q9, (16, 8, 1), (1.0, 0.6, 1.0), kind=B.EQ_NCDE_QUAD, diffusivity=D, s_free=1.1,
               adv=(0.05, 0.02, 0.0))
    c = B.rmrtlb_get_constants(h)
    B.rmrtlb_destroy(h)
    tau = D / lat.cs2 + 0.5
    np.testing.assert_allclose(c[32:34], 1 / tau, rtol=1e-14)
    # K = dt c_s^2 (1/s_1 - 1/2) recovers D (Eq. 4-10)
    np.testing.assert_allclose(lat.cs2 * (1 / c[32] - 0.5), D, rtol=1e-13)


def test_create_rejects_invalid(B):
    ok = dict(nu=0.01, nu_bulk=0.05, s_free=1.1, rho0=1.0)
    with pytest.raises(B.RmrtlbError):      # c_s^2 above min c^2
        create(B, B.D2Q9, (8, 8, 1), (1.0, 0.5, 1.0), cs2=0.3, **{k: v for k, v in ok.items()})
    with pytest.raises(B.RmrtlbError):      # negative weight on rD3Q19
        create(B, B.D3Q19, (8, 8, 8), (1.0, 1.0, 0.5), cs2=0.22, **ok)
    with pytest.raises(B.RmrtlbError):      # rate outside (0, 2)
        create(B, B.D2Q9, (8, 8, 1), (1.0, 1.0, 1.0), nu=0.01, nu_bulk=0.05, s_free=2.5, rho0=1.0)
    with pytest.raises(B.RmrtlbError):      # unaligned workspace
        p = B.make_params(**ok)
        B.rmrtlb_create(B.D2Q9, 8, 8, 1, 1.0, 1.0, 1.0, 1.0, p, 0, 0, B.ST_F32, 257, 1 << 30, 0)
    with pytest.raises(B.RmrtlbError) as ei:   # workspace too small
        p = B.make_params(**ok)
        B.rmrtlb_create(B.D2Q9, 8, 8, 1, 1.0, 1.0, 1.0, 1.0, p, 0, 0, B.ST_F32, 256, 16, 0)
    assert ei.value.status == B.ENOMEM
    for storage, rng in [(5, 0.0), (B.ST_E3M12, 1000.0), (B.ST_E3M12, 1e-9)]:   # unknown storage; E3M12 range
        p = B.make_params(storage_range=rng, **ok)
        nbytes = B.rmrtlb_workspace_bytes(B.D2Q9, 8, 8, 1, B.ST_F32)
        with pytest.raises(B.RmrtlbError) as ei:
            B.rmrtlb_create(B.D2Q9, 8, 8, 1, 1.0, 1.0, 1.0, 1.0, p, 0, 0, storage, 256, nbytes, 0)
        assert ei.value.status == B.EINVAL


def test_e3m12_workspace_and_range_accepted(B):
    """E3M12 stores 2 bytes per population like FP16; ranges from 2^-20 to
    128 are accepted (checked on the host, no kernel runs)."""
    assert B.rmrtlb_workspace_bytes(B.D3Q27, 64, 64, 32, B.ST_E3M12) == \
        B.rmrtlb_workspace_bytes(B.D3Q27, 64, 64, 32, B.ST_F16)
    for rng in (0.0, 2.0 ** -20, 0.3, 8.0, 128.0):
        p = B.make_params(nu=0.01, nu_bulk=0.05, s_free=1.1, rho0=1.0, storage_range=rng)
        nbytes = B.rmrtlb_workspace_bytes(B.D2Q9, 8, 8, 1, B.ST_E3M12)
        h = B.rmrtlb_create(B.D2Q9, 8, 8, 1, 1.0, 1.0, 1.0, 1.0, p, 0, 0, B.ST_E3M12, 256, nbytes, 0)
        B.rmrtlb_destroy(h)


def test_bgk_limit_constants(B):
    """Standard lattice, c_s^2 = 1/3 and equal rates: the S_2 block is s I."""
    s = 1.3
    nu = (1 / s - 0.5) / 3
    nub = (1 / 2) * (1 / s - 0.5) * (1 - 1 / 3)
    h = create(B, B.D2Q9, (8, 8, 1), (1.0, 1.0, 1.0), nu=nu, nu_bulk=nub, s_free=s, cs2=1 / 3, rho0=1.0)
    c = B.rmrtlb_get_constants(h)
    B.rmrtlb_destroy(h)
    np.testing.assert_allclose(c[35:44].reshape(3, 3)[:2, :2], s * np.eye(2), atol=1e-14)


def test_convolution_scratch_bytes(B):
    """Scratch of the weight gradient: FP32 partial sums of dweight per
    4096-voxel chunk or per 32 boxes of 128 voxels (whichever are more),
    of dbias per 1024 voxels, and on a plane that holds a box a 16-byte
    aligned BF16 copy of dy (4 output channels padded to 8); the input gradient's
    scratch is that copy alone (4 output channels: padded to 8)."""
    ceil = lambda a, b: -(-a // b)
    # 5 x 6 planes hold no 128-voxel box: the threads gather, no dy copy
    n, d, h, w = 2, 5, 6, 13
    v = n * d * h * w
    for cin, cout in ((8, 32), (32, 32), (32, 4)):
        assert B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout) == \
            4 * (ceil(v, 4096) * 27 * cin * cout + ceil(v, 1024) * cout)
        assert B.rmrtlb_conv3d_backward_data_scratch(n, d, h, w, cin, cout) == 0
    # 64 x 64 planes: 64 x 2 boxes, 4 * 32 * 32 boxes in 128 chunks of 32
    n, d, h, w = 4, 32, 64, 64
    v = n * d * h * w
    for cin in (8, 32):
        parts = 4 * (max(ceil(v, 4096), 128) * 27 * cin * 32 + ceil(v, 1024) * 32)
        assert B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, 32) == ceil(parts, 16) * 16 + v * 64
    parts = 4 * (max(ceil(v, 4096), 128) * 27 * 32 * 4 + ceil(v, 1024) * 4)
    assert B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, 32, 4) == ceil(parts, 16) * 16 + v * 16
    assert B.rmrtlb_conv3d_backward_data_scratch(n, d, h, w, 32, 32) == v * 64
    assert B.rmrtlb_conv3d_backward_data_scratch(n, d, h, w, 32, 4) == v * 16
    assert B.rmrtlb_conv3d_backward_weight_scratch(0, d, h, w, 32, 32) == 0


def test_state_bytes(B):
    """The checkpoint blob of a new solver: a header, the population codes as
    stored (q N elements of the storage), the simplified NCDE's B(t - dt)
    planes (d N of the compute type, that kind only), the check's sums and
    flag word, each section rounded up to 16 bytes; no residual snapshot
    before a check.  NULL buffers are rejected before any copy (host only)."""
    import ctypes
    ok = dict(nu=0.01, nu_bulk=0.05, s_free=1.1, rho0=1.0, diffusivity=0.02)
    r16 = lambda n: -(-n // 16) * 16
    sizes = []
    for lat, st, kind, esize, ct in [(B.D2Q9, B.ST_F32, 0, 4, 4), (B.D3Q27, B.ST_F16, 0, 2, 4),
                                     (B.D2Q9, B.ST_F64, 0, 8, 8), (B.D2Q5, B.ST_F32, B.EQ_NAMES["ncde_simple_linear"],
                                                                   4, 4)]:
        nx, ny, nz = (12, 10, 1) if lat in (B.D2Q9, B.D2Q5) else (8, 6, 4)
        spacing = (1.0, 0.7, 1.0) if nz == 1 else (1.0, 0.7, 0.5)
        q, d, _ = B.rmrtlb_lattice_info(lat)
        p = B.make_params(**ok)
        nbytes = B.rmrtlb_workspace_bytes(lat, nx, ny, nz, st)
        h = B.rmrtlb_create(lat, nx, ny, nz, *spacing, 1.0, p, kind, 0, st, 256, nbytes, 0)
        try:
            n = nx * ny * nz
            hist = d * n * ct if kind == B.EQ_NAMES["ncde_simple_linear"] else 0
            body = r16(q * n * esize) + r16(hist) + 64 + 16
            total = B.rmrtlb_state_bytes(h)
            sizes.append(total - body)                      # the header, the same for every solver
            assert total > body
            for fn in (lib_call(B, "rmrtlb_save_state"), lib_call(B, "rmrtlb_load_state")):
                assert fn(h, None, total) == B.EINVAL
        finally:
            B.rmrtlb_destroy(h)
    assert len(set(sizes)) == 1 and sizes[0] % 16 == 0


def lib_call(B, name):
    return getattr(B.lib(), name)
