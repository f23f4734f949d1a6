"""Warm-start network kernels (rmrtlb_cnn.h) against the FP64 oracle of
oracle/cnn.py on the same BF16-rounded inputs (the tensor-core kernels take
BF16 operands: x, w, and dy rounded to nearest even).  Tolerances: FP32
accumulation of up to 864 products, normwise 1e-5; BF16 outputs within one
BF16 rounding (2^-8 relative) of the oracle; encodings bit-exact."""
import numpy as np
import pytest

import oracle.cnn as C
from cases import normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_2206_00366_gb300 import build
    build.build()


def dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def bf16(a):
    """(BF16 device tensor, its exact FP64 values)."""
    import torch
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()


def host(t):
    import torch
    return t.to(torch.float64).cpu().numpy()


PAIRS = [(8, 32), (32, 32), (32, 4)]
SHAPE = (2, 5, 6, 13)   # 780 voxels: several 128-voxel blocks and a ragged tail
# Planes large enough for the copy-fed kernels (boxes of 16 x 8, 64 x 2,
# 8 x 16 and 128 x 1 voxels; ragged in x, in y and in both).
TMA_SHAPES = [(2, 3, 9, 20), (1, 2, 16, 64), (1, 1, 130, 8), (1, 2, 3, 200)]


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("silu", [True, False])
def test_conv_forward(cin, cout, silu):
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = SHAPE
    rng = np.random.default_rng(cin + cout)
    xg, x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wg, wv = bf16(rng.normal(scale=0.2, size=(27, cin, cout)))
    b = rng.normal(size=cout).astype(np.float32)
    z = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    a = torch.empty((n, d, h, w, cout), dtype=torch.bfloat16, device="cuda")
    bt = dev(b, torch.float32)
    B.rmrtlb_conv3d_forward(n, d, h, w, cin, cout, xg.data_ptr(), wg.data_ptr(), bt.data_ptr(),
                            silu, z.data_ptr(), a.data_ptr())
    B.rmrtlb_cnn_check()
    zo = C.conv3d(x, wv, b.astype(np.float64))
    assert normwise(host(z), zo) <= 1e-5
    ao = C.silu(zo) if silu else zo
    assert np.abs(host(a) - ao).max() <= 2.0 ** -7 * np.abs(ao).max()


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("silu", [True, False])
def test_conv_forward_copy_fed(shape, cin, cout, silu):
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = shape
    rng = np.random.default_rng(cin + 3 * cout + h)
    xg, x = bf16(rng.normal(size=(n, d, h, w, cin)))
    wg, wv = bf16(rng.normal(scale=0.2, size=(27, cin, cout)))
    b = rng.normal(size=cout).astype(np.float32)
    z = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    a = torch.empty((n, d, h, w, cout), dtype=torch.bfloat16, device="cuda")
    bt = dev(b, torch.float32)
    B.rmrtlb_conv3d_forward(n, d, h, w, cin, cout, xg.data_ptr(), wg.data_ptr(), bt.data_ptr(),
                            silu, z.data_ptr(), a.data_ptr())
    B.rmrtlb_cnn_check()
    zo = C.conv3d(x, wv, b.astype(np.float64))
    assert normwise(host(z), zo) <= 1e-5
    ao = C.silu(zo) if silu else zo
    assert np.abs(host(a) - ao).max() <= 2.0 ** -7 * np.abs(ao).max()


def test_bounded_wait_gives_up_and_reports_timeout():
    """Failure detection without a GPU fault: an mbarrier that nothing
    arrives on, waited for with the convolutions' bounded polling, gives up
    after 1000 polls; rmrtlb_cnn_check reports RMRTLB_ETIMEOUT once, and the
    context stays usable (a convolution afterwards matches the oracle)."""
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    B.rmrtlb_cnn_check()
    B.rmrtlb_cnn_wait_selftest(1000)
    with pytest.raises(B.RmrtlbError) as e:
        B.rmrtlb_cnn_check()
    assert e.value.status == B.ETIMEOUT
    B.rmrtlb_cnn_check()                     # the condition was cleared
    with pytest.raises(B.RmrtlbError) as e:
        B.rmrtlb_cnn_wait_selftest(0)
    assert e.value.status == B.EINVAL
    n, d, h, w = SHAPE
    rng = np.random.default_rng(5)
    xg, x = bf16(rng.normal(size=(n, d, h, w, 32)))
    wg, wv = bf16(rng.normal(scale=0.2, size=(27, 32, 32)))
    b = np.zeros(32, dtype=np.float32)
    z = torch.empty((n, d, h, w, 32), dtype=torch.float32, device="cuda")
    bt = dev(b, torch.float32)
    B.rmrtlb_conv3d_forward(n, d, h, w, 32, 32, xg.data_ptr(), wg.data_ptr(), bt.data_ptr(), 0, z.data_ptr(), 0)
    B.rmrtlb_cnn_check()
    assert normwise(host(z), C.conv3d(x, wv, b.astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 4)])
@pytest.mark.parametrize("with_z", [True, False])
@pytest.mark.parametrize("shape,use_scratch", [(SHAPE, False), (SHAPE, True)] + [(s, True) for s in TMA_SHAPES]
                         + [(TMA_SHAPES[0], False)])
def test_conv_backward_data(cin, cout, with_z, shape, use_scratch):
    """Thread-gathering kernel (no scratch, or a plane too small for a box)
    and, with a scratch for the BF16 copy of dy (4 channels padded to 8),
    the copy-fed kernel with mirrored taps."""
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = shape
    rng = np.random.default_rng(7 + cout + h)
    dy = rng.normal(size=(n, d, h, w, cout)).astype(np.float32)
    zin = rng.normal(size=(n, d, h, w, cin)).astype(np.float32)
    wg, wv = bf16(rng.normal(scale=0.2, size=(27, cin, cout)))
    dx = torch.empty((n, d, h, w, cin), dtype=torch.float32, device="cuda")
    zt = dev(zin, torch.float32)
    dyt = dev(dy, torch.float32)
    sb = B.rmrtlb_conv3d_backward_data_scratch(n, d, h, w, cin, cout) if use_scratch else 0
    assert (sb > 0) == (use_scratch and shape != SHAPE)
    sc = torch.empty(max(sb, 16), dtype=torch.uint8, device="cuda")
    B.rmrtlb_conv3d_backward_data(n, d, h, w, cin, cout, dyt.data_ptr(), wg.data_ptr(),
                                  zt.data_ptr() if with_z else None, dx.data_ptr(),
                                  sc.data_ptr() if use_scratch else None, sb)
    B.rmrtlb_cnn_check()
    dyb = torch.tensor(dy).to(torch.bfloat16).to(torch.float64).numpy()   # the tensor cores take BF16
    ref = C.conv3d_backward_data(dyb, wv)
    if with_z:
        ref = ref * C.silu_grad(zin.astype(np.float64))
    assert normwise(host(dx), ref) <= 1e-5


@pytest.mark.parametrize("shape", [(2, 8, 16, 40)] + TMA_SHAPES + [SHAPE])
@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_backward_weight(cin, cout, shape):
    """(2, 8, 16, 40) spans three 4096-voxel partial-sum chunks of the
    gathering kernel (4 output channels) and three 32-box chunks of the
    copy-fed one (8 x 16 boxes, the last chunk ragged); the other planes
    take every box shape the copy-fed kernel picks, ragged in x, y or both,
    and SHAPE a plane too small for a box.  Repeated calls are bitwise
    equal."""
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = shape
    rng = np.random.default_rng(11 + cin)
    xg, x = bf16(rng.normal(size=(n, d, h, w, cin)))
    dy = rng.normal(size=(n, d, h, w, cout)).astype(np.float32)
    sb = B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, cin, cout)
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    dyt = dev(dy, torch.float32)
    outs = []
    for _ in range(2):
        dw = torch.empty((27, cin, cout), dtype=torch.float32, device="cuda")
        db = torch.empty(cout, dtype=torch.float32, device="cuda")
        B.rmrtlb_conv3d_backward_weight(n, d, h, w, cin, cout, xg.data_ptr(), dyt.data_ptr(), dw.data_ptr(),
                                        db.data_ptr(), scratch.data_ptr(), sb)
        torch.cuda.synchronize()
        outs.append((host(dw), host(db)))
    dyb = torch.tensor(dy).to(torch.bfloat16).to(torch.float64).numpy()   # the tensor cores take BF16
    dwo, _ = C.conv3d_backward_weight(x, dyb)
    _, dbo = C.conv3d_backward_weight(x, dy.astype(np.float64))        # the bias sum stays FP32
    assert normwise(outs[0][0], dwo) <= 1e-5
    assert normwise(outs[0][1], dbo) <= 1e-5
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_mse():
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    count = 300_007
    rng = np.random.default_rng(5)
    y = rng.normal(size=count).astype(np.float32)
    t = rng.normal(size=count).astype(np.float32)
    dy = torch.empty(count, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    scratch = torch.empty(8192, dtype=torch.uint8, device="cuda")
    yt, tt = dev(y, torch.float32), dev(t, torch.float32)
    B.rmrtlb_mse(count, yt.data_ptr(), tt.data_ptr(), dy.data_ptr(), loss.data_ptr(), scratch.data_ptr())
    lo, go = C.mse(y.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - lo) <= 1e-6 * lo
    assert normwise(host(dy), go) <= 1e-6


def test_adam_steps_and_bf16_copy():
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n = 5000
    rng = np.random.default_rng(9)
    p = rng.normal(size=n)
    pt = dev(p, torch.float32)
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    po, mo, vo = p.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        gt = dev(g, torch.float32)
        B.rmrtlb_adam(n, pt.data_ptr(), pb.data_ptr(), gt.data_ptr(), m.data_ptr(), v.data_ptr(), step, 1e-2)
        torch.cuda.synchronize()
        po, mo, vo = C.adam_step(po, g.astype(np.float64), mo, vo, step, 1e-2)
    torch.cuda.synchronize()
    assert np.abs(host(pt) - po).max() <= 1e-6
    np.testing.assert_array_equal(host(pb), host(pt.to(torch.bfloat16)))


def test_cavity_features_bit_exact():
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n, d, h, w = 3, 4, 5, 6
    re = np.array([100.0, 777.7, 1500.0])
    x = torch.empty((n, d, h, w, 8), dtype=torch.bfloat16, device="cuda")
    ret = dev(re, torch.float64)
    B.rmrtlb_cavity_features(n, d, h, w, ret.data_ptr(), x.data_ptr())
    ref = np.stack([C.cavity_features((d, h, w), r) for r in re])
    expect = torch.tensor(ref).to(torch.float32).to(torch.bfloat16)
    assert torch.equal(x.cpu(), expect)


def test_upsample_fields():
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    d, h, w, c = 4, 6, 5, 4
    D, H, W = 12, 18, 15
    src = np.random.default_rng(2).normal(size=(d, h, w, c)).astype(np.float32)
    scale, offset = [2.0, 0.5, -1.0, 3.0], [1.0, 0.0, 0.25, 0.0]
    dst = torch.empty((c, D, H, W), dtype=torch.float64, device="cuda")
    st = dev(src, torch.float32)
    B.rmrtlb_upsample_fields(d, h, w, c, st.data_ptr(), D, H, W, scale, offset, dst.data_ptr())
    ref = C.upsample_trilinear(src.astype(np.float64), (D, H, W))
    ref = np.moveaxis(ref, -1, 0) * np.array(scale)[:, None, None, None] + np.array(offset)[:, None, None, None]
    assert normwise(dst.cpu().numpy(), ref) <= 1e-13


def test_pack_fields():
    import torch
    from paper_2206_00366_gb300 import rmrtlb as B
    n = 1001
    rng = np.random.default_rng(4)
    rho = 1.0 + 0.01 * rng.normal(size=n)
    u = 0.05 * rng.normal(size=(3, n))
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    rt, ut = dev(rho, torch.float64), dev(u, torch.float64)
    B.rmrtlb_pack_fields(n, 3, rt.data_ptr(), ut.data_ptr(), 1.0, 33.0, 20.0, out.data_ptr())
    ref = np.stack([(rho - 1.0) * 33.0, u[0] * 20.0, u[1] * 20.0, u[2] * 20.0], axis=1)
    np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))


def test_network_training_step_matches_oracle():
    """One full forward, MSE, backward and Adam step of the 4-layer network
    through the C ABI: loss and every updated parameter agree with the
    oracle network on the same BF16 weights and inputs."""
    import torch
    from paper_2206_00366_gb300.warmstart import CH, Net
    net = Net(seed=3)
    shape = (4, 6, 10)
    re = [250.0, 1200.0]
    rng = np.random.default_rng(1)
    t = rng.normal(scale=0.5, size=(2,) + shape + (4,)).astype(np.float32)
    tt = dev(t, torch.float32)
    flat16 = net.bf16.to(torch.float64).cpu().numpy()
    flat32 = net.master.cpu().numpy().astype(np.float64)
    ws = [flat16[net.off[2 * k]:net.off[2 * k + 1]].reshape(27, CH[k], CH[k + 1]) for k in range(4)]
    bs = [flat32[net.off[2 * k + 1]:net.off[2 * k + 2]] for k in range(4)]
    loss = net.train_step(re, shape, tt, 1e-3).item()
    x = np.stack([C.cavity_features(shape, r) for r in re])
    x = torch.tensor(x).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    onet = C.Net(ws, bs)
    y, cache = onet.forward(x)
    lo, dy = C.mse(y, t.astype(np.float64))
    assert abs(loss - lo) <= 2e-2 * lo       # BF16 activations between layers
    dws, dbs = onet.backward(cache, dy)
    g = net.grad.cpu().numpy()
    for k in range(4):
        gk = g[net.off[2 * k]:net.off[2 * k + 1]].reshape(27, CH[k], CH[k + 1])
        assert normwise(gk, dws[k]) <= 5e-2, k


def test_training_learns_solver_states():
    """The learned path end to end on a small case: steady states of 12
    cavities (8 x 16 x 16 cells, Re 50..200) from the solver, a few hundred
    Adam steps through the C ABI; the loss falls and the prediction for a
    held-out Re is far closer to the solver's steady velocity than the rest
    state is."""
    import torch
    from paper_2206_00366_gb300 import warmstart as WS
    coarse = (8, 16, 16)
    res = np.linspace(50.0, 200.0, 12)
    T, steps, _ = WS.generate_states(res, shape=coarse, max_steps=60000)
    assert (steps > 0).all(), steps
    net = WS.Net(seed=0)
    losses, _ = WS.train(net, T, list(res), coarse, epochs=60, batch=4, lr=3e-3, lr_end=2e-4)
    assert losses[-1] < 0.2 * losses[0], losses
    Th, sh, _ = WS.generate_states([130.0], shape=coarse, max_steps=60000)
    y = net.forward([130.0], coarse).view(coarse + (4,))
    err = torch.linalg.vector_norm(y[..., 1:] - Th[0][..., 1:]) / torch.linalg.vector_norm(Th[0][..., 1:])
    assert float(err) < 0.2, float(err)


@pytest.mark.parametrize("re", [300.0, 1000.0])
def test_trained_warm_start_gains_over_cold_start(re):
    """The committed network (trained on solver steady states of
    64 x 64 x 32 cavities) warm-starts a 192 x 192 x 96 cavity at a low and
    a high Re of its range: the solver reaches residual 1e-6 in fewer steps
    than from rest, and both runs end in the same steady state."""
    import os
    from paper_2206_00366_gb300 import warmstart as WS
    if not os.path.exists(WS.WEIGHTS):
        pytest.skip("no trained weights committed")
    net = WS.Net.load(WS.WEIGHTS)
    dom = WS.cavity((96, 192, 192), re)
    cold = WS.time_to_steady(dom, re)
    warm = WS.time_to_steady(dom, re, net=net, coarse=tuple(net.meta["shape"]))
    assert cold["state"] == 0 and warm["state"] == 0, (cold, warm)
    assert warm["steps"] < cold["steps"], (warm["steps"], cold["steps"])
    assert normwise(warm["u"].cpu().numpy(), cold["u"].cpu().numpy()) < 2e-3
