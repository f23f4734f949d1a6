"""Pins of the warm-start network oracle (oracle/cnn.py) against what does
not depend on it: scipy's n-dimensional correlation, central finite
differences, the closed form of Adam's first step, and exactness of
trilinear interpolation on linear fields."""
import numpy as np
import pytest

import oracle.cnn as C


def rnd(*shape, seed=0):
    return np.random.default_rng(seed).normal(size=shape)


def test_conv3d_equals_scipy_correlate():
    """Each output channel is the sum over input channels of scipy's
    zero-padded 3-D correlation, plus the bias."""
    ndimage = pytest.importorskip("scipy.ndimage")
    x = rnd(2, 4, 5, 6, 3, seed=1)
    w = rnd(27, 3, 2, seed=2)
    b = rnd(2, seed=3)
    y = C.conv3d(x, w, b)
    for n in range(2):
        for co in range(2):
            ref = b[co] + sum(ndimage.correlate(x[n, ..., ci], w[:, ci, co].reshape(3, 3, 3), mode="constant",
                                                cval=0.0) for ci in range(3))
            np.testing.assert_allclose(y[n, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_gradients_match_finite_differences():
    """Input, weight and bias gradients of L = sum(r * conv3d(x, w, b)) equal
    central differences (the loss is linear in each argument, so the
    difference quotient is exact up to rounding)."""
    x = rnd(1, 3, 4, 3, 2, seed=4)
    w = rnd(27, 2, 3, seed=5)
    b = rnd(3, seed=6)
    r = rnd(1, 3, 4, 3, 3, seed=7)
    L = lambda x_, w_, b_: float((r * C.conv3d(x_, w_, b_)).sum())
    dx = C.conv3d_backward_data(r, w)
    dw, db = C.conv3d_backward_weight(x, r)
    h = 1e-3
    rng = np.random.default_rng(8)
    for _ in range(12):
        i = tuple(rng.integers(0, s) for s in x.shape)
        e = np.zeros_like(x); e[i] = h
        assert abs((L(x + e, w, b) - L(x - e, w, b)) / (2 * h) - dx[i]) < 1e-9
        k = tuple(rng.integers(0, s) for s in w.shape)
        e = np.zeros_like(w); e[k] = h
        assert abs((L(x, w + e, b) - L(x, w - e, b)) / (2 * h) - dw[k]) < 1e-9
    for c in range(3):
        e = np.zeros_like(b); e[c] = h
        assert abs((L(x, w, b + e) - L(x, w, b - e)) / (2 * h) - db[c]) < 1e-9


def test_network_gradient_matches_finite_differences():
    """Through the SiLU layers: the backward pass of the 4-layer network
    equals central differences of the mean squared error."""
    rng = np.random.default_rng(9)
    ch = [8, 4, 4, 4, 4]
    ws = [rng.normal(scale=0.3, size=(27, ch[k], ch[k + 1])) for k in range(4)]
    bs = [rng.normal(scale=0.1, size=ch[k + 1]) for k in range(4)]
    x = C.cavity_features((3, 4, 5), 500.0)[None]
    t = rng.normal(size=(1, 3, 4, 5, 4))
    net = C.Net(ws, bs)
    y, cache = net.forward(x)
    loss, dy = C.mse(y, t)
    dws, dbs = net.backward(cache, dy)

    def L(k, idx, h, bias=False):
        w2 = [w.copy() for w in ws]
        b2 = [b.copy() for b in bs]
        (b2 if bias else w2)[k][idx] += h
        return C.mse(C.Net(w2, b2).forward(x)[0], t)[0]

    h = 1e-5
    for k in range(4):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in ws[k].shape)
            fd = (L(k, idx, h) - L(k, idx, -h)) / (2 * h)
            assert abs(fd - dws[k][idx]) < 1e-7 * max(1.0, abs(fd)), (k, idx, fd, dws[k][idx])
        c = (int(rng.integers(0, bs[k].size)),)
        fd = (L(k, c, h, True) - L(k, c, -h, True)) / (2 * h)
        assert abs(fd - dbs[k][c]) < 1e-7 * max(1.0, abs(fd))


def test_silu_and_its_derivative():
    z = np.linspace(-6, 6, 49)
    np.testing.assert_allclose(C.silu(z), z / (1 + np.exp(-z)), rtol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(C.silu_grad(z), (C.silu(z + h) - C.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)
    assert C.silu(0.0) == 0.0 and C.silu_grad(0.0) == 0.5


def test_adam_first_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2, so every
    parameter moves by lr * g / (|g| + eps)."""
    g = rnd(50, seed=10)
    p = rnd(50, seed=11)
    p1, m, v = C.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_mse_value_and_gradient():
    y, t = rnd(3, 4, seed=12), rnd(3, 4, seed=13)
    loss, g = C.mse(y, t)
    assert abs(loss - ((y - t) ** 2).sum() / 12) < 1e-15
    np.testing.assert_allclose(g, (y - t) / 6)


def test_trilinear_upsampling_reproduces_linear_fields():
    """A linear field sampled at the coarse centres is reproduced exactly at
    every fine centre that lies between coarse centres; factor 1 is the
    identity."""
    d, h, w = 4, 5, 6
    D, H, W = 12, 15, 18
    cz = (np.arange(d) + 0.5) / d
    cy = (np.arange(h) + 0.5) / h
    cx = (np.arange(w) + 0.5) / w
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    src = np.stack([1 + 2 * X - Y + 3 * Z, X - Z], axis=-1)
    out = C.upsample_trilinear(src, (D, H, W))
    fz = (np.arange(D) + 0.5) / D
    fy = (np.arange(H) + 0.5) / H
    fx = (np.arange(W) + 0.5) / W
    FZ, FY, FX = np.meshgrid(fz, fy, fx, indexing="ij")
    exact = np.stack([1 + 2 * FX - FY + 3 * FZ, FX - FZ], axis=-1)
    inside = ((FZ >= cz[0]) & (FZ <= cz[-1]) & (FY >= cy[0]) & (FY <= cy[-1]) & (FX >= cx[0]) & (FX <= cx[-1]))
    np.testing.assert_allclose(out[inside], exact[inside], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(C.upsample_trilinear(src, (d, h, w)), src)


def test_cavity_features():
    f = C.cavity_features((2, 3, 4), 1500.0)
    assert f.shape == (2, 3, 4, 8)
    np.testing.assert_allclose(f[..., 0][0, 0], [-0.75, -0.25, 0.25, 0.75])
    np.testing.assert_allclose(f[..., 3], 1.0)
    np.testing.assert_allclose(f[..., 6], f[..., 2] ** 2)
