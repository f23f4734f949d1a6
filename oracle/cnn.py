"""Plain FP64 oracle for the warm-start convolutional network.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the oracle legs of ``bench.py`` may import it; it shares nothing with the
CUDA library.

The paper has no learned component: its RMRT-LB step is the solver whose
steady states the network learns to predict, and a warm-started run is
accepted only when the solver's own residual converges.  Everything here is a plain textbook definition, written out
loop by loop over the 27 taps with numpy matrix products over channels:

* 3-D cross-correlation with a 3 x 3 x 3 kernel and zero padding ("same"
  size), its gradients with respect to the input, the weights and the bias;
* SiLU, z * sigmoid(z), and its derivative;
* mean squared error;
* one Adam step (Kingma and Ba, "Adam: a method for stochastic
  optimization", ICLR 2015, Algorithm 1, with bias-corrected moments);
* trilinear interpolation between two cell-centred grids of one box.

Layout: activations (n, D, H, W, C), channels last, x fastest among the
spatial axes; weights (27, Cin, Cout) with tap t = 9 (dz + 1) + 3 (dy + 1)
+ (dx + 1); the output at voxel v reads the input at v + (dz, dy, dx).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _window(xp: np.ndarray, dz: int, dy: int, dx: int, shape) -> np.ndarray:
    """xp padded by one voxel on each spatial side; the (D, H, W) window
    whose voxel v holds x[v + (dz, dy, dx)] (zero outside)."""
    D, H, W = shape
    return xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]


def _pad(x: np.ndarray) -> np.ndarray:
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[v, co] = b[co] + sum_t sum_ci x[v + tap_t, ci] w[t, ci, co]."""
    n, D, H, W, ci = x.shape
    assert w.shape[:2] == (27, ci)
    xp = _pad(np.asarray(x, dtype=np.float64))
    y = np.zeros((n, D, H, W, w.shape[2])) + np.asarray(b, dtype=np.float64)
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += _window(xp, dz, dy, dx, (D, H, W)) @ w[t]
    return y


def conv3d_backward_data(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dL/dx[v, ci] = sum_t sum_co dy[v - tap_t, co] w[t, ci, co]."""
    n, D, H, W, co = dy.shape
    dyp = _pad(np.asarray(dy, dtype=np.float64))
    dx = np.zeros((n, D, H, W, w.shape[1]))
    for t, (dz, dyy, dxx) in enumerate(TAPS):
        dx += _window(dyp, -dz, -dyy, -dxx, (D, H, W)) @ w[t].T
    return dx


def conv3d_backward_weight(x: np.ndarray, dy: np.ndarray):
    """dL/dw[t, ci, co] = sum_v x[v + tap_t, ci] dy[v, co]; dL/db = sum_v dy."""
    n, D, H, W, ci = x.shape
    co = dy.shape[-1]
    xp = _pad(np.asarray(x, dtype=np.float64))
    g = np.asarray(dy, dtype=np.float64).reshape(-1, co)
    dw = np.zeros((27, ci, co))
    for t, (dz, dyy, dxx) in enumerate(TAPS):
        dw[t] = _window(xp, dz, dyy, dxx, (D, H, W)).reshape(-1, ci).T @ g
    return dw, g.sum(axis=0)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def mse(y: np.ndarray, t: np.ndarray):
    """(mean of (y - t)^2, its gradient 2 (y - t) / count)."""
    r = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float((r * r).mean()), 2.0 * r / r.size


def adam_step(p, g, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Algorithm 1 of Kingma and Ba); returns new (p, m, v).
    step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def upsample_trilinear(src: np.ndarray, out_shape) -> np.ndarray:
    """Trilinear interpolation of src (d, h, w, C) onto (D, H, W): both
    grids are cell-centred in the same box, so fine voxel I of N along an
    axis sits at source coordinate s = (I + 1/2) n / N - 1/2, clamped to
    [0, n - 1] (constant extension beyond the outermost centres)."""
    src = np.asarray(src, dtype=np.float64)
    out = src
    for ax, N in enumerate(out_shape):
        n = out.shape[ax]
        s = np.clip((np.arange(N) + 0.5) * n / N - 0.5, 0.0, n - 1)
        i0 = np.floor(s).astype(int)
        i1 = np.minimum(i0 + 1, n - 1)
        f = s - i0
        shape = [1] * out.ndim
        shape[ax] = N
        f = f.reshape(shape)
        out = np.take(out, i0, axis=ax) * (1.0 - f) + np.take(out, i1, axis=ax) * f
    return out


def cavity_features(shape, re: float, re_ref=(800.0, 700.0)) -> np.ndarray:
    """The network input of one cavity, (D, H, W, 8): cell-centred
    coordinates xh, yh, zh in (-1, 1), the scaled Reynolds number
    rh = (Re - 800) / 700, and xh zh, yh zh, zh^2, rh zh (the lid sits at
    zh = 1)."""
    D, H, W = shape
    z = (np.arange(D) + 0.5) / D * 2.0 - 1.0
    y = (np.arange(H) + 0.5) / H * 2.0 - 1.0
    x = (np.arange(W) + 0.5) / W * 2.0 - 1.0
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = (re - re_ref[0]) / re_ref[1] * np.ones_like(X)
    return np.stack([X, Y, Z, r, X * Z, Y * Z, Z * Z, r * Z], axis=-1)


class Net:
    """conv(8 -> c) SiLU, conv(c -> c) SiLU, conv(c -> c) SiLU, conv(c -> 4)."""

    def __init__(self, weights, biases):
        self.w = [np.asarray(w, dtype=np.float64) for w in weights]
        self.b = [np.asarray(b, dtype=np.float64) for b in biases]

    def forward(self, x):
        """Returns the output and the per-layer (input, pre-activation)."""
        cache = []
        a = np.asarray(x, dtype=np.float64)
        for k, (w, b) in enumerate(zip(self.w, self.b)):
            z = conv3d(a, w, b)
            cache.append((a, z))
            a = silu(z) if k + 1 < len(self.w) else z
        return a, cache

    def backward(self, cache, dy):
        """Gradients (dW list, db list) of a loss with dL/dy = dy."""
        dws, dbs = [None] * len(self.w), [None] * len(self.w)
        g = dy
        for k in reversed(range(len(self.w))):
            a, z = cache[k]
            if k + 1 < len(self.w):
                g = g * silu_grad(z)
            dws[k], dbs[k] = conv3d_backward_weight(a, g)
            if k > 0:
                g = conv3d_backward_data(g, self.w[k])
        return dws, dbs
