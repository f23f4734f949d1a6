"""Learned warm start for steady lid-driven cavities on rD3Q27.

A small convolutional network (four 3 x 3 x 3 convolutions, 8 -> 32 -> 32 ->
32 -> 4 channels, SiLU, BF16 weights and activations, FP32 master weights)
maps the cell-centred coordinates and the Reynolds number of a cavity to its
steady density and velocity in scaled units.  Its training data are steady
states of the RMRT-LB solver itself (rmrtlb_batch_* on many small cavities
at once); training and inference run in the kernels of rmrtlb_cnn.h,
driven from here; the prediction is upsampled to the target grid and turned
into the solver's initial state f^eq + f^ne (Eq. fne, rmrtlb_batch_init_fields).
The solver's own residual then decides convergence, exactly as for a cold
start, so a poor prediction costs steps but never changes the answer.

The paper has no learned part: this module is the warm-start extension of
the solver, not a step of the method.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import rmrtlb as B

CH = (8, 32, 32, 32, 4)
RE_RANGE = (100.0, 1500.0)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cavity_warmstart.npz")


def _ptr(t) -> int:
    return t.data_ptr()


def cavity(shape, re, lid_u=0.05, spacing=(1.0, 1.0, 0.5), s_free=1.1):
    """rmrtlb_domain fields of a cubic-cell-count cavity (nz, ny, nx) =
    shape with Reynolds number Re = U nx dx / nu, lid on the top z face."""
    nz, ny, nx = shape
    nu = lid_u * nx * spacing[0] / re
    return dict(nx=nx, ny=ny, nz=nz, dx=spacing[0], dy=spacing[1], dz=spacing[2], nu=nu, nu_bulk=nu,
                s_free=s_free, lid_u=lid_u, cs2=0.0)


def scales(dom):
    """(rho_scale, u_scale): targets are ((rho - rho0) c_s^2 / U^2, u / U)."""
    cs2 = min(dom["dx"], dom["dy"], dom["dz"]) ** 2 / 3.0 if dom.get("cs2", 0) <= 0 else dom["cs2"]
    U = dom["lid_u"]
    return cs2 / (U * U), 1.0 / U


def generate_states(res, shape=(32, 64, 64), tol=1e-6, max_steps=60000, chunk=500, lid_u=0.05,
                    spacing=(1.0, 1.0, 0.5), device="cuda", log=None):
    """Steady states of cavities with the given Reynolds numbers, computed by
    the batched solver (FP32 storage, raw moments) from rest.  Returns
    (targets FP32 (n, nz, ny, nx, 4) on the device, steps to converge (-1:
    not converged within max_steps or unstable), seconds)."""
    import torch
    n = len(res)
    nz, ny, nx = shape
    N = nx * ny * nz
    T = torch.zeros((n,) + tuple(shape) + (4,), dtype=torch.float32, device=device)
    steps = np.full(n, -1, dtype=np.int64)
    rho = torch.empty(N, dtype=torch.float64, device=device)
    u = torch.empty((3, N), dtype=torch.float64, device=device)
    t0 = time.perf_counter()
    for c0 in range(0, n, chunk):
        doms = [cavity(shape, float(r), lid_u, spacing) for r in res[c0:c0 + chunk]]
        b = B.Batch(doms, storage="f32", check_every=100, tol=tol, device=device, lattice="D3Q27", basis="raw")
        b.tune(3)
        b.run(max_steps)
        _, conv, act, _ = b.status()
        for k, d in enumerate(doms):
            if act[k] != 0:
                continue
            steps[c0 + k] = conv[k]
            B.rmrtlb_batch_fields(b.h, k, _ptr(rho), _ptr(u))
            rs, us = scales(d)
            B.rmrtlb_pack_fields(N, 3, _ptr(rho), _ptr(u), 1.0, rs, us, _ptr(T[c0 + k]))
        torch.cuda.synchronize()
        if log:
            log(f"states {c0 + len(doms)}/{n}: converged {int((steps[:c0 + len(doms)] > 0).sum())}, "
                f"{time.perf_counter() - t0:.1f} s")
        del b
    return T, steps, time.perf_counter() - t0


class Net:
    """The network's parameters in one flat FP32 master buffer (W1, b1, ...,
    W4, b4; W as (27, cin, cout)), its BF16 copy, the Adam moments and the
    gradient, plus the activation buffers of the last batch shape used."""

    def __init__(self, seed=0, device="cuda", flat=None):
        import torch
        sizes = []
        for k in range(4):
            sizes += [27 * CH[k] * CH[k + 1], CH[k + 1]]
        self.off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        total = int(self.off[-1])
        if flat is None:
            rng = np.random.default_rng(seed)
            flat = np.zeros(total, dtype=np.float32)
            for k in range(4):
                std = np.sqrt(2.0 / (27 * CH[k])) * (0.3 if k == 3 else 1.0)
                flat[self.off[2 * k]:self.off[2 * k + 1]] = rng.normal(0.0, std, sizes[2 * k])
        self.device = device
        self.master = torch.tensor(np.asarray(flat, dtype=np.float32), device=device)
        self.bf16 = torch.empty(total, dtype=torch.bfloat16, device=device)
        self.m = torch.zeros(total, dtype=torch.float32, device=device)
        self.v = torch.zeros(total, dtype=torch.float32, device=device)
        self.grad = torch.zeros(total, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.scratch_mse = torch.empty(8192, dtype=torch.uint8, device=device)
        self.step_count = 0
        # BF16 copy through the optimiser kernel with a zero step (no change)
        B.rmrtlb_adam(total, _ptr(self.master), _ptr(self.bf16), _ptr(self.grad), _ptr(self.m), _ptr(self.v), 1, 0.0)
        self._shape = None

    # parameter views (byte addresses inside the flat buffers)
    def w16(self, k):
        return _ptr(self.bf16) + 2 * int(self.off[2 * k])

    def bias(self, k):
        return _ptr(self.master) + 4 * int(self.off[2 * k + 1])

    def gw(self, k):
        return _ptr(self.grad) + 4 * int(self.off[2 * k])

    def gb(self, k):
        return _ptr(self.grad) + 4 * int(self.off[2 * k + 1])

    def _buffers(self, n, shape):
        import torch
        if self._shape == (n,) + tuple(shape):
            return
        d, h, w = shape
        V = n * d * h * w
        dev = self.device
        self.x = torch.empty(V * CH[0], dtype=torch.bfloat16, device=dev)
        self.z = [torch.empty(V * CH[k + 1], dtype=torch.float32, device=dev) for k in range(4)]
        self.a = [torch.empty(V * CH[k + 1], dtype=torch.bfloat16, device=dev) for k in range(3)]
        self.dy = torch.empty(V * CH[4], dtype=torch.float32, device=dev)
        self.g = [torch.empty(V * 32, dtype=torch.float32, device=dev) for _ in range(2)]
        sb = max(B.rmrtlb_conv3d_backward_weight_scratch(n, d, h, w, CH[k], CH[k + 1]) for k in range(4))
        self.scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
        # BF16 copy of dy for the copy-fed input gradient (0 bytes where it does not apply)
        sd = max(B.rmrtlb_conv3d_backward_data_scratch(n, d, h, w, CH[k], CH[k + 1]) for k in range(1, 4))
        self.scratch_dy = torch.empty(max(sd, 16), dtype=torch.uint8, device=dev)
        self.re = torch.empty(n, dtype=torch.float64, device=dev)
        self._shape = (n,) + tuple(shape)

    def forward(self, re, shape):
        """Network output (FP32, (n, d, h, w, 4) flat) for cavities of the
        given Reynolds numbers on a d x h x w grid."""
        import torch
        n = len(re)
        self._buffers(n, shape)
        d, h, w = shape
        self.re.copy_(torch.as_tensor(np.asarray(re, dtype=np.float64)))
        B.rmrtlb_cavity_features(n, d, h, w, _ptr(self.re), _ptr(self.x))
        inp = self.x
        for k in range(4):
            out = self.a[k] if k < 3 else None
            B.rmrtlb_conv3d_forward(n, d, h, w, CH[k], CH[k + 1], _ptr(inp), self.w16(k), self.bias(k), k < 3,
                                    _ptr(self.z[k]), _ptr(out) if out is not None else None)
            inp = out
        return self.z[3]

    def train_step(self, re, shape, targets, lr, beta1=0.9, beta2=0.999):
        """One Adam step on the MSE against targets (FP32 (n, d, h, w, 4)
        contiguous on the device).  Returns the loss as a device tensor."""
        n = len(re)
        d, h, w = shape
        y = self.forward(re, shape)
        count = y.numel()
        B.rmrtlb_mse(count, _ptr(y), _ptr(targets), _ptr(self.dy), _ptr(self.loss), _ptr(self.scratch_mse))
        g = self.dy
        acts = [self.x] + self.a
        sb = self.scratch.numel()
        for k in reversed(range(4)):
            B.rmrtlb_conv3d_backward_weight(n, d, h, w, CH[k], CH[k + 1], _ptr(acts[k]), _ptr(g), self.gw(k),
                                            self.gb(k), _ptr(self.scratch), sb)
            if k > 0:
                nxt = self.g[k % 2]
                B.rmrtlb_conv3d_backward_data(n, d, h, w, CH[k], CH[k + 1], _ptr(g), self.w16(k),
                                              _ptr(self.z[k - 1]), _ptr(nxt), _ptr(self.scratch_dy),
                                              self.scratch_dy.numel())
                g = nxt
        self.step_count += 1
        B.rmrtlb_adam(self.master.numel(), _ptr(self.master), _ptr(self.bf16), _ptr(self.grad), _ptr(self.m),
                      _ptr(self.v), self.step_count, lr, beta1, beta2)
        return self.loss

    def save(self, path, meta=None):
        np.savez(path, master=self.master.cpu().numpy(), meta=json.dumps(meta or {}))

    @classmethod
    def load(cls, path, device="cuda"):
        z = np.load(path)
        net = cls(device=device, flat=z["master"])
        net.meta = json.loads(str(z["meta"]))
        return net


def train(net, T, res, shape, epochs, batch=4, lr=2e-3, lr_end=1e-4, seed=0, log=None):
    """Adam with a cosine learning-rate decay over `epochs` passes of the
    samples (T: device targets (n, d, h, w, 4); res: their Reynolds numbers)."""
    import torch
    rng = np.random.default_rng(seed)
    n = len(res)
    steps = epochs * (n // batch)
    k = 0
    t0 = time.perf_counter()
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        acc = torch.zeros(1, dtype=torch.float64, device=net.device)
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            rate = lr_end + 0.5 * (lr - lr_end) * (1 + np.cos(np.pi * k / max(steps, 1)))
            tb = T[torch.as_tensor(idx, device=T.device)].contiguous()
            acc += net.train_step([res[j] for j in idx], shape, tb, float(rate))
            k += 1
        B.rmrtlb_cnn_check()
        mean = float(acc.item()) / max(1, n // batch)
        losses.append(mean)
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {mean:.3e}, {time.perf_counter() - t0:.1f} s")
    return losses, time.perf_counter() - t0


def warm_fields(net, re, coarse, fine, dom, rho0=1.0):
    """Predicted (rho, u) of a cavity on its fine grid: the network on the
    coarse grid, trilinear upsampling, unscaling.  FP64 device tensors
    rho (nz, ny, nx) and u (3, nz, ny, nx)."""
    import torch
    y = net.forward([re], coarse)
    B.rmrtlb_cnn_check()
    D, H, W = fine
    dst = torch.empty((4, D, H, W), dtype=torch.float64, device=net.device)
    rs, us = scales(dom)
    d, h, w = coarse
    B.rmrtlb_upsample_fields(d, h, w, 4, _ptr(y), D, H, W, [1.0 / rs, 1.0 / us, 1.0 / us, 1.0 / us],
                             [rho0, 0.0, 0.0, 0.0], _ptr(dst))
    # the network runs on the legacy stream; the solver reads the fields on
    # its own (non-blocking) stream
    torch.cuda.synchronize()
    return dst[0], dst[1:4]


def time_to_steady(dom, re, net=None, coarse=None, tol=1e-6, max_steps=2_000_000, noneq=True, tune=True,
                   device="cuda"):
    """Steps and wall time for one cavity to reach residual `tol`, from rest
    (net None) or from the network's prediction (inference, upsampling and
    initialisation included in the time).  Returns a dict with the final
    fields as FP64 device tensors."""
    import torch
    b = B.Batch([dom], storage="f32", check_every=100, tol=tol, device=device, lattice="D3Q27", basis="raw")
    if tune:
        b.tune(3)
    fine = (dom["nz"], dom["ny"], dom["nx"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if net is not None:
        rho, u = warm_fields(net, re, coarse, fine, dom)
        b.init_fields(0, rho, u, noneq=noneq)
    t_init = time.perf_counter() - t0
    issued = b.run(max_steps)
    wall = time.perf_counter() - t0
    res, conv, act, _ = b.status()
    N = dom["nx"] * dom["ny"] * dom["nz"]
    rho_f = torch.empty(N, dtype=torch.float64, device=device)
    u_f = torch.empty((3, N), dtype=torch.float64, device=device)
    B.rmrtlb_batch_fields(b.h, 0, _ptr(rho_f), _ptr(u_f))
    return dict(steps=int(conv[0]), issued=int(issued), state=int(act[0]), residual=float(res[0]), wall_s=wall,
                init_s=t_init, rho=rho_f, u=u_f)


def main(argv=None):
    """Train on solver-generated steady states and save the weights:
    python -m paper_2206_00366_gb300.warmstart --states 2000 --epochs 30 --out W.npz
    (the arguments the committed weights were trained with)"""
    import argparse

    import torch
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--states", type=int, default=2000)
    ap.add_argument("--shape", type=int, nargs=3, default=(32, 64, 64), help="nz ny nx of the training cavities")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-steps", type=int, default=60000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--holdout", type=float, default=0.1)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)
    rng = np.random.default_rng(a.seed)
    res = rng.uniform(*RE_RANGE, size=a.states)
    shape = tuple(a.shape)
    T, steps, t_gen = generate_states(res, shape=shape, tol=a.tol, max_steps=a.max_steps, log=log)
    ok = np.flatnonzero(steps > 0)
    nval = int(round(a.holdout * len(ok)))
    val, trn = ok[:nval], ok[nval:]
    net = Net(seed=a.seed)
    Tt = T[torch.as_tensor(trn, device=T.device)].contiguous()
    losses, t_train = train(net, Tt, [float(res[i]) for i in trn], shape, a.epochs, a.batch, a.lr, log=log)
    # held-out error of the predicted velocity, relative L2 per cavity
    errs = []
    for i in val:
        y = net.forward([float(res[i])], shape).view(shape + (4,))
        t = T[int(i)]
        errs.append(float(torch.linalg.vector_norm(y[..., 1:] - t[..., 1:]) / torch.linalg.vector_norm(t[..., 1:])))
    meta = dict(states=a.states, converged=int(len(ok)), train=int(len(trn)), holdout=int(len(val)), shape=shape,
                tol=a.tol, max_steps=a.max_steps, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed,
                re_range=RE_RANGE, generate_s=round(t_gen, 1), train_s=round(t_train, 1),
                final_loss=losses[-1], holdout_u_rel_l2_median=float(np.median(errs)) if errs else None,
                steps_to_steady_median=int(np.median(steps[ok])) if len(ok) else None)
    net.save(a.out, meta)
    log(json.dumps(meta))


if __name__ == "__main__":
    main()
