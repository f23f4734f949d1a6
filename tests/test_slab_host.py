"""Slab decomposition bookkeeping on CPU: gloo process groups of 2 and 3
ranks, each holding one slab of a periodic grid, against one oracle run of
the whole grid (bit-exact in FP64).

Each rank runs the library's scheme with the oracle's collision: it keeps
the post-collision populations of its own nodes, hands the planes that cross
its faces round the ring (paper_2206_00366_gb300.slab.split, .crossing and
.ring_exchange, the code the GPU path uses), and gathers from its own
periodic slab (Eq. 2-2b).  The CUDA pack/unpack kernels that move the same
planes are checked against a single-grid GPU run in
test_gpu_slab.py."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2206_00366_gb300 import slab as SL  # noqa: E402

CASES = {
    "D2Q9": dict(shape=(12, 10, 1), spacing=(1.0, 0.6, 1.0)),
    "D3Q27": dict(shape=(6, 5, 7), spacing=(1.0, 0.8, 0.5)),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(lattice):
    import oracle.rmrt as R
    import workloads as W
    c = CASES[lattice]
    lat = R.make_lattice(lattice, c["spacing"])
    S = R.relaxation_matrix(lat, R.rates_from_viscosity(lat, 0.02, 0.03, 1.1))
    m = R.Model()
    nx, ny, nz = c["shape"]
    f0 = W.random_populations(lat.q, (nz, ny, nx), seed=9, amp=0.05)
    return R, lat, S, m, f0


def collide_nodes(R, lat, m, S, f):
    """The oracle's collision node by node (numpy's batched products round
    differently for different batch widths; one node at a time makes the
    slabs and the whole grid compute every node identically)."""
    fl = f.reshape(lat.q, -1)
    out = np.empty_like(fl)
    for n in range(fl.shape[1]):
        out[:, n:n + 1] = R.collide(lat, m, S, fl[:, n:n + 1])
    return out.reshape(f.shape)


def gather(lat, B):
    """Pull streaming inside one periodic slab: node x reads B_j(x - e_j)."""
    out = np.empty_like(B)
    for j in range(lat.q):
        sh = [0, 0, 0]
        for al in range(lat.d):
            sh[2 - al] = int(lat.e[j, al])
        out[j] = np.roll(B[j], shift=sh, axis=(0, 1, 2))
    return out


def _worker(rank, world, port, lattice, steps, out, pipelined=False):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    R, lat, S, m, f0 = _setup(lattice)
    ax = 1 + SL.field_axis(lat.d)                       # axis of a population array (q, nz, ny, nx)
    off, cnt = SL.split(f0.shape[ax], world)[rank]
    f = np.take(f0, np.arange(off, off + cnt), axis=ax).copy()
    up_dirs, down_dirs = SL.crossing(lat.e, lat.d, +1), SL.crossing(lat.e, lat.d, -1)

    def plane(a, i):
        idx = [slice(None)] * a.ndim
        idx[ax - 1] = i
        return tuple(idx)
    n = f.shape[ax]
    for _ in range(steps):
        B = collide_nodes(R, lat, m, S, f)                                # post-collision, at the node
        up = torch.from_numpy(np.stack([B[j][plane(B[j], -1)] for j in up_dirs]).copy())
        down = torch.from_numpy(np.stack([B[j][plane(B[j], 0)] for j in down_dirs]).copy())
        from_below, from_above = torch.empty_like(up), torch.empty_like(down)
        reqs = SL.start_exchange(up, down, from_below, from_above, rank, world)
        if pipelined:
            # the interior planes 2 .. n - 3 pull only from planes 1 .. n - 2,
            # none of which the exchange replaces: gather them while it is in flight
            inner = np.take(gather(lat, B), np.arange(2, n - 2), axis=ax) if n >= 5 else None
        SL.finish_exchange(reqs)
        for k, j in enumerate(up_dirs):
            B[j][plane(B[j], -1)] = from_below[k].numpy()
        for k, j in enumerate(down_dirs):
            B[j][plane(B[j], 0)] = from_above[k].numpy()
        f = gather(lat, B)
        if pipelined and inner is not None:
            idx = [slice(None)] * f.ndim
            idx[ax] = slice(2, n - 2)
            f[tuple(idx)] = inner
    out.put((rank, off, f))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("pipelined", [False, True])
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q27"])
def test_slabs_reproduce_the_single_grid(lattice, world, pipelined):
    """pipelined: each rank gathers its interior planes 2 .. n - 3 while the
    exchange is in flight (posted by start_exchange, waited by
    finish_exchange), the split the GPU path makes with
    rmrtlb_step_interior / rmrtlb_step_boundary."""
    import torch.multiprocessing as mp
    steps = 5
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, lattice, steps, q, pipelined)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    parts = sorted((q.get() for _ in range(world)), key=lambda t: t[0])
    R, lat, S, m, f0 = _setup(lattice)
    whole = f0
    for _ in range(steps):
        whole = gather(lat, collide_nodes(R, lat, m, S, whole))
    ref = R.step(lat, m, S, f0, steps)                       # the oracle's own (batched) step, to round-off
    assert np.abs(whole - ref).max() <= 1e-14 * np.abs(ref).max()
    ax = 1 + SL.field_axis(lat.d)
    got = np.concatenate([p[2] for p in parts], axis=ax)
    np.testing.assert_array_equal(got, whole)


def test_split_and_crossing_sets():
    assert SL.split(7, 3) == [(0, 3), (3, 2), (5, 2)]
    assert SL.split(2048, 4) == [(0, 512), (512, 512), (1024, 512), (1536, 512)]
    with pytest.raises(ValueError):
        SL.split(2, 3)
    import oracle.rmrt as R
    for name, n in (("D2Q9", 3), ("D3Q19", 5), ("D3Q27", 9), ("D2Q5", 1), ("D3Q7", 1)):
        lat = R.make_lattice(name, (1.0, 0.8, 0.6) if lat_d(name) == 3 else (1.0, 0.8))
        up, down = SL.crossing(lat.e, lat.d, +1), SL.crossing(lat.e, lat.d, -1)
        assert len(up) == len(down) == n
        a = 1 if lat.d == 2 else 2
        # the two sets are each other's opposites
        assert sorted(tuple(-lat.e[j]) for j in up) == sorted(tuple(lat.e[j]) for j in down)
        assert all(lat.e[j, a] == 1 for j in up)


def lat_d(name):
    return 2 if name.startswith("D2") else 3


def test_global_check_reduces_sums_and_residual():
    """The reduction of the slabs' raw check sums gives the whole grid's
    totals and its residual sqrt(sum |du|^2 / sum |u|^2), not a mean of the
    slabs' residuals; flags are OR-ed; no previous snapshot anywhere gives
    -1."""
    rng = np.random.default_rng(3)
    u0, u1 = rng.normal(size=(2, 30)), rng.normal(size=(2, 30))
    rho = 1 + 0.01 * rng.normal(size=30)
    whole = np.sqrt(((u1 - u0) ** 2).sum() / (u1 ** 2).sum())
    sums = []
    for sl, fl in ((slice(0, 11), 0), (slice(11, 30), 4)):
        du2 = ((u1[:, sl] - u0[:, sl]) ** 2).sum()
        sums.append([rho[sl].sum(), *(rho[sl] * u1[0, sl]).sum(keepdims=True), 0.0, 0.0,
                     (0.5 * rho[sl] * (u1[:, sl] ** 2).sum(0)).sum(), du2, (u1[:, sl] ** 2).sum(), fl])
    g = SL.global_check(sums)
    assert g[0] == pytest.approx(rho.sum(), rel=1e-15)
    assert g[5] == pytest.approx(whole, rel=1e-14)
    assert int(g[7]) == 4
    sums[1][5] = -1.0
    assert SL.global_check(sums)[5] == -1.0
