"""Slab decomposition of one periodic grid, one slab per rank.

The grid is cut along its slowest axis (y on rD2Q9 / rD2Q5, z on the 3-D
lattices); every slab runs as an ordinary periodic solver of its own extent,
and after each step the populations that propagation (Eq. 2-2b) carries
across the slab faces are handed round the ring of slabs through
rmrtlb_halo_pack / rmrtlb_halo_unpack (the C ABI documents why the periodic
wrap of a slab is exactly where its neighbours' values belong).  The check
sums are reduced over the ranks in FP64 every check.

The exchange overlaps the next step's interior: populations that cross a
face only enter the two planes next to it, so each step runs as
rmrtlb_step_interior (planes 2 .. n - 3, needing no halo) while the previous
step's crossing planes are in flight, then the halo is unpacked and
rmrtlb_step_boundary steps the four planes next to the faces and completes
the step (bitwise the same step as rmrtlb_step).

This module holds the host-side bookkeeping only: the partition, the ring
exchange of device buffers over torch.distributed (NCCL between GPUs; any
backend that moves tensors works), and the global reductions; every step of
the method runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import rmrtlb as B


def split(n: int, parts: int):
    """(offset, count) of each part when n planes are cut into `parts`
    slabs as evenly as possible (the first n % parts get one more)."""
    if parts < 1 or n < parts:
        raise ValueError(f"cannot cut {n} planes into {parts} slabs")
    base, extra = divmod(n, parts)
    out, off = [], 0
    for r in range(parts):
        c = base + (1 if r < extra else 0)
        out.append((off, c))
        off += c
    return out


def field_axis(d: int) -> int:
    """Axis of a field array (nz, ny, nx) along which slabs are cut."""
    return 1 if d == 2 else 0


def crossing(e: np.ndarray, d: int, sign: int):
    """Directions j (increasing) whose component along the slab axis is sign."""
    a = 1 if d == 2 else 2
    return [j for j in range(e.shape[0]) if int(e[j, a]) == sign]


def start_exchange(send_up, send_down, recv_from_below, recv_from_above, rank: int, world: int, group=None):
    """Posts one exchange on the periodic ring of slabs and returns its
    requests: send_up goes to rank + 1 and send_down to rank - 1;
    recv_from_below receives rank - 1's up buffer and recv_from_above rank +
    1's down buffer.  The four operations are posted in the same order on
    every rank, so the two messages between a pair of neighbours (or, with
    two ranks, the two each way) match.  With NCCL the transfers wait for
    the work already on the current CUDA stream and run beside what is
    enqueued after them."""
    import torch.distributed as dist
    up, down = (rank + 1) % world, (rank - 1) % world
    if dist.get_backend(group) == "nccl":
        ops = [dist.P2POp(dist.isend, send_up, up, group), dist.P2POp(dist.irecv, recv_from_below, down, group),
               dist.P2POp(dist.isend, send_down, down, group), dist.P2POp(dist.irecv, recv_from_above, up, group)]
        return dist.batch_isend_irecv(ops)
    return [dist.isend(send_up, up, group), dist.irecv(recv_from_below, down, group),
            dist.isend(send_down, down, group), dist.irecv(recv_from_above, up, group)]


def finish_exchange(reqs):
    """Waits for an exchange (with NCCL: makes the current CUDA stream wait)."""
    for r in reqs:
        r.wait()


def ring_exchange(send_up, send_down, recv_from_below, recv_from_above, rank: int, world: int, group=None):
    """start_exchange and finish_exchange in one call."""
    finish_exchange(start_exchange(send_up, send_down, recv_from_below, recv_from_above, rank, world, group))


def global_check(sums) -> np.ndarray:
    """rmrtlb_stats-layout totals of the whole grid from the raw check sums
    of every slab (list of rmrtlb_check_sums arrays, or their sum with
    out[5] < 0 meaning no previous snapshot): mass, momentum, kinetic
    energy, residual sqrt(sum |u - u_prev|^2 / sum |u|^2), -, flags."""
    s = np.asarray(sums, dtype=np.float64).reshape(-1, 8)
    tot = s.sum(axis=0)
    out = np.zeros(8)
    out[0:5] = tot[0:5]
    out[5] = np.sqrt(tot[5] / tot[6]) if (s[:, 5] >= 0).all() and tot[6] > 0 else -1.0
    out[6] = -1.0
    out[7] = float(np.bitwise_or.reduce(s[:, 7].astype(np.int64)))
    return out


class Slab:
    """This rank's slab of a periodic grid (global shape (nx, ny, nz))."""

    def __init__(self, lattice, global_shape, spacing, dt=1.0, params=None, eq_kind="nse", basis="raw",
                 storage="f32", rank=0, world=1, group=None, device="cuda"):
        import torch
        q, d, self.e = B.rmrtlb_lattice_info(B.LATTICE_NAMES.get(lattice, lattice))
        self.d, self.rank, self.world, self.group = d, rank, world, group
        nx, ny, nz = global_shape
        n_axis = ny if d == 2 else nz
        self.parts = split(n_axis, world)
        off, cnt = self.parts[rank]
        self.offset, self.count = off, cnt
        local = (nx, cnt, nz) if d == 2 else (nx, ny, cnt)
        # global index of this slab's first node: the 16-bit rounding then
        # draws the same random bits as the whole grid would
        p = dict(params or {})
        p["node_offset"] = off * (nx if d == 2 else nx * ny)
        # the periodic check must see the state after the exchange: the slab
        # runs it itself (rmrtlb_check) instead of inside rmrtlb_step
        self.check_every = int(p.get("check_every", 0))
        p["check_every"] = 0
        self.steps = 0
        self._pending = None            # requests of the exchange in flight
        self.solver = B.Solver(lattice, local, spacing, dt, p, eq_kind, basis, storage, device=device)
        nbytes = B.rmrtlb_halo_bytes(self.solver.h)
        self.bufs = [torch.empty(nbytes, dtype=torch.uint8, device=device) for _ in range(4)]

    def local(self, field):
        """This slab's part of a global field (..., nz, ny, nx)."""
        ax = field.ndim - 3 + field_axis(self.d)
        idx = [slice(None)] * field.ndim
        idx[ax] = slice(self.offset, self.offset + self.count)
        return field[tuple(idx)]

    def init_equilibrium(self, rho, u=None):
        """f = f^eq of the global fields' slab part (numpy or CUDA tensors)."""
        self.finish()
        lr = np.ascontiguousarray(self.local(rho)) if isinstance(rho, np.ndarray) else self.local(rho).contiguous()
        lu = None
        if u is not None:
            lu = np.ascontiguousarray(self.local(u)) if isinstance(u, np.ndarray) else self.local(u).contiguous()
        self.solver.init_equilibrium(lr, lu)
        self.steps = 0

    def after_exchange(self):
        """Count the step and run the periodic check when one is due."""
        self.steps += 1
        if self.check_every > 0 and self.steps % self.check_every == 0:
            B.rmrtlb_check(self.solver.h)

    def pack(self):
        up, down = self.bufs[0], self.bufs[1]
        B.rmrtlb_halo_pack(self.solver.h, up.data_ptr(), down.data_ptr())
        return up, down

    def unpack(self, from_below, from_above):
        B.rmrtlb_halo_unpack(self.solver.h, from_below.data_ptr(), from_above.data_ptr())

    def step(self, n=1):
        """n steps, each followed by the exchange of the crossing planes.  The
        exchange of one step runs beside the interior of the next, also
        across calls: the last exchange is left in flight and lands at the
        next step, or at finish() (which every method that reads or replaces
        the state calls first)."""
        import torch
        if self.world == 1:
            for _ in range(n):
                self.solver.step(1)
                self.after_exchange()
            return
        h = self.solver.h
        # the library's kernels run on the solver's stream, and the exchange is ordered against it
        with torch.cuda.stream(self.solver.stream):
            for _ in range(n):
                B.rmrtlb_step_interior(h)
                self._land()
                B.rmrtlb_step_boundary(h)
                up, down = self.pack()
                self._pending = start_exchange(up, down, self.bufs[2], self.bufs[3], self.rank, self.world,
                                               self.group)

    def _land(self):
        """Completes the exchange in flight: wait, unpack, count the step."""
        if self._pending is not None:
            finish_exchange(self._pending)
            self._pending = None
            self.unpack(self.bufs[2], self.bufs[3])
            self.after_exchange()

    def finish(self):
        """Lands the exchange in flight (the slabs then hold the whole grid's
        state); a no-op when none is."""
        import torch
        if self._pending is not None:
            with torch.cuda.stream(self.solver.stream):
                self._land()

    def moments(self, rho=None, u=None):
        self.finish()
        return self.solver.moments(rho, u)

    def check(self):
        """Totals of the whole grid at the last periodic check (FP64
        allreduce of the slabs' raw sums)."""
        import torch
        import torch.distributed as dist
        self.finish()
        s = B.rmrtlb_check_sums(self.solver.h)
        if self.world == 1:
            return global_check([s])
        dev = self.bufs[0].device
        t = torch.tensor(s[:7], dtype=torch.float64, device=dev)
        # flag bits and "no previous snapshot" as 0/1 values reduced by max
        # (an OR that every backend supports)
        bits = torch.tensor([(int(s[7]) >> k) & 1 for k in range(4)] + [1 if s[5] < 0 else 0],
                            dtype=torch.float64, device=dev)
        dist.all_reduce(t, group=self.group)
        dist.all_reduce(bits, op=dist.ReduceOp.MAX, group=self.group)
        tot = np.zeros(8)
        tot[:7] = t.cpu().numpy()
        b = bits.cpu().numpy().astype(np.int64)
        tot[5] = -1.0 if b[4] else tot[5]
        tot[7] = float(sum(int(b[k]) << k for k in range(4)))
        return global_check([tot])


class LocalSlabs:
    """Several slabs of one grid driven from one process on one device (the
    exchange is a device copy between their buffers): the decomposition's
    arithmetic without a process group, for tests and single-GPU use."""

    def __init__(self, parts, lattice, global_shape, spacing, dt=1.0, params=None, eq_kind="nse", basis="raw",
                 storage="f32", device="cuda"):
        self.slabs = [Slab(lattice, global_shape, spacing, dt, params, eq_kind, basis, storage, rank=r, world=parts,
                           device=device) for r in range(parts)]

    def init_equilibrium(self, rho, u=None):
        for s in self.slabs:
            s.init_equilibrium(rho, u)

    def step(self, n=1):
        """The schedule of Slab.step with the exchange as device copies: each
        step's interior runs before the previous step's halo is unpacked."""
        import torch
        w = len(self.slabs)
        if w == 1:
            for _ in range(n):
                self.slabs[0].solver.step(1)
                self.slabs[0].after_exchange()
            return
        packed = None

        def land():
            torch.cuda.synchronize()
            for r, s in enumerate(self.slabs):
                s.unpack(packed[(r - 1) % w][0], packed[(r + 1) % w][1])
            torch.cuda.synchronize()
            for s in self.slabs:
                s.after_exchange()
        for _ in range(n):
            for s in self.slabs:
                B.rmrtlb_step_interior(s.solver.h)
            if packed is not None:
                land()
            for s in self.slabs:
                B.rmrtlb_step_boundary(s.solver.h)
            packed = [s.pack() for s in self.slabs]
        if packed is not None:
            land()

    def moments(self):
        """Global (rho, u) assembled from the slabs."""
        rs, us = zip(*[s.moments() for s in self.slabs])
        d = self.slabs[0].d
        ax = field_axis(d)
        return np.concatenate(rs, axis=ax), np.concatenate(us, axis=ax + 1)

    def populations(self):
        d = self.slabs[0].d
        return np.concatenate([s.solver.get_populations() for s in self.slabs], axis=field_axis(d) + 1)

    def check(self):
        return global_check([B.rmrtlb_check_sums(s.solver.h) for s in self.slabs])
