"""Host logic of the replicated multi-rank run (one process per GPU, no
data-path collective), on CPU with gloo and world size 2: the timing is the
maximum over ranks and the throughput counts every rank's nodes; the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 20.0][rank]
    m = bench.max_over_ranks(local_ms)
    out.put((rank, m, bench.replica_mlups(world, 1000, 10, m * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, m, mlups in got:
        assert m == 20.0                                  # the slowest rank sets the time
        assert abs(mlups - 2 * 1000 * 10 / 0.020 / 1e6) < 1e-12


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_mlups(1, 8388608, 100, 1.0) == pytest.approx(838.8608)


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun only rank 0 runs the oracle arm; the others exit 0
    without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_concurrent_oracle_processes_start_together():
    """The all-cores oracle timing: two one-thread oracle processes on their
    own bands start their timed steps on one signal and both finish."""
    import bench
    wall = bench._oracle_children(64, 8, 2, 2)
    assert 0.0 < wall < 120.0
    assert bench.host_cores() >= 1
