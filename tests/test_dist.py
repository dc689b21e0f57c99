"""The N > 1 path of bench.py on CPU: replicas only (each rank runs its own
layer, no collective on the data path), so what needs covering is the timing
plumbing, the max over ranks and the barrier, with world_size 2 over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, rk, local = bench.dist_env()
        assert (ws, rk, local) == (world, rank, rank)
        bench.barrier(ws)
        mx = bench.reduce_max(float(10 * rank + 1), ws)
        out.put((rank, mx))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_barrier_over_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]  # every rank sees the slowest rank's value


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)  # no process group needed
