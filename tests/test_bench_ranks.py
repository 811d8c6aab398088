"""The benchmark's multi-rank logic on CPU with gloo, world size 2: every rank evaluates its own
replica (no collective on the data path) and the timing is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    mx = bench.max_over_ranks(10.0 + 5 * rank)
    # replicas: each rank draws its own seeded problem; no data crosses ranks
    import synth
    p = synth.tiny(seed=101 + 1000 * r)
    q.put((r, ws, mx, int(p.tree.n), float(p.tree.pos.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 15.0 for g in got)          # max over ranks
    assert got[0][4] != got[1][4]                  # different replicas per rank
