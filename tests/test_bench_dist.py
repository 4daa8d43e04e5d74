"""Host-side logic of bench.py's N-GPU mode (independent replicas): the
max-over-ranks timing, the barrier and the reference arm's rank handling,
run as two gloo ranks on CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.dist_max(w, 1.0 + rank)          # rank 1 is the slowest
    # reference arm: only rank 0 works; the others return 0 without output
    class A:
        steps, warmup = 1, 3
    rc = bench.run_reference(A, w, r) if r == 1 else 0
    q.put((rank, t, rc))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(world))
    assert [g[1] for g in got] == [2.0, 2.0]
    assert all(g[2] == 0 for g in got)
