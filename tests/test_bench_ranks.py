"""The bench's multi-rank host logic on CPU: two gloo ranks run as replicas.

Each rank solves its own right-hand sides (no collective on the data path);
the only collective is the max over ranks of the timed interval, and the
whole-job throughput is the units all ranks processed over that time."""
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    r, w, local = bench.dist_init(None)
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        # rank 1 is the slow one: every rank must report its time
        slowest = bench.max_over_ranks(1.5 + rank, w, device="cpu")
        seeds = [bench.rhs_seed(r, k) for k in range(4)] + [bench.rhs_seed(r, k, 500)
                                                            for k in range(16)]
        queue.put((r, w, local, slowest, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    queue = ctx.SimpleQueue()
    mp.spawn(_rank_main, args=(world, port, queue), nprocs=world, join=True)
    out = sorted(queue.get() for _ in range(world))
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert [o[3] for o in out] == [2.5, 2.5]
    assert len(set(out[0][4])) == len(out[0][4])
    assert not set(out[0][4]) & set(out[1][4])


def test_single_rank_and_rate(capsys):
    bench.run_reference(None, 1, 2)  # a rank other than 0 exits without work
    assert capsys.readouterr().out == ""
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(4, 5, 10.0) == 2.0
    assert bench.rhs_seed(0, 3) == 3 and bench.rhs_seed(2, 3, 500) == 2503
