"""bench.py's multi-rank plumbing on CPU (gloo, world size 2): one process per
rank, barrier, max-over-ranks timing, and distinct query seeds per rank (weak
scaling: every rank serves its own queries, no data-path collective)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    try:
        bench.dist_init(world, "gloo")
        r, lr, w = bench.dist_env()
        bench.barrier(w)
        mx = bench.max_over_ranks(float(10 + 5 * r), w)
        q.put((r, w, mx, bench.rank_seed(20, r)))
    finally:
        import torch.distributed as dist

        if dist.is_initialized():
            dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_agree_on_max_time_and_use_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)  # every rank sees the slowest rank's time
    assert out[0][3] != out[1][3]


def test_single_rank_is_a_no_op():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.rank_seed(20, 0) == 20
