"""Host side of bench.py's multi-process path on CPU (gloo, world size 2):
each rank times its own share of queries, the job's time is the slowest
rank's, and the reported throughput is all ranks' units over that time.
No GPU and no collective on the data path are involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    d = bench.Dist("gloo")
    try:
        ms = d.max(100.0 + 50.0 * rank)          # rank 1 is the slower one
        d.barrier()
        q.put((rank, ms, bench.aggregate(ms, 1000, d.world)))
    finally:
        d.close()


def test_slowest_rank_sets_the_time_and_units_add_up():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, ms, v in out:
        assert ms == pytest.approx(150.0)
        assert v == pytest.approx(2 * 1000 / 0.150)
