"""Multi-process (replica) aggregation of bench.py, on CPU with the gloo backend.

Each rank runs its own independent replica; the job time is the slowest
rank's and the work is the sum over ranks (weak scaling).  No data-path
collective exists in the method, so only these two reductions and the
barrier are exercised."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier(ws)
    t = bench.max_over_ranks(100.0 + 50.0 * rank, ws)
    w = bench.sum_over_ranks(1000.0 * (rank + 1), ws)
    # every reduction of the benchmark, as each rank calls it (a rank-only call would hang the others)
    tot = bench.replica_totals(ws, {"comp": 10.0 + rank, "plain": 20.0 - rank}, 30.0 + 5 * rank, 1e12)
    q.put((r, local, t, w, tot))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and [g[1] for g in got] == [0, 1]
    assert all(g[2] == 150.0 for g in got)       # slowest rank's time
    assert all(g[3] == 3000.0 for g in got)      # total work of all replicas
    for g in got:
        tot = g[4]
        assert tot["comp"] == {"t_max": 11.0, "pairs": 2e12} and tot["plain"] == {"t_max": 20.0, "pairs": 2e12}
        assert tot["e2e"] == {"t_max": 35.0, "pairs": 2e12}


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0 and bench.sum_over_ranks(7.0, 1) == 7.0
