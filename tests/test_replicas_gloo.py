"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas only, no
data-path collective) — each rank times its own sequence, the ranks meet at
the barrier, and the slowest rank's time is the one reported."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, pg = bench.dist_setup(world, backend="gloo")
    bench.barrier(pg)
    worst = bench.max_over_ranks(pg, 10.0 + r)     # rank r "took" 10 + r ms
    bench.barrier(pg)
    q.put((r, w, worst, bench.replica_seed(r)))
    pg.destroy_process_group()


def test_two_gloo_ranks_meet_at_barrier_and_report_the_max():
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    assert all(w == 2 for _, w, _, _ in res)
    assert all(worst == 11.0 for _, _, worst, _ in res)     # the max over ranks
    assert res[0][3] != res[1][3]                           # independent sequences


def test_single_process_path_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r, w, local, pg = bench.dist_setup(1)
    assert (r, w, local, pg) == (0, 1, 0, None)
    assert bench.max_over_ranks(pg, 3.5) == 3.5
