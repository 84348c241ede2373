"""The multi-process logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

The solver runs on one GPU with no collectives; with several GPUs each rank
solves its own replica, and bench.py only needs a barrier and a max over
ranks of its timings. These are checked here without a GPU.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    vals = bench.allreduce_max([float(rank + 1), 10.0 - rank, -float(rank)], w)
    out.put((rank, vals))
    bench.barrier(w)
    dist.destroy_process_group()


def test_bench_ranks_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r] == [2.0, 10.0, 0.0]


def test_bench_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.allreduce_max([1.0, 2.0], 1) == [1.0, 2.0]
    bench.barrier(1)


def _rank_dies(rank, world, port, out):
    """Rank 1 joins and then exits with an error before the first barrier;
    rank 0's barrier must end with an error instead of waiting for it."""
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "BENCH_PG_TIMEOUT_S": "10"})
    sys.path.insert(0, ROOT)
    import bench

    w, r, _ = bench.dist_init()
    if r == 1:
        os._exit(3)  # a replica that failed
    try:
        bench.barrier(w)
        out.put((r, "passed"))
    except Exception as e:  # noqa: BLE001 - any error is the expected outcome
        out.put((r, type(e).__name__))


def test_bench_rank_failure_is_reported():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    r, what = q.get(timeout=120)
    assert r == 0 and what != "passed"
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
