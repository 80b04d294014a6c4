"""The multi-rank timing path of bench.py on CPU: two gloo ranks, barrier and
max-over-ranks (the value of a weak-scaling run is the units of all ranks
over the slowest rank's time)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    ws, r = bench.init_dist("gloo")
    bench.barrier()
    got = bench.max_over_ranks(10.0 + rank)
    q.put((r, ws, got, bench.dist_env()))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, got, env in out:
        assert ws == 2 and got == 11.0 and env[0] == 2


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    ops, parts, tb = bench.fp64_ops_per_launch([0, 1, 4096, 4097])
    assert parts == 1 + 1 + 1 + 2
    assert tb == (0 + 1 + 4096 + 4097) + 8 * 5
    assert ops == parts * (15 * 3000 + 7) + tb * 22
