"""Multi-rank host logic of bench.py on CPU: two gloo ranks (the replicas-only
multi-GPU mode has no data-path collective; the ranks only agree on the
slowest replica's timing, which rank 0 reports)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 2.5])
    td.barrier()
    q.put((rank, out))
    td.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 2.5]


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks([3, 1.5]) == [3.0, 1.5]
