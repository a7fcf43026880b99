"""The N > 1 host path of bench.py on CPU: world_size 2 over gloo.  The
workload is replicated (one independent solve per rank, no data-path
collective); the only cross-rank step is the max over ranks of the timed
totals, from which the whole-job throughput is computed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

TOTALS = {0: [100.0, 400.0, 120.0], 1: [250.0, 300.0, 90.0]}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        tot, val = bench.aggregate(TOTALS[rank], world, units=1000, steps=5)
        q.put((rank, tot, val))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [max(a, b) for a, b in zip(TOTALS[0], TOTALS[1])]
    for rank, tot, val in res:
        assert tot == want  # every rank sees the slowest rank's totals
        # whole-job throughput: units of all ranks / the slowest time
        assert val == [2 * 1000 * 5 / (t / 1e3) for t in want]


def test_single_rank_is_identity():
    tot, val = bench.aggregate([200.0], 1, units=10, steps=2)
    assert tot == [200.0] and val == [100.0]
