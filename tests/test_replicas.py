"""The multi-GPU path runs independent replicas (the work shards over sources and slices
with no exchange): two gloo ranks on the CPU check the host logic of the bench's job
aggregation (the slowest rank's time, units of every rank) and that only rank 0 of the
reference arm works and prints."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)          # rank 1 is the slow one
        value = bench.job_value(1000, 4, world, ms)
        out = io.StringIO()
        with redirect_stdout(out):
            if rank != 0:
                bench.run_reference(type("A", (), {"gpus": world, "steps": 1, "warmup": 0})())
        q.put((rank, ms, value, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, printed in res:
        assert ms == 15.0                                   # max over ranks
        assert value == pytest.approx(1000 * 4 * 2 / 0.015)  # both replicas' units over the slowest time
        if rank == 1:
            assert printed == ""                            # the reference arm works on rank 0 only
