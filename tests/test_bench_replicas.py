"""The multi-GPU path of bench.py is replicas only: every rank times its own
replica, the job time is the slowest rank's, and the whole-job rate sums the
replicas.  Checked with two gloo ranks on CPU (no GPU, no NCCL)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        # rank r took 100 (r + 1) ms for 10 steps of its replica
        total_ms, rate = bench.replica_timing(100.0 * (rank + 1), 10, world)
        # the reference arm runs on rank 0 only; the other ranks return without work or output
        printed = ""
        if rank != 0:
            buf = io.StringIO()
            with redirect_stdout(buf):
                bench.run_reference(None)
            printed = buf.getvalue()
        dist.barrier()
        out.put((rank, total_ms, rate, printed))
    finally:
        dist.destroy_process_group()


def test_replica_timing_and_reference_rank_rule():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, rate, printed in res:
        assert total_ms == pytest.approx(200.0)          # the slowest rank's time
        assert rate == pytest.approx(2 * 10 / 0.2)       # both replicas' steps over the job time
    assert res[1][3] == ""                                # rank 1 printed nothing


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_timing(250.0, 50, 1) == (250.0, pytest.approx(200.0))
