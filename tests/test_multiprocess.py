"""The N > 1 path of the benchmark on CPU: world-size-2 gloo process groups.

Every rank advances its own copy of the workload (replicas, no collective on
the data path); the only collective is the max over ranks of the timed region,
and rank 0 alone reports. The reference arm runs on rank 0 only.
"""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)
    ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    val = bench.whole_job_rate(world, 1000, 5, ms)
    dist.barrier()
    # the reference arm: only rank 0 does work and prints
    class A:
        workload = "flame1d_128_n9"
        ref_side = 3
        warmup = 0
        steps = 1
        gpus = world
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(A(), rank, world)
    q.put((rank, local_ms, ms, val, rc, buf.getvalue()))
    dist.destroy_process_group()


def test_two_rank_timing_and_reporting():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=240) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, local_ms, ms, val, rc, text in out:
        assert ms == 200.0                      # max over ranks, on every rank
        assert val == pytest.approx(2 * 1000 * 5 / 0.2)
        assert rc == 0
        if rank == 0:
            assert '"impl": "reference"' in text
        else:
            assert text == ""
