"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would start
them.  Each rank advances its own replica (weak scaling, no exchange on the
data path); the job's time is the slowest rank's, and only rank 0 prints."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench.dist_env() == (rank, world, rank)
        # the slowest rank sets the job time
        ms = [12.5, 20.0][rank]
        bench.rank_barrier(world)
        ms_max = bench.rank_max(ms, world, "cpu")
        value = bench.job_throughput(1000, 50, world, ms_max)
        # the reference arm: rank 0 alone runs and prints, the others return
        args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                 "--workload", "fcc", "--nc", "6"])
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(args, rank, world)
        out.put((rank, ms_max, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_bookkeeping():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, ms_max, value, printed = q.get(timeout=300)
        res[rank] = (ms_max, value, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        assert res[rank][0] == 20.0                       # max over ranks
        assert res[rank][1] == pytest.approx(1000 * 50 * 2 / 20.0e-3)
    assert '"impl": "reference"' in res[0][2]
    assert res[1][2] == ""
