"""The multi-rank path of bench.py on the CPU: two gloo ranks on 127.0.0.1, as torchrun would start
them.  Each rank advances its own replica of the workload (no data-path collective), so what is
shared is the host-side bookkeeping: the barrier and the maximum of the ranks' timed region, and
the whole-job throughput computed from it."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), DFGKS_BENCH_GLOO="1")
    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (ws, rank, rank) and dist.get_backend() == "gloo"
    dist.barrier()
    local_ms = 100.0 + 25.0 * rank                  # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, w)
    out[rank] = (m, bench.replica_throughput(1000.0, w, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(rank_main, args=(ws, free_port(), out), nprocs=ws, join=True)
    assert out[0] == out[1]
    m, value = out[0]
    assert m == 125.0                               # the max over ranks, on every rank
    assert value == pytest.approx(1000.0 * ws / 0.125)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.replica_throughput(10.0, 1, 1000.0) == pytest.approx(10.0)
