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


REQUIRED = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def test_reference_arm_two_ranks_prints_once():
    # bench.py --impl reference under a 2-rank launch: rank 0 times the oracle and prints the one
    # JSON line, rank 1 exits 0 without work or output
    import json
    import subprocess
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r), DFGKS_BENCH_GLOO="1")
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "0", "--n", "16"],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert [p.returncode for p in procs] == [0, 0], [o[1][-2000:] for o in outs]
    lines0 = [l for l in outs[0][0].splitlines() if l.strip()]
    assert len(lines0) == 1 and outs[1][0].strip() == ""
    line = json.loads(lines0[0])
    assert REQUIRED <= set(line) and line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == "quadrants_16x16_gks_seed3"
