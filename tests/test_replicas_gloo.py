"""The multi-rank path of bench.py (replicas only: one independent
reconstruction per rank, no data-path collective) with two gloo ranks on
the CPU: the timing is the maximum over ranks, the whole-job rate counts the
units of every rank, every rank draws its own mock, and the reference arm
runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup("gloo")
    t_local = 2.0 + r            # rank 1 is the slower one
    t_max = bench.max_over_ranks(t_local, w)
    rate = bench.whole_job_rate(5, w, t_local)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((r, w, t_max, rate, bench.replica_seeds(r)))


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 3.0 for r in res)                  # max over ranks
    assert all(abs(r[3] - 2 * 5 / 3.0) < 1e-12 for r in res)  # all units / slowest rank
    assert res[0][4] != res[1][4]                          # independent replicas


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), 2, 1) is None
    assert capsys.readouterr().out == ""
