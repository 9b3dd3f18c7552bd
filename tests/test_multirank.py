"""The multi-GPU form of bench.py is replicas only: every rank decodes its own
copy of the workload and the job's rate is the ranks' units over the slowest
rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    mine = [120.0, 200.0][rank]                     # this rank's timed region, ms
    t = bench.max_over_ranks(mine, ws, "cpu")
    rate = bench.whole_job_rate(1_000_000, ws, t * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in res:
        assert t == 200.0
        assert rate == pytest.approx(2 * 1_000_000 / 0.2 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, workload, ref_seconds = 3, 3, "plain_uniform_bits_1e6", 1.0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
