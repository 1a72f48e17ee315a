"""The multi-rank path of bench.py on CPU: two gloo ranks agree on the
slowest rank's time and on the whole-job throughput; the reference arm does
no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(ms, device="cpu")
    v = bench.job_value(512 ** 3, 10, m, world)
    torch.save((m, v), os.path.join(out, "r%d.pt" % rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [torch.load(tmp_path / ("r%d.pt" % r)) for r in range(world)]
    for m, v in res:
        assert m == 150.0
        assert v == pytest.approx(2 * 512 ** 3 * 10 / 0.150)


def test_single_process_time_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_value(100, 2, 1000.0, 1) == pytest.approx(200.0)


def test_reference_arm_idles_on_other_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
