"""The N > 1 host logic of bench.py on CPU: two gloo ranks, MAX of the timed regions,
whole-job rate over all ranks, and the reference arm printing on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, world)
    rate = bench.whole_job_rate(8 * 5, world, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, rate))


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, mx, rate in res:
        assert mx == 150.0
        assert abs(rate - 2 * 40 / 0.150) < 1e-9


def test_reference_arm_is_silent_off_rank_zero(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, n = 1, 1, 64
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
