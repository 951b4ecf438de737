"""Multi-process replica path of bench.py on CPU (gloo, world size 2).

Queries are independent, so N GPUs run N replicas with no collective on the
data path; the only exchange is the host-side max of the ranks' times.  These
tests run that host logic as two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(1.5 + rank, "cpu")
    seeds = bench.replica_seeds(rank, 7, 64)
    out.put((rank, slowest, seeds, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_share_the_slowest_time_and_draw_disjoint_seeds():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    assert [g[1] for g in got] == [2.5, 2.5]           # max over ranks on every rank
    assert [g[3][:2] for g in got] == [(0, 2), (1, 2)]  # RANK / WORLD_SIZE read from the env
    s0, s1 = set(got[0][2]), set(got[1][2])
    assert len(s0) == len(s1) == 64 and not (s0 & s1)


def test_job_throughput_counts_every_rank():
    import bench
    assert bench.job_throughput(640, 2, 0.5) == 2560.0
    assert bench.max_over_ranks(3.0, "cpu") == 3.0  # no process group: identity


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        train_frames = None
        steps = 1
        warmup = 0
        gpus = 2
    assert bench.run_reference(A()) is None
