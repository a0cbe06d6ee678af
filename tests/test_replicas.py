"""The multi-GPU path runs independent replicas: two ranks on the gloo
backend (CPU) agree on the slowest rank's time, each has its own seed, and
the whole-job rate counts the units of both ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2211_12867_gb300.replicas import ReplicaGroup
    grp = ReplicaGroup("gloo")
    ms = grp.max_over_ranks(10.0 + 5.0 * rank)      # rank 1 is the slower one
    grp.barrier()
    q.put((rank, grp.seed, ms, grp.job_rate(1000, ms / 1e3)))
    grp.close()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0, 1]                 # distinct seeds
    assert all(o[2] == 15.0 for o in out)                # max over ranks
    assert all(o[3] == pytest.approx(2 * 1000 / 0.015) for o in out)


def test_single_process_needs_no_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2211_12867_gb300.replicas import ReplicaGroup
    grp = ReplicaGroup("gloo")
    assert grp.world == 1 and grp.max_over_ranks(3.5) == 3.5 and grp.job_rate(10, 2.0) == 5.0
    grp.close()
