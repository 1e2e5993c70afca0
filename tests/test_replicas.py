"""Multi-rank host logic (replicas only) on CPU with the gloo backend,
world size 2: distinct replica ids, max-over-ranks timing, whole-job rate."""
import os
import socket

import pytest

from paper_0707_1581_gb300 import replicas


def test_rank_info_defaults_and_env():
    assert replicas.rank_info({}) == replicas.RankInfo(0, 1, 0)
    assert replicas.rank_info({"RANK": "3", "WORLD_SIZE": "8", "LOCAL_RANK": "3"}) == replicas.RankInfo(3, 8, 3)


def test_replica_ids_are_distinct():
    ids = [replicas.replica_id(r) for r in range(8)]
    assert len(set(ids)) == 8
    with pytest.raises(ValueError):
        replicas.replica_id(-1)


def test_aggregate_is_weak_scaling():
    one = replicas.aggregate_mlups(512 ** 3, 100, 1, 0.4)
    two = replicas.aggregate_mlups(512 ** 3, 100, 2, 0.4)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(512 ** 3 * 100 / 0.4 / 1e6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        info = replicas.rank_info()
        m = replicas.max_over_ranks(times[rank], dist)
        rate = replicas.aggregate_mlups(1000, 10, info.world, m)
        out.put((rank, replicas.replica_id(info.rank), m, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_max_over_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    times = [0.25, 0.5]
    procs = [mp.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [0, 1]                 # one replica id per rank
    assert all(r[2] == 0.5 for r in res)                 # both ranks see the slowest time
    assert all(r[3] == pytest.approx(2 * 1000 * 10 / 0.5 / 1e6) for r in res)
