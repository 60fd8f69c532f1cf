"""Replica path on CPU with two gloo ranks: the shards of every unit count
cover each unit exactly once, and the timing reduction returns the largest
rank's value on every rank (the benchmark's max-over-ranks clock)."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2609_30644_gb300 import replicas
    dist = replicas.init("gloo")
    r, w, _ = replicas.env()
    covered = {n: list(replicas.shard(n, r, w)) for n in (0, 1, 7, 65536, 65537)}
    m = replicas.max_over_ranks(dist, 10.0 * (r + 1))
    replicas.barrier(dist)
    out.put((r, covered, m))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(m == 20.0 for _, _, m in res)
    for n in (0, 1, 7, 65536, 65537):
        units = res[0][1][n] + res[1][1][n]
        assert sorted(units) == list(range(n))
        assert abs(len(res[0][1][n]) - len(res[1][1][n])) <= 1


def test_single_rank_is_identity(monkeypatch):
    from paper_2609_30644_gb300 import replicas
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert replicas.init("gloo") is None
    assert replicas.max_over_ranks(None, 3.5) == 3.5
    assert list(replicas.shard(5, 0, 1)) == list(range(5))


COSTS = [5.0, 1.0, 9.0, 3.0, 3.0, 7.0, 2.0, 8.0, 1.0, 4.0, 6.0]


def _dispatch_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2609_30644_gb300 import replicas
    dist = replicas.init("gloo")
    r, w, _ = replicas.env()
    ran = []

    def solve(i):               # stands in for planning problem i on this rank's GPU
        ran.append(i)
        return {"problem": i, "rank": r, "cost": COSTS[i] * 10}

    res = replicas.dispatch(dist, COSTS, solve, r, w)
    out.put((r, replicas.assign(COSTS, w), ran, res))
    dist.destroy_process_group()


def test_dispatch_whole_problems_over_two_gloo_ranks():
    """Whole problems are assigned to ranks (one GPU each) by estimated cost;
    both ranks compute the same partition, each runs only its own problems,
    and every rank receives all results in problem order."""
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dispatch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, part0, ran0, out0), (r1, part1, ran1, out1) = res
    assert part0 == part1                              # same partition on both ranks
    assert sorted(ran0) == part0[0] and sorted(ran1) == part0[1]
    assert sorted(ran0 + ran1) == list(range(len(COSTS)))
    loads = [sum(COSTS[i] for i in part) for part in part0]
    assert abs(loads[0] - loads[1]) <= max(COSTS)
    assert out0 == out1
    assert [o["problem"] for o in out0] == list(range(len(COSTS)))
    assert all(o["rank"] == (0 if o["problem"] in part0[0] else 1) for o in out0)


def test_assign_single_rank_and_balance():
    from paper_2609_30644_gb300 import replicas
    assert replicas.assign(COSTS, 1) == [list(range(len(COSTS)))]
    parts = replicas.assign(COSTS, 4)
    assert sorted(i for p in parts for i in p) == list(range(len(COSTS)))
    loads = [sum(COSTS[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(COSTS)
    assert replicas.dispatch(None, [1.0, 2.0], lambda i: -i, 0, 1) == [0, -1]
