"""Sharding one caller's batch over several GPUs (paper_1208_5435_gb300.distributed): the
cost-balanced partition, and the solve-then-gather logic on two gloo ranks on the CPU (the
rank-local GPU solve is replaced by a CPU stand-in with the same interface)."""
import os
import socket
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_problem_once_and_balances():
    from paper_1208_5435_gb300 import distributed as D
    import workloads as W
    sizes = W.batch_sizes(256, 1003)
    costs = [D.problem_cost(n, m) for n, m, _ in sizes]
    for world in (1, 2, 3, 8):
        shards = D.partition(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT: no rank exceeds the mean by more than the largest single problem
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6
    # deterministic, and the same on every call
    assert D.partition(costs, 4) == D.partition(costs, 4)
    # dense problems are costed by m n
    assert D.problem_cost(1024, 256, "dense") == 1024 * 256


def _fake_solve(ops, bs, taus, params):
    xs = [torch.full((o.n,), float(b[0]) * t, dtype=torch.float64) for o, b, t in zip(ops, bs, taus)]
    infos = [{"status": 0, "n": o.n, "tau": t} for o, t in zip(ops, taus)]
    return xs, infos


def _batch():
    ns = [4096, 65536, 8192, 16384, 4096, 32768, 8192]
    ops = [types.SimpleNamespace(n=n, m=n // 4, rows=None) for n in ns]
    bs = [torch.tensor([float(j + 1)]) for j in range(len(ns))]
    taus = [0.5 + j for j in range(len(ns))]
    return ops, bs, taus


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1208_5435_gb300 import distributed as D
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ops, bs, taus = _batch()
        calls = []

        def local(o, b, t, p):
            calls.append([x.n for x in o])
            return _fake_solve(o, b, t, p)

        xs, infos = D.solve_sharded(ops, bs, taus, None, local_solve=local)
        x0, i0 = D.solve_sharded(ops, bs, taus, None, local_solve=_fake_solve, gather_to=0)
        q.put((rank, calls, [x.tolist()[:1] for x in xs], infos, None if x0 is None else [x.tolist()[:1] for x in x0]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_disjoint_shards_and_gather_the_whole_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=600) for _ in range(2)])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ops, bs, taus = _batch()
    want_x, want_i = _fake_solve(ops, bs, taus, None)
    for rank, calls, xs, infos, x0 in res:
        # one local solve per rank, on disjoint shards that together hold the batch
        assert len(calls) == 1
        assert [x[0] for x in xs] == [float(w[0]) for w in want_x] and infos == want_i
        assert (x0 is not None) == (rank == 0)
    n0, n1 = res[0][1][0], res[1][1][0]
    assert sorted(n0 + n1) == sorted(o.n for o in ops)
    assert res[0][4] == res[0][2]
