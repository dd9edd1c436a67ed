"""The multi-GPU logic of bench.py on the CPU: two gloo ranks (world_size 2) take disjoint
shards of the same workload, and the timing and solved counts reduce to whole-job numbers
(slowest rank's time, counts summed).  No GPU: the reductions run on CPU tensors."""
import hashlib
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(a):
    return hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest()


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        # whole-job reductions
        out["max"] = bench.max_over_ranks(1.5 + rank, world)
        out["sum"] = bench.sum_over_ranks(10 + rank, world)
        out["tp"] = bench.job_throughput(ok=4 + rank, total_ms=100.0 * (rank + 1), steps=2, world=world)
        # shards of the uneven batch and of the shared-A workload
        dct = bench.rank_problems("dct_batch_256", rank, count=3)
        out["dct"] = [(p.n, p.m, _digest(p.b), _digest(p.rows)) for p in dct]
        bf = bench.rank_problems("bf16_4096x16384_64rhs", rank, count=2)
        out["bf16"] = (_digest(bf[0].a_bf16), [_digest(p.b) for p in bf])
        gathered = [None] * world
        dist.all_gather_object(gathered, out)
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_reductions_give_whole_job_numbers(two_ranks):
    r0, r1 = two_ranks
    assert r0["max"] == r1["max"] == 2.5
    assert r0["sum"] == r1["sum"] == 21.0
    # (4 + 5) problems over the slowest rank's 200 ms for 2 steps = 9 / 0.1 s
    v, ms = r0["tp"]
    assert ms == 200.0 and abs(v - 90.0) < 1e-9 and r1["tp"] == r0["tp"]


def test_shards_are_disjoint_with_the_same_sizes(two_ranks):
    r0, r1 = two_ranks
    assert [x[:2] for x in r0["dct"]] == [x[:2] for x in r1["dct"]]  # weak scaling: same sizes
    assert not set(x[2] for x in r0["dct"]) & set(x[2] for x in r1["dct"])  # own data
    assert r0["bf16"][0] == r1["bf16"][0]  # one shared A
    assert not set(r0["bf16"][1]) & set(r1["bf16"][1])  # own right-hand sides


def test_rank_zero_shard_is_the_single_gpu_workload():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    a = bench.rank_problems("dct_batch_256", 0, count=2)
    b = W.make_workload("dct_batch_256", count=2)
    assert all(np.array_equal(x.b, y.b) and np.array_equal(x.rows, y.rows) for x, y in zip(a, b))


def test_phase_curve_takes_the_largest_half_successful_ratio():
    import bench
    cells = [(100, k) for k in range(1, 6)] + [(200, k) for k in range(1, 4)]
    succ = [1.0, 1.0, 0.5, 0.25, 0.75, 1.0, 0.0, 0.0]
    # per m: the largest k/m with a success fraction >= 1/2 (k = 5 for m = 100, k = 1 for m = 200)
    assert bench.phase_curve(cells, succ) == {"100": 0.05, "200": 0.005}


@pytest.mark.parametrize("workload", sorted(__import__("workloads").WORKLOADS))
def test_oracle_samples_stay_small(workload):
    """The CPU-baseline and reference legs time the oracle's direct solve (an m x m Woodbury
    factorisation per iteration): every workload's sample keeps m <= 4096 and n <= 16384 (a
    full-size m = 16384 sample ran ~20 min)."""
    import argparse
    import bench
    probs, desc = bench.oracle_sample_problems(argparse.Namespace(workload=workload))
    assert probs and desc
    assert max(p.m for p in probs) <= 4096 and max(p.n for p in probs) <= 16384, workload


def test_reference_arm_line():
    """bench.py --impl reference: the oracle on the host cores, one JSON line with the
    contract's keys (impl, metric, value, unit, cpu_baseline, e2e with zero copies)."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "dense_fp64_256x1024", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "dense_fp64_256x1024"


def test_oracle_extrapolation_to_the_batch():
    """The CPU baseline of the 256 batch: per-class times fitted by a power law in n and summed
    over every problem of the batch (measured classes at their mean time)."""
    import types
    import bench
    tf, a = bench.fit_class_times({4096: [1.0, 1.0], 8192: [8.0]})
    assert abs(a - 3.0) < 1e-12 and abs(tf(16384) - 64.0) < 1e-9 and abs(tf(65536) - 4096.0) < 1e-6
    probs = [types.SimpleNamespace(n=n) for n in (4096, 8192, 16384, 65536)]
    rate, a2, total = bench.extrapolated_batch_rate(probs, {4096: [1.0], 8192: [8.0]})
    assert abs(total - (1 + 8 + 64 + 4096)) < 1e-6 and abs(rate - 4 / total) < 1e-12
    # one measured class: the direct solve's cost model n^3
    _, a1 = bench.fit_class_times({4096: [2.0]})
    assert a1 == 3.0


def test_reference_arm_batch_line():
    """--impl reference on the 256 batch: one problem per step, extrapolated to the batch."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "dct_batch_256", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and 0 < line["value"] < 1.0
    assert line["cpu_baseline"]["extrapolated"] is True and line["cpu_baseline"]["value"] == line["value"]
    assert "n^3.00" in line["cpu_baseline"]["sample"]
