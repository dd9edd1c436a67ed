"""Benchmark: mfIPM solves/sec at kkt_rel <= 1e-6, batched vs plain, on GB300.

Workload (default): 256 independent partial-DCT problems, n uniform in {2^12..2^16},
m = n/4, k uniform in [n/100, n/20] N(0,1) spikes, sigma = 1e-3 noise, tau =
0.01*||A^T b||_inf (workloads.WORKLOADS["dct_batch_256"]).  One step = one
mfipm_solve_batched call over the whole batch (one persistent launch).  Inputs are
resident in HBM when the timed region starts; L2 is flushed (a 512 MiB write) before
every timed step.  The "plain" leg solves the same problems one mfipm_solve call at a
time.  The e2e leg goes through the public API with pinned host inputs and outputs.

N > 1 GPUs (torchrun): every rank solves its own batch (weak scaling, no collective on
the data path); value = problems solved by all ranks / max-over-ranks time.

--impl reference times the CPU oracle (direct-solve float64 IPM) on a bounded sample of
the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

KKT_GATE = 1e-6
METRIC = "mfIPM solves/sec at KKT resid 1e-6 (batched vs plain); A,A^T GB/s vs HBM peak"
UNIT = "solves/s"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dct_batch_256")
    ap.add_argument("--count", type=int, default=None, help="truncate the batch (smaller profiling runs)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------- N GPUs
# One process per GPU; each solves its own shard of the workload (same sizes, its own random
# stream), so per-GPU work is fixed as N grows (weak scaling) and nothing is exchanged on
# the data path.  Only the timing and the solved counts are reduced, once, after the run.
RANK_STRIDE = 100000


def rank_problems(workload, rank, count=None):
    """This rank's shard: the workload's problems with the random streams of rank r."""
    return W.make_workload(workload, count=count, offset=rank * RANK_STRIDE)


def max_over_ranks(x, world, device="cpu"):
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device="cpu"):
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_throughput(ok, total_ms, steps, world, device="cpu"):
    """Whole-job units per second: solved units summed over ranks / slowest rank's time."""
    ok_all = sum_over_ranks(ok, world, device)
    ms = max_over_ranks(total_ms, world, device)
    return ok_all / (ms / steps / 1e3), ms


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mfipm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- reference arm
def oracle_sample_problems(args):
    """Smallest-class problems of the workload: the oracle's direct Newton solves grow with m^3."""
    if args.workload in ("dct_batch_256", "haar_batch_256"):
        probs = [p for p in W.make_workload(args.workload) if p.n == 4096]
        return probs, f"problems of the n=4096, m=1024 class of {args.workload}"
    if W.WORKLOADS[args.workload]["kind"] == "scaling":
        return W.make_workload(args.workload), "the whole size sweep n = 2^5 .. 2^12"
    if W.WORKLOADS[args.workload]["kind"] == "phase":
        cells = W.phase_cells()
        probs = W.make_workload(args.workload)
        pick = [j for j, (m, k) in enumerate(cells) if k == max(1, m // 10)]
        return [probs[j] for j in pick], "trial 0 of the cells k = m/10 (m = 100..900) of the phase-transition grid"
    probs = W.make_workload(args.workload, count=2)
    if probs[0].kind == "dct" and probs[0].n > 4096:
        # the direct solve grows with m^3: the same workload scaled to n = 4096 (same m/n, k/n)
        probs = W.make_workload(args.workload, count=2, scale_n=4096)
        return probs, f"{args.workload} scaled to n = 4096 (m = {probs[0].m}, k = {int((probs[0].x_hat != 0).sum())})"
    return probs, f"first problems of {args.workload}"


def time_oracle(probs, budget_s, tol=1e-10):
    from oracle import mfipm_oracle as O
    t0 = time.perf_counter()
    done = 0
    for p in probs:
        op = (O.Operator.from_dense(p.A) if p.kind == "dense" else
              O.Operator.from_haar_rows(p.n, p.rows) if p.kind == "haar" else O.Operator.from_dct_rows(p.n, p.rows))
        O.ipm(op, p.b, p.tau, O.OracleParams(tol=tol))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


BATCH_WORKLOADS = ("dct_batch_256", "haar_batch_256")
ORACLE_CLASSES = (4096, 8192)   # the classes of the batch whose direct solve fits a few seconds


def oracle_op(p):
    from oracle import mfipm_oracle as O
    return (O.Operator.from_dense(p.A) if p.kind == "dense" else
            O.Operator.from_haar_rows(p.n, p.rows) if p.kind == "haar" else O.Operator.from_dct_rows(p.n, p.rows))


def fit_class_times(times):
    """Per-class oracle time t(n) = t0 (n / n0)^a fitted on log-log through the measured classes
    (a from the measured pair; with one class a = 3, the Woodbury direct solve's m^2 n + m^3 cost
    at m = n/4).  Returns (t(n) function, a)."""
    ns = sorted(times)
    n0, t0 = ns[0], float(np.mean(times[ns[0]]))
    if len(ns) >= 2:
        n1, t1 = ns[-1], float(np.mean(times[ns[-1]]))
        a = float(np.log(t1 / t0) / np.log(n1 / n0))
    else:
        a = 3.0
    return (lambda n: t0 * (n / n0) ** a), a


def extrapolated_batch_rate(probs, times):
    """Solves/s of the oracle on the WHOLE batch, extrapolated from the measured per-class times."""
    tf, a = fit_class_times(times)
    total = sum(float(np.mean(times[p.n])) if p.n in times else tf(p.n) for p in probs)
    return len(probs) / total, a, total


def stratified_oracle(probs, budget_s, tol=1e-10):
    """Time the oracle on the first problem of each reachable class of the batch (smallest first,
    while the budget lasts).  Returns ({n: [seconds]}, {batch index: oracle x})."""
    from oracle import mfipm_oracle as O
    times, xs = {}, {}
    # one untimed solve of the smallest class first: loading the linear-algebra libraries and
    # starting their threads is not the oracle's cost per problem
    j0 = next((j for n in ORACLE_CLASSES for j, p in enumerate(probs) if p.n == n), None)
    if j0 is not None:
        O.ipm(oracle_op(probs[j0]), probs[j0].b, probs[j0].tau, O.OracleParams(tol=tol))
    t_start = time.perf_counter()
    for n in ORACLE_CLASSES:
        j = next((j for j, p in enumerate(probs) if p.n == n), None)
        if j is None:
            continue
        if times and time.perf_counter() - t_start > budget_s:
            break
        t0 = time.perf_counter()
        res = O.ipm(oracle_op(probs[j]), probs[j].b, probs[j].tau, O.OracleParams(tol=tol))
        times[n] = [time.perf_counter() - t0]
        xs[j] = res.x
    return times, xs


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload in BATCH_WORKLOADS:
        return run_reference_batch(args)
    probs, desc = oracle_sample_problems(args)
    tol = W.WORKLOADS[args.workload].get("tol", 1e-10)
    # one problem per step; the size sweep of pcg_vs_direct is one step as in the GPU leg
    step = probs if W.WORKLOADS[args.workload]["kind"] == "scaling" else probs[:1]
    for _ in range(args.warmup):
        time_oracle(step, 1e9, tol)
    done, secs = 0, 0.0
    for _ in range(args.steps):
        d, s = time_oracle(step, 1e9, tol)
        done += d
        secs += s
    value = done / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{len(step)} problem(s) per step: {desc}; direct-solve float64 IPM, tol {tol:g}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    """The oracle on the 256-problem batch: each timed step solves one problem, taking the
    reachable classes (n = 4096, 8192) in turn; the value is the batch's solves/s extrapolated
    from the per-class mean times with a fitted power law (the larger classes are out of a
    direct solve's reach in minutes)."""
    from oracle import mfipm_oracle as O
    probs = W.make_workload(args.workload)
    firsts = [next(j for j, p in enumerate(probs) if p.n == n) for n in ORACLE_CLASSES if any(p.n == n for p in probs)]
    for _ in range(args.warmup):
        p = probs[firsts[0]]
        O.ipm(oracle_op(p), p.b, p.tau, O.OracleParams(tol=1e-10))
    times, secs = {}, 0.0
    for i in range(args.steps):
        p = probs[firsts[i % len(firsts)]]
        t0 = time.perf_counter()
        O.ipm(oracle_op(p), p.b, p.tau, O.OracleParams(tol=1e-10))
        dt = time.perf_counter() - t0
        times.setdefault(p.n, []).append(dt)
        secs += dt
    value, a, total = extrapolated_batch_rate(probs, times)
    desc = (f"one problem per step, classes n = {sorted(times)} in turn (mean s: "
            f"{ {n: round(float(np.mean(t)), 3) for n, t in times.items()} }); direct-solve float64 IPM, tol 1e-10; "
            f"extrapolated to all {len(probs)} problems by t(n) ~ n^{a:.2f} ({total:.0f} s per batch); an upper "
            f"bound on the oracle's throughput: its m^2 n Woodbury term takes over only above these sizes")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": desc, "extrapolated": True},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": desc, "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- ours
PCG_BYTES_PER_INDEX = 96     # per PCG iteration: the 2n-form float32 PCG, 12 float32 2n-streams
OUTER_BYTES_PER_INDEX = 160  # per outer (IPM) iteration: the float64 outer passes


def algorithmic_bytes(probs, infos):
    """Algorithmic bytes of one launch by the roofline model of the partial-DCT solver: per
    index, 96 B per PCG iteration (the float32 PCG state of the 2n system -- x, r, p,
    Theta^-1 and the operator's w -- streamed as 12 float32 2n-vectors) and 160 B per outer
    IPM iteration (the float64 iterate, residual and direction passes).  These are the bytes a
    design with every vector in HBM moves; the shared-memory operator and the L2-resident
    state make the measured DRAM traffic lower, so achieved / peak can exceed what HBM alone
    would allow only by staying on chip."""
    tot = 0
    for p, i in zip(probs, infos):
        tot += p.n * (PCG_BYTES_PER_INDEX * i["pcg_iters"] + OUTER_BYTES_PER_INDEX * i["ipm_iters"])
    return tot


def pcg_fft_flops(probs, infos):
    """Float32 flops of the PCG's operator products: one A^T A w per PCG iteration, a forward and
    an inverse complex FFT of L = n/2 points (5 L log2 L each, the radix-2 count)."""
    return sum(i["pcg_iters"] * 2 * 5 * (p.n // 2) * np.log2(p.n // 2) for p, i in zip(probs, infos))


def operator_bytes(probs, infos):
    """The operator's algorithmic bytes: each product with A or A^T reads its input and writes its
    output (8 bytes per float64 or per float32 pair of n entries: 4n per product)."""
    return sum(4 * p.n * i["n_mat"] for p, i in zip(probs, infos))


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1208_5435_gb300 as M
    from paper_1208_5435_gb300 import build as B

    torch.cuda.set_device(local_rank)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    B.build()
    L = M.lib()
    dev = torch.device("cuda", local_rank)
    if W.WORKLOADS[args.workload]["kind"] == "phase":
        return run_phase(args, rank, world, local_rank)
    if W.WORKLOADS[args.workload]["kind"] == "scaling":
        return run_scaling(args, rank, world, local_rank)
    probs = rank_problems(args.workload, rank, count=args.count)
    if probs[0].a_bf16 is not None:
        return run_bf16(args, rank, world, local_rank, probs)
    if args.workload == "dct_adjoint_32x1M":
        return run_adjoint(args, rank, world, local_rank, probs)
    if probs[0].kind == "dense":
        return run_dense(args, rank, world, local_rank, probs)
    Op = M.PartialHaar if probs[0].kind == "haar" else M.PartialDCT
    ops = [Op(p.n, torch.from_numpy(p.rows).to(dev)) for p in probs]
    bs = [torch.from_numpy(p.b).to(dev) for p in probs]
    taus = [p.tau for p in probs]
    params = M.SolverParams()
    ws = torch.empty(M.workspace_bytes(ops, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return M.solve_batched(ops, bs, taus, params, ws=ws)

    # the autotuner picks the cluster size and the single-CTA limit on this batch (untimed);
    # it tunes the partial-DCT kernel only
    if Op is M.PartialDCT:
        tuning = M.autotune(ops, bs, taus, params, ws=ws)[2]
    else:
        tuning = {"cluster_size": 0, "cta_max_n": 0, "candidates": 0, "best_ms": None, "default_ms": None}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L.mfipm_set_timing(1)
    kern_ms, step_ms, infos = [], [], None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with RooflineRange(s_ == args.steps - 1):
                e0.record(stream)
                xs, infos = step()
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(L.mfipm_last_kernel_ms())
    torch.cuda.synchronize()
    launches_per_step = last_call_launches(L)
    if world > 1:
        torch.distributed.barrier()
    L.mfipm_set_timing(0)
    ok = sum(1 for i in infos if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    value, total_ms = job_throughput(ok, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps

    # plain: the same problems, one mfipm_solve each (one timed pass)
    plain = None
    if not args.no_plain:
        wsp = torch.empty(max(M.workspace_bytes([o], params) for o in ops), dtype=torch.uint8, device=dev)
        def solve_one(o, b_, t_):
            # a problem that ends NOT_CONVERGED or NUMERIC counts as unsolved; other codes raise
            x_, d_ = M.solve(o, b_, t_, params, ws=wsp, raise_on_failure=False)
            if d_["return_code"] not in (0, 2, 3):
                raise RuntimeError(f"mfipm_solve returned {d_['return_code']}")
            return x_, d_

        for j in range(min(3, len(ops))):
            solve_one(ops[j], bs[j], taus[j])
        torch.cuda.synchronize()
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pinfo = [solve_one(o, b_, t_)[1] for o, b_, t_ in zip(ops, bs, taus)]
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        pok = sum(1 for i in pinfo if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
        plain = {"value": pok / (pms / 1e3), "unit": UNIT, "ms_per_batch": pms,
                 "solved": pok, "kernel_launches_per_problem": 5}

    # e2e: public API from pinned host buffers, x read back, every step
    hb = [torch.from_numpy(p.b).pin_memory() for p in probs]
    hr = [torch.from_numpy(p.rows).pin_memory() for p in probs]
    hx = [torch.empty(p.n, dtype=torch.float64).pin_memory() for p in probs]
    h2d = sum(t.numel() * 8 for t in hb) + sum(t.numel() * 8 for t in hr)
    d2h = sum(t.numel() * 8 for t in hx)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dops = [Op(p.n, r.to(dev, non_blocking=True)) for p, r in zip(probs, hr)]
        dbs = [b_.to(dev, non_blocking=True) for b_ in hb]
        xs_, inf_ = M.solve_batched(dops, dbs, taus, params, ws=ws)
        for h, d in zip(hx, xs_):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_ok = sum(1 for i in inf_ if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    e2e_value, _ = job_throughput(e2e_ok, sum(e2e_ms), args.steps, world, dev)

    # the same batch with the native float64 outer loop (mfipm_outer = MFIPM_OUTER_FP64)
    fp64_outer = None
    if Op is M.PartialDCT:
        p64 = M.SolverParams(outer=1)
        M.solve_batched(ops, bs, taus, p64, ws=ws)
        torch.cuda.synchronize()
        f_ms, f_inf = [], None
        for _ in range(min(args.steps, 3)):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, f_inf = M.solve_batched(ops, bs, taus, p64, ws=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            f_ms.append(e0.elapsed_time(e1))
        f_ok = sum(1 for i in f_inf if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
        f_value, f_tot = job_throughput(f_ok, sum(f_ms), len(f_ms), world, dev)
        fp64_outer = {"value": f_value, "unit": UNIT, "ms_per_step": f_tot / len(f_ms), "solved": f_ok,
                      "dtype": "f32 PCG / f64 outer", "kkt_max": max(i["kkt_rel"] for i in f_inf),
                      "ipm_mean": statistics.mean(i["ipm_iters"] for i in f_inf),
                      "pcg_mean": statistics.mean(i["pcg_iters"] for i in f_inf)}

    # roofline of the dominant kernel (the persistent solver kernel)
    peak, peak_kind = measured_peaks()
    kms = statistics.mean(kern_ms)
    abytes = algorithmic_bytes(probs, infos)
    achieved = abytes / (kms / 1e3) / 1e9
    obytes = operator_bytes(probs, infos)
    tj = load_traffic(args.workload)
    traffic = tj["bytes_per_launch"] if tj and tj.get("problems") == len(probs) else None
    fma = ctypes.c_double(0.0)
    fma_peak = fma.value if L.mfipm_fp32_fma_peak(ctypes.byref(fma), None) == 0 else None
    fft_tf = pcg_fft_flops(probs, infos) / (kms / 1e3) / 1e12
    if rank != 0:
        return
    cpu, err_vs_oracle = None, None
    if not args.no_cpu and world == 1:
        if args.workload in BATCH_WORKLOADS:
            ctimes, cxs = stratified_oracle(probs, 20.0)
            crate, a, ctot = extrapolated_batch_rate(probs, ctimes)
            cpu = {"value": crate, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "extrapolated": True,
                   "sample": (f"one problem of each class n = {sorted(ctimes)} timed (s: "
                              f"{ {n: round(t[0], 2) for n, t in ctimes.items()} }); direct-solve float64 IPM, "
                              f"tol 1e-10; extrapolated to all {len(probs)} problems by t(n) ~ n^{a:.2f} "
                              f"({ctot:.0f} s per batch); an upper bound on the oracle's throughput: its "
                              f"m^2 n Woodbury term takes over only above these sizes")}
            err_vs_oracle = {str(probs[j].n): float(np.linalg.norm(xs[j].cpu().numpy() - xo) / np.linalg.norm(xo))
                             for j, xo in cxs.items()}
        else:
            sp, desc = oracle_sample_problems(args)
            d, s_ = time_oracle(sp, 15.0)
            cpu = {"value": d / s_, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                   "sample": f"{d} problem(s) in {s_:.1f} s: {desc}; direct-solve float64 IPM, tol 1e-10"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 PCG / double-float outer (~48-bit)", "data": "synthetic",
        "config": {"workload": args.workload, "problems": len(probs), "sum_n": int(sum(p.n for p in probs)),
                   "tol": params.tol, "tol_pcg": params.tol_pcg, "l2": "flushed (512 MiB write) before each step",
                   "solved_at_kkt_1e-6": ok,
                   "tuned": {"cluster_size": tuning["cluster_size"], "cta_max_n": tuning["cta_max_n"],
                             "candidates": tuning["candidates"], "best_ms": tuning["best_ms"],
                             "default_ms": tuning["default_ms"]}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "ipm_kernel (persistent, one cluster per problem)", "kernel_ms": kms,
                     "algorithmic_bytes": abytes,
                     "bytes_model": f"{PCG_BYTES_PER_INDEX} B per index per PCG iteration + "
                                    f"{OUTER_BYTES_PER_INDEX} B per index per IPM iteration"},
        "alu": {"bound": "alu", "achieved": fft_tf, "peak": fma_peak, "unit": "TFLOP/s",
                "frac": (fft_tf / fma_peak) if fma_peak else None, "peak_kind": "measured (FP32 FMA loop)",
                "counts": "float32 FFT flops of the PCG products only (5 L log2 L per L = n/2 point FFT, "
                          "two per product); the double-float residual chains are not counted"},
        "operator": {"gbs": obytes / (kms / 1e3) / 1e9, "frac_of_hbm": obytes / (kms / 1e3) / 1e9 / peak,
                     "n_mat_total": int(sum(i["n_mat"] for i in infos))},
        "fp64_outer": fp64_outer,
        "error_vs_oracle": {"relx_by_n": err_vs_oracle, "kkt_max": max(i["kkt_rel"] for i in infos)},
        "plain": plain,
        "batched_over_plain": (value / world / plain["value"]) if plain else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu,
        "gpu_launches": launches_per_step * args.steps,  # counted by the library per solve call
        "clocks": clk.summary(),
        "iterations": {"ipm_mean": statistics.mean(i["ipm_iters"] for i in infos),
                       "pcg_mean": statistics.mean(i["pcg_iters"] for i in infos),
                       "correctors_total": int(sum(i["correctors"] for i in infos)),
                       "correctors_max": int(max(i["correctors"] for i in infos)),
                       "kkt_max": max(i["kkt_rel"] for i in infos)},
    }
    print(json.dumps(line), flush=True)


PHASE_RE = 1e-5  # reconstruction counted as a success when ||x - x_hat|| / ||x_hat|| <= 1e-5 (Sec. 5.8)


def phase_curve(cells, success):
    """Per m: the largest k/m whose success fraction over the trials is >= 1/2 (Sec. 5.8)."""
    out = {}
    for (m, k), s in zip(cells, success):
        if s >= 0.5:
            out[m] = max(out.get(m, 0.0), k / m)
    return {str(m): round(out.get(m, 0.0), 4) for m in sorted({m for m, _ in cells})}


def run_phase(args, rank, world, local_rank):
    """The phase-transition workload: one step = one mfipm_solve_batched call over one trial of
    every (m, k) cell (4500 noiseless partial-DCT problems, n = 1024).  Each timed step solves
    another trial (all trials resident in HBM before timing), so the steps also give the
    empirical phase transition: per m, the largest k/m solved to r.e. <= 1e-5 in at least
    half of the trials."""
    import torch
    import paper_1208_5435_gb300 as M

    dev = torch.device("cuda", local_rank)
    L = M.lib()
    w = W.WORKLOADS[args.workload]
    cells = W.phase_cells()[: args.count or None]
    base = rank * RANK_STRIDE
    trials = [W.make_workload(args.workload, count=args.count, offset=base + t) for t in range(args.steps)]
    dev_trials = []
    for probs in trials:
        ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows).to(dev)) for p in probs]
        bs = [torch.from_numpy(p.b).to(dev) for p in probs]
        dev_trials.append((ops, bs, [p.tau for p in probs]))
    params = M.SolverParams(tol=w["tol"])
    ws = torch.empty(M.workspace_bytes(dev_trials[0][0], params), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ops0, bs0, taus0 = dev_trials[0]
    tuning = M.autotune(ops0, bs0, taus0, params, ws=ws)[2]
    for _ in range(args.warmup):
        M.solve_batched(ops0, bs0, taus0, params, ws=ws)
    torch.cuda.synchronize()
    L.mfipm_set_timing(1)
    step_ms, kern_ms, results = [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for s_, (ops, bs, taus) in enumerate(dev_trials):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with RooflineRange(s_ == args.steps - 1):
                e0.record(stream)
                xs, infos = M.solve_batched(ops, bs, taus, params, ws=ws)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(L.mfipm_last_kernel_ms())
            results.append((xs, infos))
    torch.cuda.synchronize()
    launches_per_step = last_call_launches(L)
    if world > 1:
        torch.distributed.barrier()
    L.mfipm_set_timing(0)
    ok = sum(1 for _, infos in results for i in infos if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    value, total_ms = job_throughput(ok / args.steps, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    # reconstruction success per cell over this rank's trials (after the timed region)
    succ = np.zeros(len(cells))
    for probs, (xs, _) in zip(trials, results):
        for j, (p, x) in enumerate(zip(probs, xs)):
            xh = x.cpu().numpy()
            succ[j] += np.linalg.norm(xh - p.x_hat) <= PHASE_RE * np.linalg.norm(p.x_hat)
    succ_all = succ.copy()
    if world > 1:
        t = torch.from_numpy(succ_all).to(dev)
        torch.distributed.all_reduce(t)
        succ_all = t.cpu().numpy()
    frac = succ_all / (args.steps * world)

    # e2e: trial 0 through the public API from pinned host buffers, x read back
    probs0 = trials[0]
    hb = [torch.from_numpy(p.b).pin_memory() for p in probs0]
    hr = [torch.from_numpy(p.rows).pin_memory() for p in probs0]
    hx = [torch.empty(p.n, dtype=torch.float64).pin_memory() for p in probs0]
    h2d = sum(t.numel() * 8 for t in hb) + sum(t.numel() * 8 for t in hr)
    d2h = sum(t.numel() * 8 for t in hx)
    e2e_ms = []
    for it in range(1 + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dops = [M.PartialDCT(p.n, r.to(dev, non_blocking=True)) for p, r in zip(probs0, hr)]
        dbs = [b_.to(dev, non_blocking=True) for b_ in hb]
        xs_, inf_ = M.solve_batched(dops, dbs, taus0, params, ws=ws)
        for h, d in zip(hx, xs_):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_ok = sum(1 for i in inf_ if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    e2e_value, _ = job_throughput(e2e_ok, sum(e2e_ms), args.steps, world, dev)

    peak, peak_kind = measured_peaks()
    infos_last = results[-1][1]
    kms = kern_ms[-1]
    abytes = algorithmic_bytes(trials[-1], infos_last)
    tj = load_traffic(args.workload)
    traffic = tj["bytes_per_launch"] if tj and tj.get("problems") == len(cells) else None
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        sp, desc = oracle_sample_problems(args)
        d, s = time_oracle(sp, 15.0, w["tol"])
        cpu = {"value": d / s, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{d} problem(s) in {s:.1f} s: {desc}; direct-solve float64 IPM, tol {w['tol']:g}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 PCG / double-float outer (~48-bit)", "data": "synthetic",
        "config": {"workload": args.workload, "problems": len(cells), "n": w["n"],
                   "cells": "m = 100..900 step 100, k = 1..m", "tau": "1e-6 ||A^T b||_inf, noiseless b",
                   "trials": args.steps * world, "tol": params.tol,
                   "l2": "flushed (512 MiB write) before each step", "solved_at_kkt_1e-6": ok,
                   "tuned": {"cluster_size": tuning["cluster_size"], "cta_max_n": tuning["cta_max_n"],
                             "candidates": tuning["candidates"]}},
        "roofline": {"bound": "hbm", "achieved": abytes / (kms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": abytes / (kms / 1e3) / 1e9 / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "ipm_kernel (persistent, one CTA per problem)", "kernel_ms": kms,
                     "algorithmic_bytes": abytes},
        "phase_transition": {"success_re": PHASE_RE, "k_over_m_at_50pct": phase_curve(cells, frac),
                             "successes": int(succ_all.sum()), "solves": len(cells) * args.steps * world,
                             "processed_per_s": len(cells) * world / (ms_per_step / 1e3)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu,
        "gpu_launches": launches_per_step * args.steps,  # counted by the library per solve call
        "clocks": clk.summary(),
        "iterations": {"ipm_mean": statistics.mean(i["ipm_iters"] for i in infos_last),
                       "pcg_mean": statistics.mean(i["pcg_iters"] for i in infos_last),
                       "kkt_max": max(i["kkt_rel"] for i in infos_last)},
    }
    print(json.dumps(line), flush=True)


def direct_ipm_gpu(A, b, tau, tol=1e-10, max_iter=100, eta=0.995):
    """Comparison arm of the PCG-against-direct leg (Sec. 5.7) on the same GPU: the
    Algorithm of Sec. 5.1 (sigma1/sigma2/sigma3, alpha_bar, alpha_tilde as the library's
    defaults, readings R1-R8) with every Newton system of Eq. redNewtonA solved by a Cholesky
    factorisation (the vendor library's, through torch, float64) of the m x m matrix
    I + A (Theta_u + Theta_v) A^T (Sherman-Morrison-Woodbury).  Not the library's path: the
    direct variant the paper compares its PCG against.  Returns (x, Newton directions)."""
    import torch
    n = A.shape[1]
    atb = A.T @ b
    c = torch.cat([tau - atb, tau + atb])
    z = torch.ones(2 * n, dtype=torch.float64, device=A.device)
    s = torch.ones_like(z)
    aP_prev = aD_prev = 1.0

    def FFt(v):
        t = A.T @ (A @ (v[:n] - v[n:]))
        return torch.cat([t, -t])

    def newton(d, r):
        th = 1.0 / d
        Mw = (A * (th[:n] + th[n:])[None, :]) @ A.T
        Mw.diagonal().add_(1.0)
        Lc = torch.linalg.cholesky(Mw)
        Dr = th * r
        y = torch.cholesky_solve((A @ (Dr[:n] - Dr[n:]))[:, None], Lc)[:, 0]
        aty = A.T @ y
        return Dr - th * torch.cat([aty, -aty])

    def step(v, dv):
        neg = dv < 0
        if not bool(neg.any()):
            return 1.0
        return min(1.0, eta * float(torch.min(-v[neg] / dv[neg])))

    k = 0
    for k in range(1, max_iter + 1):
        r = A @ (z[:n] - z[n:]) - b
        fz = s - c - FFt(z)
        mu = float(z @ s) / (2 * n)
        P = tau * float(z.sum()) + 0.5 * float(r @ r)
        if float(z @ s) / (1.0 + abs(P)) <= tol:
            break
        sigma = 0.5 if (k != 1 and (aP_prev <= 0.5 or aD_prev <= 0.5)) else 0.1
        d = s / z
        fs = sigma * mu - z * s
        dz = newton(d, fz + fs / z)
        ds = fs / z - d * dz
        aP, aD = step(z, dz), step(s, ds)
        if aP <= 0.1 or aD <= 0.1:
            zt, st = z + aP * dz, s + aD * ds
            fzt = st - c - FFt(zt)
            fst = 0.8 * float(zt @ st) / (2 * n) - zt * st
            dz2 = newton(d, fzt + fst / z)
            dz, ds = dz + dz2, ds + fst / z - d * dz2
            aP, aD = step(z, dz), step(s, ds)
        z, s = z + aP * dz, s + aD * ds
        aP_prev, aD_prev = aP, aD
    return z[:n] - z[n:], k - 1


def run_scaling(args, rank, world, local_rank):
    """PCG against a direct solver (Sec. 5.7): one Gaussian problem per n = 2^5..2^12 (m = n/4,
    tau = 1e-3, noiseless).  One step = one mfipm_solve per size, in turn (float64 PCG in the
    persistent kernel).  Beside each size: the IPM iterations of the oracle's float64 IPM with
    exact (direct) Newton directions and its host time, the paper's comparison of iteration
    counts and of time growth."""
    import torch
    import paper_1208_5435_gb300 as M

    dev = torch.device("cuda", local_rank)
    L = M.lib()
    probs = rank_problems(args.workload, rank, count=args.count)
    params = M.SolverParams()
    ops = [M.Dense(torch.from_numpy(p.A).to(dev)) for p in probs]
    bs = [torch.from_numpy(p.b).to(dev) for p in probs]
    ws = torch.empty(max(M.workspace_bytes([o], params) for o in ops), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for o, b_, p in zip(ops, bs, probs):
            M.solve(o, b_, p.tau, params, ws=ws)
    torch.cuda.synchronize()
    L.mfipm_set_timing(1)
    per = [[] for _ in probs]
    kern_last, infos, xs_last = [0.0] * len(probs), [None] * len(probs), [None] * len(probs)
    step_ms = []
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with RooflineRange(s_ == args.steps - 1):
                e0.record(stream)
                for j, (o, b_, p) in enumerate(zip(ops, bs, probs)):
                    ej = torch.cuda.Event(enable_timing=True)
                    ej.record(stream)
                    xs_last[j], infos[j] = M.solve(o, b_, p.tau, params, ws=ws)
                    kern_last[j] = L.mfipm_last_kernel_ms()
                    per[j].append((ej, torch.cuda.Event(enable_timing=True)))
                    per[j][-1][1].record(stream)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    L.mfipm_set_timing(0)
    ok = sum(1 for i in infos if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    value, total_ms = job_throughput(ok, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    gpu_ms = [statistics.median(a.elapsed_time(b_) for a, b_ in ev) for ev in per]

    # e2e: A and b of every size from pinned host memory, x read back
    hA = [torch.from_numpy(p.A).pin_memory() for p in probs]
    hb = [torch.from_numpy(p.b).pin_memory() for p in probs]
    hx = [torch.empty(p.n, dtype=torch.float64).pin_memory() for p in probs]
    e2e_ms = []
    for it in range(1 + args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_ok = 0
        for a_, b_, h, p in zip(hA, hb, hx, probs):
            xe, ie = M.solve(M.Dense(a_.to(dev, non_blocking=True)), b_.to(dev, non_blocking=True), p.tau, params, ws=ws)
            h.copy_(xe, non_blocking=True)
            e2e_ok += ie["status"] == 0 and ie["kkt_rel"] <= KKT_GATE
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value, _ = job_throughput(e2e_ok, sum(e2e_ms), args.steps, world, dev)
    peak, peak_kind = measured_peaks()
    big = len(probs) - 1
    abytes = infos[big]["n_mat"] * probs[big].m * probs[big].n * 8
    tj = load_traffic(args.workload)
    traffic = tj["bytes_per_launch"] if tj else None
    if rank != 0:
        return
    # the direct variant on the same GPU (vendor Cholesky, float64), per size: the paper's
    # comparison of time growth, now on one machine
    direct = []
    for p in probs:
        Ad, bd = torch.from_numpy(p.A).to(dev), torch.from_numpy(p.b).to(dev)
        direct_ipm_gpu(Ad, bd, p.tau, params.tol)  # warm (library handles, workspace)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd, itd = direct_ipm_gpu(Ad, bd, p.tau, params.tol)
        torch.cuda.synchronize()
        direct.append((1e3 * (time.perf_counter() - t0), itd, xd.cpu().numpy()))
    # the oracle with direct Newton solves, per size (host), within a bounded budget
    rows, cpu = [], None
    from oracle import mfipm_oracle as O
    t_all, done = 0.0, 0
    for j, p in enumerate(probs):
        row = {"n": p.n, "m": p.m, "k": int(np.count_nonzero(p.x_hat)), "gpu_ms": gpu_ms[j],
               "gpu_ipm_iters": infos[j]["ipm_iters"], "gpu_pcg_iters": infos[j]["pcg_iters"],
               "gpu_kkt_rel": infos[j]["kkt_rel"], "direct_gpu_ms": direct[j][0],
               "direct_gpu_ipm_iters": direct[j][1],
               "x_rel_vs_direct_gpu": float(np.linalg.norm(xs_last[j].cpu().numpy() - direct[j][2])
                                            / max(np.linalg.norm(direct[j][2]), 1e-300))}
        if not args.no_cpu and t_all < 20.0:
            t0 = time.perf_counter()
            r = O.ipm(O.Operator.from_dense(p.A), p.b, p.tau, O.OracleParams(tol=params.tol))
            dt = time.perf_counter() - t0
            t_all += dt
            done += 1
            # Newton directions taken (the oracle counts its gap checks, one more)
            row.update({"direct_ipm_iters": r.iters - 1, "direct_host_ms": 1e3 * dt})
        rows.append(row)
    if done:
        cpu = {"value": done / t_all, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{done} of the {len(probs)} sizes (smallest first) in {t_all:.1f} s: float64 IPM "
                         f"with direct Newton solves, tol {params.tol:g}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sizes": [p.n for p in probs], "m": "n/4", "k": "ceil(m/20)",
                   "tau": probs[0].tau, "tol": params.tol, "l2": "flushed (512 MiB write) before each step",
                   "solved_at_kkt_1e-6": ok},
        "roofline": {"bound": "hbm", "achieved": abytes / (kern_last[big] / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": abytes / (kern_last[big] / 1e3) / 1e9 / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": f"ipm_kernel (dense float64), n = {probs[big].n}",
                     "kernel_ms": kern_last[big], "algorithmic_bytes": abytes},
        "pcg_vs_direct": rows,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": sum((p.A.size + p.m) * 8 for p in probs),
                "d2h_bytes_per_step": sum(p.n * 8 for p in probs)},
        "cpu_baseline": cpu, "gpu_launches": len(probs) * args.steps,  # one persistent launch per solve
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_dense(args, rank, world, local_rank, probs):
    """Plain float64 mfIPM on one dense Gaussian problem (256 x 1024): one step = one mfipm_solve
    (the persistent kernel on one cluster; float64 PCG).  A (2 MiB) stays in L2, so the
    roofline's algorithmic bytes (A read once per product with A or A^T) are an L2-resident
    stream reported against HBM for comparability."""
    import torch
    import paper_1208_5435_gb300 as M

    dev = torch.device("cuda", local_rank)
    L = M.lib()
    p0 = probs[0]
    op = M.Dense(torch.from_numpy(p0.A).to(dev))
    b = torch.from_numpy(p0.b).to(dev)
    params = M.SolverParams()
    ws = torch.empty(M.workspace_bytes([op], params), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        M.solve(op, b, p0.tau, params, ws=ws)
    torch.cuda.synchronize()
    L.mfipm_set_timing(1)
    step_ms, kern_ms = [], []
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with RooflineRange(s_ == args.steps - 1):
                e0.record(stream)
                x, info = M.solve(op, b, p0.tau, params, ws=ws)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(L.mfipm_last_kernel_ms())
    L.mfipm_set_timing(0)
    ok = 1 if info["status"] == 0 and info["kkt_rel"] <= KKT_GATE else 0
    value, total_ms = job_throughput(ok, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    kms = statistics.mean(kern_ms)
    abytes = info["n_mat"] * p0.m * p0.n * 8
    peak, peak_kind = measured_peaks()
    tj = load_traffic(args.workload)
    traffic = tj["bytes_per_launch"] if tj else None
    # e2e: A and b from pinned host memory, x read back
    hA = torch.from_numpy(p0.A).pin_memory()
    hb = torch.from_numpy(p0.b).pin_memory()
    hx = torch.empty(p0.n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(1 + args.steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eop = M.Dense(hA.to(dev, non_blocking=True))
        xe, ie = M.solve(eop, hb.to(dev, non_blocking=True), p0.tau, params, ws=ws)
        hx.copy_(xe, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_ok = 1 if ie["status"] == 0 and ie["kkt_rel"] <= KKT_GATE else 0
    e2e_value = sum_over_ranks(e2e_ok, world, dev) / (max_over_ranks(sum(e2e_ms), world, dev) / args.steps / 1e3)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        from oracle import mfipm_oracle as O
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < 10.0:
            O.ipm(O.Operator.from_dense(p0.A), p0.b, p0.tau, O.OracleParams(tol=1e-10))
            done += 1
        secs = time.perf_counter() - t0
        cpu = {"value": done / secs, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{done} solve(s) of the same problem in {secs:.1f} s: direct-solve float64 IPM"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "m": p0.m, "n": p0.n, "tol": params.tol,
                   "l2": "flushed (512 MiB write) before each step", "solved_at_kkt_1e-6": ok},
        "roofline": {"bound": "hbm", "achieved": abytes / (kms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": abytes / (kms / 1e3) / 1e9 / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "ipm_kernel (dense float64, one cluster)", "kernel_ms": kms,
                     "algorithmic_bytes": abytes},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (p0.A.size + p0.m) * 8,
                "d2h_bytes_per_step": p0.n * 8},
        "cpu_baseline": cpu, "gpu_launches": args.steps,  # one persistent launch per solve
        "clocks": clk.summary(),
        "iterations": {"ipm": info["ipm_iters"], "pcg": info["pcg_iters"], "kkt": info["kkt_rel"]},
    }
    print(json.dumps(line), flush=True)


def run_bf16(args, rank, world, local_rank, probs):
    """Shared-A bf16 workload: one step = one mfipm_solve_batched over all right-hand sides."""
    import ctypes
    import torch
    import paper_1208_5435_gb300 as M

    dev = torch.device("cuda", local_rank)
    L = M.lib()
    bits = torch.from_numpy(probs[0].a_bf16.view(np.int16)).view(torch.bfloat16).to(dev)
    op = M.DenseBF16(bits, probs[0].a_scale)
    ops = [op] * len(probs)
    bs = [torch.from_numpy(p.b).to(dev) for p in probs]
    taus = [p.tau for p in probs]
    params = M.SolverParams()
    ws = torch.empty(M.workspace_bytes(ops, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    tuning = M.autotune(ops, bs, taus, params, ws=ws)[2]  # split-K of the two GEMMs (untimed)
    for _ in range(args.warmup):
        M.solve_batched(ops, bs, taus, params, ws=ws)
    torch.cuda.synchronize()
    step_ms = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xs, infos = M.solve_batched(ops, bs, taus, params, ws=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    ok = sum(1 for i in infos if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    value, total_ms = job_throughput(ok, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    ms_, by_, pr_, la_ = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    assert L.mfipm_last_operator_stats(ctypes.byref(ms_), ctypes.byref(by_), ctypes.byref(pr_), ctypes.byref(la_)) == 0
    launches = int(la_.value)  # the kernels of the last solve call (lockstep solve and the norm of A)

    # e2e: A and the right-hand sides from pinned host memory, x read back, every step
    hA = torch.from_numpy(probs[0].a_bf16.view(np.int16)).pin_memory()
    hb = [torch.from_numpy(p.b).pin_memory() for p in probs]
    hx = [torch.empty(p.n, dtype=torch.float64).pin_memory() for p in probs]
    dA = torch.empty(hA.shape, dtype=torch.int16, device=dev)
    h2d = hA.numel() * 2 + sum(t.numel() * 8 for t in hb)
    d2h = sum(t.numel() * 8 for t in hx)
    e2e_ms = []
    for it in range(1 + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dA.copy_(hA, non_blocking=True)
        eop = M.DenseBF16(dA.view(torch.bfloat16), probs[0].a_scale)
        xs_, inf_ = M.solve_batched([eop] * len(probs), [b_.to(dev, non_blocking=True) for b_ in hb], taus, params,
                                    ws=ws)
        for h, d_ in zip(hx, xs_):
            h.copy_(d_, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_ok = sum(1 for i in inf_ if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE)
    e2e_value, _ = job_throughput(e2e_ok, sum(e2e_ms), args.steps, world, dev)
    # the tensor-core GEMMs of one PCG operator product, timed alone on their real shapes
    m, n, R = probs[0].m, probs[0].n, len(probs)
    W_ = torch.randn(2 * R, n, device=dev).to(torch.bfloat16)
    T_ = torch.randn(2 * R, m, device=dev).to(torch.bfloat16)
    At = bits.T.contiguous()
    s1, s2 = max(1, tuning["splits1"]), max(1, tuning["splits2"])  # the split-K the solve uses
    g1, g2 = tuning["stages1"] or 4, tuning["stages2"] or 4         # and its ring stages
    C1 = torch.empty(s1, 2 * R, m, device=dev)
    C2 = torch.empty(s2, 2 * R, n, device=dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    def gemm_pair():
        assert L.mfipm_gemm_bf16(bits.data_ptr(), W_.data_ptr(), C1.data_ptr(), m, 2 * R, n, s1, g1, sh) == 0
        assert L.mfipm_gemm_bf16(At.data_ptr(), T_.data_ptr(), C2.data_ptr(), n, 2 * R, m, s2, g2, sh) == 0
    for _ in range(3):
        gemm_pair()
    reps = 20
    g_ms = []
    for r_ in range(reps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with RooflineRange(r_ == reps - 1):
            e0.record(stream)
            gemm_pair()
            e1.record(stream)
        torch.cuda.synchronize()
        g_ms.append(e0.elapsed_time(e1))
    gms = statistics.median(g_ms)
    # algorithmic: A read by both GEMMs, W and T in, one float32 product out each (split-K
    # partial slices are the implementation's extra traffic, not counted)
    gbytes = 2 * (m * n * 2) + 2 * R * (n + m) * 2 + (2 * R * m + 2 * R * n) * 4
    gflop = 2 * 2 * m * n * 2 * R
    peak, peak_kind = measured_peaks()
    tj = load_traffic(args.workload)
    traffic = tj["bytes_per_launch"] if tj else None
    traffic_cfg = {"splits": tj["splits"], "stages": tj["stages"]} if tj else None
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        from oracle import mfipm_oracle as O
        A = probs[0].A
        t0 = time.perf_counter()
        O.ipm(O.Operator.from_dense(A), probs[0].b, probs[0].tau, O.OracleParams(tol=1e-10, solver="woodbury"))
        secs = time.perf_counter() - t0
        cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"1 of {len(probs)} right-hand sides, {secs:.1f} s: direct-solve float64 IPM (Woodbury m x m)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 A / f32 PCG / double-float outer (~48-bit)", "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "rhs": R, "l2": "flushed (512 MiB write) before each step",
                   "solved_at_kkt_1e-6": ok,
                   "tuned": {"splits1": tuning["splits1"], "splits2": tuning["splits2"],
                             "stages1": tuning["stages1"], "stages2": tuning["stages2"],
                             "best_ms": tuning["best_ms"], "default_ms": tuning["default_ms"]}},
        "roofline": {"bound": "hbm", "achieved": gbytes / (gms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": gbytes / (gms / 1e3) / 1e9 / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_config": traffic_cfg,
                     "kernel": "tc_gemm_kernel pair (T = A W, Y = A^T T), timed alone", "kernel_ms": gms,
                     "algorithmic_bytes": gbytes, "tensor_tflops": gflop / (gms / 1e3) / 1e12},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "cpu_baseline": cpu, "clocks": clk.summary(),
        "iterations": {"ipm_mean": statistics.mean(i["ipm_iters"] for i in infos),
                       "pcg_mean": statistics.mean(i["pcg_iters"] for i in infos),
                       "kkt_max": max(i["kkt_rel"] for i in infos)},
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args, rank, world, local_rank, probs):
    """Differentiation at scale: one step = mfipm_solve_batched over the 32 partial-DCT problems
    (n = 2^20, the lockstep multi-pass solver) followed by mfipm_backward of
    L = 1/2||x* - x_hat||^2 for all of them.  A problem counts once both its forward solve
    (kkt_rel <= 1e-6) and its adjoint solve succeed."""
    import ctypes
    import torch
    import paper_1208_5435_gb300 as M

    dev = torch.device("cuda", local_rank)
    L = M.lib()
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows).to(dev)) for p in probs]
    bs = [torch.from_numpy(p.b).to(dev) for p in probs]
    xh = [torch.from_numpy(p.x_hat).to(dev) for p in probs]
    taus = [p.tau for p in probs]
    params = M.SolverParams()
    ws = torch.empty(M.workspace_bytes(ops, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ms_, by_, pr_, la_ = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()

    def op_stats():
        assert L.mfipm_last_operator_stats(ctypes.byref(ms_), ctypes.byref(by_), ctypes.byref(pr_),
                                           ctypes.byref(la_)) == 0
        return ms_.value, by_.value, pr_.value, la_.value

    def step(b_list, stats=None):
        xs, infos, zss = M.solve_batched(ops, b_list, taus, params, return_zs=True, ws=ws)
        if stats is not None:
            stats.append(op_stats())
        gxs = [x - h for x, h in zip(xs, xh)]
        gbs, gts, _, binfos = M.backward(ops, b_list, taus, xs, zss, gxs, params, ws=ws)
        if stats is not None:
            stats.append(op_stats())
        return xs, infos, gbs, gts, binfos

    for _ in range(args.warmup):
        step(bs)
    torch.cuda.synchronize()
    L.mfipm_set_timing(1)
    step_ms, stats = [], []
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with RooflineRange(s_ == args.steps - 1):
                e0.record(stream)
                xs, infos, gbs, gts, binfos = step(bs, stats)
                e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    L.mfipm_set_timing(0)
    ok = sum(1 for i, bi in zip(infos, binfos) if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE and bi["status"] == 0)
    value, total_ms = job_throughput(ok, sum(step_ms), args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    op_ms = sum(s[0] for s in stats)
    op_bytes = sum(s[1] for s in stats)
    op_products = sum(s[2] for s in stats)
    launches = sum(s[3] for s in stats)
    peak, peak_kind = measured_peaks()
    achieved = op_bytes / (op_ms / 1e3) / 1e9
    # the capture holds the first product of the step (every problem live); per product on
    # average, its per-problem traffic times the problems a product served on average
    tj = load_traffic(args.workload)
    traffic = (tj["bytes_per_launch"] / tj["problems"] * (op_bytes / max(op_products, 1)) / (8.0 * probs[0].n)
               if tj and tj.get("n") == probs[0].n else None)

    # e2e: host b, rows and x_hat in pinned memory; x and grad_b read back every step
    hb = [torch.from_numpy(p.b).pin_memory() for p in probs]
    hr = [torch.from_numpy(p.rows).pin_memory() for p in probs]
    hh = [torch.from_numpy(p.x_hat).pin_memory() for p in probs]
    hx = [torch.empty(p.n, dtype=torch.float64).pin_memory() for p in probs]
    hg = [torch.empty(p.m, dtype=torch.float64).pin_memory() for p in probs]
    h2d = sum(t.numel() * 8 for t in hb + hr + hh)
    d2h = sum(t.numel() * 8 for t in hx + hg) + 8 * len(probs)
    e2e_ms = []
    for it in range(1 + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dops = [M.PartialDCT(p.n, r.to(dev, non_blocking=True)) for p, r in zip(probs, hr)]
        dbs = [b_.to(dev, non_blocking=True) for b_ in hb]
        dxh = [h.to(dev, non_blocking=True) for h in hh]
        xs_, inf_, zss_ = M.solve_batched(dops, dbs, taus, params, return_zs=True, ws=ws)
        gb_, gt_, _, bi_ = M.backward(dops, dbs, taus, xs_, zss_, [x - h for x, h in zip(xs_, dxh)], params, ws=ws)
        for h, d in zip(hx, xs_):
            h.copy_(d, non_blocking=True)
        for h, d in zip(hg, gb_):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_ok = sum(1 for i, bi in zip(inf_, bi_) if i["status"] == 0 and i["kkt_rel"] <= KKT_GATE and bi["status"] == 0)
    e2e_value, _ = job_throughput(e2e_ok, sum(e2e_ms), args.steps, world, dev)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        from oracle import mfipm_oracle as O
        small = W.make_workload(args.workload, count=4, scale_n=4096)
        t0 = time.perf_counter()
        done = 0
        for p in small:
            op = O.Operator.from_dct_rows(p.n, p.rows)
            res = O.ipm(op, p.b, p.tau, O.OracleParams(tol=1e-10))
            O.adjoint_kkt(op, p.b, p.tau, res.z, res.s, res.x - p.x_hat)
            done += 1
            if time.perf_counter() - t0 > 15.0:
                break
        secs = time.perf_counter() - t0
        cpu = {"value": done / secs, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{done} problem(s) in {secs:.1f} s of the same workload scaled to n = 4096 "
                         f"(m = 1024, k = 40; the direct solve cannot reach n = 2^20): float64 IPM + KKT adjoint"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 PCG / double-float outer (~48-bit)", "data": "synthetic",
        "config": {"workload": args.workload, "problems": len(probs), "n": probs[0].n, "m": probs[0].m,
                   "solve": "forward solve + adjoint (mfipm_backward) per problem",
                   "tol": params.tol, "tol_pcg": params.tol_pcg,
                   "l2": "inputs larger than L2 (about 4 GB of solver state) and a 512 MiB flush per step",
                   "solved_at_kkt_1e-6": ok},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "operator product y = A^T A w (pass_a + pass_b + pass_c, float32), "
                               "CUDA events inside the timed solves",
                     "kernel_ms": op_ms / max(op_products, 1), "products": op_products,
                     "algorithmic_bytes": op_bytes / max(op_products, 1)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "iterations": {"ipm_mean": statistics.mean(i["ipm_iters"] for i in infos),
                       "pcg_mean": statistics.mean(i["pcg_iters"] for i in infos),
                       "bwd_pcg_mean": statistics.mean(i["pcg_iters"] for i in binfos),
                       "kkt_max": max(i["kkt_rel"] for i in infos),
                       "operator_ms_share": op_ms / total_ms},
    }
    print(json.dumps(line), flush=True)


def kernel_hash(files=None):
    """Hash of the CUDA sources (all of them, or the listed files that define one kernel)."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1208_5435_gb300", "csrc")
    for f in sorted(files or os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


def last_call_launches(L):
    """Kernels of ours the last solve, batched solve or backward call launched (library count)."""
    ms_, by_, pr_, la_ = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    assert L.mfipm_last_operator_stats(ctypes.byref(ms_), ctypes.byref(by_), ctypes.byref(pr_), ctypes.byref(la_)) == 0
    return int(la_.value)


def load_traffic(workload):
    """DRAM bytes (read + write) that one ncu capture measured for this workload's roofline
    kernel, kept only while the CUDA sources are the ones that were captured (all of them, or
    the entry's `sources`: the files that define the captured kernel)."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None
    tj = json.load(open(tpath)).get(workload)
    if tj and tj.get("kernel_hash") == kernel_hash(tj.get("sources")):
        return tj
    return None


class RooflineRange:
    """NVTX range "roofline" around the launches whose DRAM traffic the roofline reports
    (ncu --nvtx --nvtx-include roofline/ captures exactly those)."""

    def __init__(self, on):
        self.on = on

    def __enter__(self):
        if self.on:
            import torch
            torch.cuda.nvtx.range_push("roofline")
        return self

    def __exit__(self, *a):
        if self.on:
            import torch
            torch.cuda.nvtx.range_pop()


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
