"""Benchmark of the P-GVIMP hot path on B300: plans/s for a batch of
dense-horizon planning problems (2-D point robot, double integrator, N=750,
500x500 SDF at 0.05 m from 25 disks and boxes, Gauss-Hermite 5 points per
dimension, 30 proximal iterations, step 0.5), served mixed precision
(FP32 quadrature / FP64 recursions) next to the plain all-FP64 path.

One JSON line on rank 0.  A step plans the whole batch: prior build,
initial iterate and marginals, 30 iterations of quadrature + gradients +
KL-bounded step search + update, on device-resident inputs (`value`); `e2e`
adds the host-to-device copy of every plan's inputs and the device-to-host
copy of the results each step.  `--impl reference` times the FP64 CPU oracle
(the reference arm of this build) on the host cores.

Multi-GPU: plans are independent, so ranks run replicas on disjoint batches
(weak scaling); the only collectives are the barrier and the max over ranks
of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The server overlaps batches on up to 32 streams; with CUDA's default of 8
# hardware work queues, streams share queues and their kernels serialise.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "plans/sec and p50/p99 plan latency, served FP32/FP64 vs plain FP64, 1 B300"
ITERS, N_STEPS, GH_P = 30, 750, 5
MAP_POOL = 32   # distinct seeded maps; every plan also has its own seeded goal offset


# --------------------------------------------------------------------- inputs

def plan_problem(i: int, base=None):
    """Plan i of the batch workload: map i % MAP_POOL and a goal offset
    U(-0.5, 0.5)^2 m drawn from the plan's own seed."""
    from dataclasses import replace

    import numpy as np

    import workloads as W
    pb, op = base[i % MAP_POOL] if base else W.c2_point2d_dense(request=i % MAP_POOL, N=N_STEPS, iters=ITERS)
    rng = np.random.Generator(np.random.PCG64(3_000_000 + i))
    muN = pb.muN.copy()
    muN[:2] += rng.uniform(-0.5, 0.5, size=2)
    return replace(pb, muN=muN), op


def make_batch_problems(count: int, rank: int = 0):
    """Rank r plans indices r*count .. r*count + count - 1 (disjoint across
    replicas); each map is built once."""
    import workloads as W
    idx = [rank * count + i for i in range(count)]
    base = {k: W.c2_point2d_dense(request=k, N=N_STEPS, iters=ITERS) for k in sorted({j % MAP_POOL for j in idx})}
    pairs = [plan_problem(j, base) for j in idx]
    return [p for p, _ in pairs], [o for _, o in pairs]


# ------------------------------------------------------------------ work count

def fp64_flops_per_trial_state(n: int) -> int:
    """FP64 flops (FMA = 2) of one Thm 1 trial per state, counted from the
    trial sweep: forward (two eliminations sharing the off-diagonal blocks,
    right-hand side, carries) 8n^3 + 25n^2 + 5n; backward (selected inverse,
    back substitution, KL and prior-cost terms) 3n^3 + 33n^2 + 2n."""
    return 11 * n ** 3 + 58 * n ** 2 + 7 * n


def fp64_flops_per_iter_state(n: int, dc: int) -> int:
    """FP64 flops per state per iteration outside the trials: the update of
    Lambda (5 n^2) and the gradient assembly from the FP32 moments
    (Cholesky / inverse of the dc x dc marginal block, g and G)."""
    return 5 * n * n + dc ** 3 + 2 * dc * dc * dc + 2 * dc * dc + 4 * dc


def algorithmic_fp64_flops(problems, trials_per_plan, iters=ITERS):
    tot = 0
    for pb, trials in zip(problems, trials_per_plan):
        S = pb.N + 1
        tot += S * (trials * fp64_flops_per_trial_state(pb.n) + iters * fp64_flops_per_iter_state(pb.n, 2))
    return tot


def fp64_peak_tflops():
    """FP64 peak derived from unit counts and clock: 148 SMs x 2 DFMA lanes per
    SM per clock x 2 flops x 2032 MHz = 1.203 TFLOP/s (B300 data sheet 1.25).
    Measured with a DFMA-throughput loop on this machine: 0.935 TFLOP/s."""
    return 148 * 2 * 2 * 2.032e9 / 1e12


def fp32_peak_tflops():
    """FP32 peak derived from unit counts and clock: 148 SMs x 128 FFMA lanes per
    SM per clock x 2 flops x 2032 MHz = 76.99 TFLOP/s.  Measured with an
    FFMA-throughput loop on this machine: 68.2 TFLOP/s."""
    return 148 * 128 * 2 * 2.032e9 / 1e12


# FP32 flops per emulated FP64 flop in the double-float recursions, counted
# from the double-float primitives: an FMA is 4 FFMA/FMUL + 11 FADD/FSUB (18
# flops for 2 FP64 flops), a multiply 10 flops, an add 11 flops; with the
# trial's FP64 op mix (600 FMA : 129 add : 168 mul per state) that is
# (600*18 + 129*11 + 168*10) / (600*2 + 129 + 168) = 9.29.  This is the
# algorithmic FP32 work per FP64 flop, what `achieved` counts.
DF_EXPANSION = 9.29

# What the lane-form kernel (k_iterate_lane, sixteen lanes per plan) executes,
# from ncu counters of 2,368 dense-horizon plans x 30 iterations (N = 750):
# with double-float recursions 5.244e12 FP32 flops (2 FFMA + FADD + FMUL) over
# 336,790 trials x 751 states = 20,720 per state-trial; with FP64 recursions
# 196 FP32 flops per state-trial (the quadrature) and 3,424 FP64 flops per
# state-trial against the 1,685 counted (its per-lane pivot reciprocals are
# IEEE divisions and its row sums are replicated over the row's four lanes).
# The double-float recursions thus execute 20,524 FP32 flops per state-trial,
# a measured expansion of 12.2 FP32 flops per counted FP64 flop.
LANE_DF_EXECUTED_FP32_PER_STATE_TRIAL = 5.244e12 / (336790 * 751)
LANE_DF_MEASURED_EXPANSION = 12.2

# DRAM bytes (read + write) per state per trial of the thread-form kernel with
# FP64 recursions (k_iterate<4, float, double>), from an ncu capture of 2,368
# dense-horizon plans x 30 iterations: 399.9 GB read + 164.3 GB written over
# 335,500 trials x 751 states = 2,239 B, the algorithmic touch of one state
# (about 2.5 KB).  The same capture counts 1,417 executed FP64 flops per
# state-trial (2 DFMA + DADD + DMUL) against the 1,685 counted.
THREAD_F64_DRAM_BYTES_PER_STATE_TRIAL = (399.921e9 + 164.257e9) / (335500 * 751)

# DRAM bytes (read + write) per state per trial of the lane-form double-float
# kernel, from the same capture: 416.2 GB read + 178.6 GB written over 336,790
# trials x 751 states = 2,352 B.  The algorithmic touch of one state-trial (both
# sweeps read the five blocks, the scratch is written and read back, the
# outputs written) is about 2.5 KB, so the kernel makes no wasted re-reads.  A
# full launch's traffic is this times its state-trials (traffic grows in
# proportion to the state-trials: the per-plan working set, ~1 MB, exceeds
# what L2 holds for a resident wave of plans).
LANE_DF_DRAM_BYTES_PER_STATE_TRIAL = (416.199e9 + 178.616e9) / (336790 * 751)


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to PGVIMP_CLOCKS_DIR (default: the system temp directory)
        import tempfile
        out_dir = os.environ.get("PGVIMP_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"pgvimp_clocks_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU baseline

# Iterations of the element-wise sample check.  The dense-horizon plans are
# ill-conditioned: the oracle against itself, with the goal moved by a relative
# 1e-12, differs in the marginal covariances by up to 4.2e-5 after one
# iteration and 7.2e-3 after two (16 sampled plans), so only the first
# iteration is compared element-wise; the whole plan is checked through
# invariants that hold at any size.
SAMPLE_ITERS = 1


def _oracle_one(args):
    idx, = args
    sys.path.insert(0, ROOT)
    import oracle
    pb, op = plan_problem(idx)
    t = time.perf_counter()
    oracle.plan(pb, op)
    return time.perf_counter() - t


def _oracle_sample(args):
    """The first SAMPLE_ITERS iterations of plan `idx` (for the sample check),
    and how far they move when the goal moves by a relative 1e-12."""
    idx, = args
    sys.path.insert(0, ROOT)
    from dataclasses import replace

    import numpy as np

    import oracle
    pb, op = plan_problem(idx)
    op1 = replace(op, iters=SAMPLE_ITERS)
    s = oracle.plan(pb, op1)
    resp = []
    for rel in (1e-12, 2.0 ** -24):   # the problem's own response to a tiny and to an FP32-sized change of the goal
        t = oracle.plan(replace(pb, muN=pb.muN * (1 + rel)), op1)
        resp.append((float(np.linalg.norm(s.mu - t.mu) / np.linalg.norm(s.mu)),
                     float(np.max(np.linalg.norm(s.Sd - t.Sd, axis=(1, 2)) / np.linalg.norm(s.Sd, axis=(1, 2))))))
    return idx, s.mu, s.Sd, [l["beta"] for l in s.logs], resp


def cpu_baseline(workers: int | None = None, plans_per_worker: int = 1, samples: bool = False):
    """The FP64 oracle on the host cores, one plan per process (spawned), on
    a bounded sample of the workload: `workers` full plans.  With `samples`,
    afterwards and untimed, the first iterations of the same plans for the
    sample check."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    workers = workers or max(1, min(os.cpu_count() or 1, 16))
    ctx = mp.get_context("spawn")
    n_plans = workers * plans_per_worker
    with ctx.Pool(workers) as pool:
        t0 = time.perf_counter()
        times = pool.map(_oracle_one, [(i,) for i in range(n_plans)])
        wall = time.perf_counter() - t0
        outs = pool.map(_oracle_sample, [(i,) for i in range(n_plans)]) if samples else None
    res = {"value": n_plans / wall, "unit": "plans/s", "cores": workers, "kind": "oracle",
           "sample": f"{n_plans} full plans of the batch workload (one per spawned process), "
                     f"median {statistics.median(times):.1f} s per plan single-threaded",
           "wall_s": wall}
    return res, outs


def sample_check(samples, precision):
    """The sampled plans of the batch (the oracle's CPU-baseline plans),
    SAMPLE_ITERS iterations on the GPU in the batch's precision and form,
    against the oracle element by element: relative 2-norm of mu over the
    trajectory, largest relative Frobenius error of a Sigma_ii block, and the
    step sizes."""
    from dataclasses import replace

    import numpy as np
    import torch

    from paper_2411_03416_b300 import _lib as L
    idx = [i for i, *_ in samples]
    pairs = [plan_problem(i) for i in idx]
    probs = [p for p, _ in pairs]
    opts = [replace(o, iters=SAMPLE_ITERS) for _, o in pairs]
    st = torch.cuda.Stream()
    b = L.Batch(probs, opts, precision)
    b.upload(st.cuda_stream)
    b.reset(st.cuda_stream)
    b.run(0, st.cuda_stream)
    b.download_results(st.cuda_stream)
    torch.cuda.synchronize()
    tol_mu, tol_sigma = (1e-9, 1e-9) if precision == 0 else (1e-4, 1e-3)
    # the conditioning bound: the oracle's own response to a relative change of the goal at the precision's
    # rounding level (1e-12 for FP64; 2^-24, the FP32 unit roundoff, for the FP32 quadrature of the mixed forms)
    level = 0 if precision == 0 else 1
    emu, esig, same_beta, ok = 0.0, 0.0, 0, True
    resp_max = [[0.0, 0.0], [0.0, 0.0]]
    for k, (_, mu, Sd, betas, resp) in enumerate(samples):
        r = b.result(k, full=False)
        e1 = float(np.linalg.norm(r.mu - mu) / np.linalg.norm(mu))
        e2 = float(np.max(np.linalg.norm(r.Sd - Sd, axis=(1, 2)) / np.linalg.norm(Sd, axis=(1, 2))))
        smu, ssig = resp[level]
        ok = ok and e1 <= max(tol_mu, 10 * smu) and e2 <= max(tol_sigma, 10 * ssig)
        emu, esig = max(emu, e1), max(esig, e2)
        for j in range(2):
            resp_max[j] = [max(resp_max[j][0], resp[j][0]), max(resp_max[j][1], resp[j][1])]
        same_beta += int([l["beta"] for l in r.logs] == betas)
    b.close()
    return {"plans": len(samples), "iterations": SAMPLE_ITERS, "max_rel_mu": emu, "max_rel_sigma": esig,
            "same_step_sizes": same_beta, "tol_mu": tol_mu, "tol_sigma": tol_sigma,
            "oracle_response_to_goal_change": {"rel_1e-12": {"mu": resp_max[0][0], "sigma": resp_max[0][1]},
                                               "rel_2^-24": {"mu": resp_max[1][0], "sigma": resp_max[1][1]}},
            "criterion": "per plan: error <= max(tolerance, 10 x the oracle's response at the precision's rounding "
                         "level)", "pass": ok}


# ------------------------------------------------------------------------ main

def dist_init():
    """Replicas: one process per GPU (NCCL), or gloo ranks on a host without
    a GPU (the multi-rank host logic is tested that way)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)   # each rank's collectives on its own GPU
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = max(1, min(os.cpu_count() or 1, 16))
    for _ in range(args.warmup):
        cpu_baseline(cores)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(cores)[0])
    v = statistics.median(x["value"] for x in vals)
    ms = 1000.0 * statistics.median(x["wall_s"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "plans/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.batch, ws),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "plans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(batch, ws):
    return {"workload": f"dense-horizon 2-D point robot plans, batch of {batch} per GPU",
            "N": N_STEPS, "state_dim": 4, "quadrature": f"Gauss-Hermite {GH_P} points per dim (25 distinct after "
            "the exact reduction)", "iterations": ITERS, "sdf": "500x500 FP32 at 0.05 m, 25 disks/boxes",
            "batch_per_gpu": batch, "global_batch": batch * ws, "maps": f"{MAP_POOL} seeded maps, per-plan goal offset",
            "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{ws}"}


# ------------------------------------------------------------------- serving

SERVE_BUDGET = 80 << 30   # HBM admission budget of the serving mix


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v, dtype=float), q)) if len(v) else None


def run_served(mix, precision, plan_threads, max_inflight=32, max_batch=16, window_ms=2.0, submitters=4):
    """Replays the mix's arrival times against a server (continuous batching)
    and returns plans/s (count / time from the first arrival to the last
    result on the host) and p50/p99 latency (arrival to result on the host)."""
    import threading

    import paper_2411_03416_b300 as pg
    srv = pg.Server(SERVE_BUDGET, precision=precision, plan_threads=plan_threads, max_inflight=max_inflight,
                    max_batch=max_batch, batch_window_ms=window_ms)
    seen = set()
    for rq in mix:                          # load every kernel the mix uses before timing
        key = (rq.problem.n, rq.problem.dyn_kind)
        if key not in seen:
            seen.add(key)
            srv.poll(srv.submit(rq.problem, rq.options))
    ready = [srv.prepare(rq.problem, rq.options) for rq in mix]
    ids = [None] * len(mix)
    lags = []
    t0 = time.perf_counter()
    s0 = srv.stats()["now_ms"]

    def submitter(first):
        for k in range(first, len(mix), submitters):
            d = t0 + mix[k].arrival_s - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids[k] = srv.submit(ready[k])
            lags.append(time.perf_counter() - t0 - mix[k].arrival_s)

    ths = [threading.Thread(target=submitter, args=(j,)) for j in range(submitters)]
    for th in ths:
        th.start()
    lat, done, sizes = [], [], []
    for k, rq in enumerate(mix):
        while ids[k] is None:
            time.sleep(1e-4)
        _, _, info = srv.poll(ids[k], timeout_ms=-1)
        lat.append(info["done_ms"] - (s0 + 1000.0 * rq.arrival_s))
        done.append(info["done_ms"] - s0)
        sizes.append(info["batch_size"])
    for th in ths:
        th.join()
    st = srv.stats()
    srv.close()
    span_s = max(done) / 1000.0
    return {"plans_per_s": len(mix) / span_s, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
            "makespan_s": span_s, "requests": len(mix), "batches": st["batches"] - len(seen),
            "mean_batch": sum(sizes) / len(sizes), "submit_lag_ms_max": 1000.0 * max(lags),
            "host_launch_ms": st["host_launch_ms"], "host_collect_ms": st["host_collect_ms"],
            "graph_launches": st["graph_launches"], "graph_instantiations": st["graph_instantiations"],
            "precision": precision, "plan_threads": plan_threads, "max_inflight": max_inflight,
            "max_batch": max_batch, "batch_window_ms": window_ms}


def run_plain(mix):
    """Plain per-request FP64: one plan at a time through the single-plan calls
    (pgvimp_create / plan / get / destroy) on one stream, no batching, in
    arrival order; latency from arrival to the result on the host.  Each
    request keeps its options' execution form."""
    import paper_2411_03416_b300 as pg
    from paper_2411_03416_b300 import _lib as L
    seen = set()
    for rq in mix:
        key = (rq.problem.n, rq.problem.dyn_kind)
        if key not in seen:
            seen.add(key)
            c = pg.Context(rq.problem, rq.options, L.PREC_PLAIN_FP64)
            c.plan()
            c.get()
            c.close()
    lat = []
    t0 = time.perf_counter()
    for rq in mix:
        d = t0 + rq.arrival_s - time.perf_counter()
        if d > 0:
            time.sleep(d)
        c = pg.Context(rq.problem, rq.options, L.PREC_PLAIN_FP64)
        c.plan()
        c.get()
        c.close()
        lat.append(1000.0 * (time.perf_counter() - t0 - rq.arrival_s))
    span_s = time.perf_counter() - t0
    return {"plans_per_s": len(mix) / span_s, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
            "makespan_s": span_s, "requests": len(mix), "precision": 0}


def serving(args):
    from dataclasses import replace

    import workloads as W
    from paper_2411_03416_b300 import autotune
    mix = W.c5_mix(args.serve_count)
    # block size per (n, dynamics, horizon bucket), tuned on one request of each bucket
    tuner = autotune.Tuner()
    reps = {}
    for rq in mix:
        reps.setdefault(autotune.bucket(rq.problem), (rq.problem, rq.options))
    t = time.perf_counter()
    tuner.tune(reps.values(), precision=1, repeats=1, copies=148)   # one plan per SM: a loaded GPU
    tune_s = time.perf_counter() - t
    mix = [replace(rq, options=tuner.apply(rq.problem, rq.options)) for rq in mix]
    out = {"workload": f"serving mix: {args.serve_count} requests, Poisson arrivals at 2000/s; 50% 2-D point robot "
                       "N~U{50..1000}, 30% planar quadrotor SLR N~U{100..500}, 20% 7-DOF arm N~U{100..300}; "
                       "own seeded map per request; 80 GB admission budget",
           "latency": "arrival to result on the host (server clock)"}
    # served FP32/FP64: FP32 quadrature, FP64 recursions, block form, continuous batching
    out["autotune"] = {"seconds": tune_s, "table": {f"n{k[0]}/dyn{k[1]}/log2N{k[2]}": v for k, v in tuner.table.items()}}
    # untimed: the first server flights of a process pay about 2 s of one-time host cost on the scheduler thread
    # (a first replay of the mix measured 77 plans/s with 2.2 s of launch time, the same form replayed next 112)
    out["warmup_replay"] = {k: v for k, v in run_served(mix[:128], 1, -1).items()
                            if k in ("plans_per_s", "host_launch_ms", "requests")}
    out["served_fp32_fp64"] = run_served(mix, 1, -1)
    out["served_fp32_double_float"] = run_served(mix, 2, -1)
    out["served_plain_fp64"] = run_served(mix, 0, -1)
    sample = mix[:args.plain_count]
    out["plain_sample"] = f"first {len(sample)} requests of the mix (arrival times kept)"
    out["plain_fp64_per_request"] = run_plain(sample)
    out["served_fp32_fp64_on_sample"] = run_served(sample, 1, -1)
    return out


# ---------------------------------------------------- the other configurations

def other_configs(args):
    """Batch throughput of the other workloads in their throughput form, the
    single-plan latency of every workload in the block (latency) form, and the
    roofline fraction of each batch's fused kernel.  One timed run each, after
    one untimed run; CUDA events on the launching stream."""
    from dataclasses import replace

    import torch

    import workloads as W
    from paper_2411_03416_b300 import _lib as L
    st = torch.cuda.Stream()
    sh = st.cuda_stream

    def timed(probs, opts, prec):
        b = L.Batch(probs, opts, prec)
        b.upload(sh)
        for k in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b.reset(sh)
            e0.record(st)
            b.run(0, sh)
            e1.record(st)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        b.download_results(sh)
        torch.cuda.synchronize()
        trials = [sum(l["trials"] for l in b.result(i, full=False).logs) for i in range(len(probs))]
        b.close()
        return ms, trials

    cfgs = {
        "C1 point robot, N=50, GH 3, 20 iterations": (lambda r: W.c1_point2d(request=r), 75776, 4, 2),
        "C3 7-DOF arm, N=200, degree-3 rule, 25 iterations": (lambda r: W.c3_arm(request=r), 4736, 7, 2),
        "C4 planar quadrotor SLR, N=300, 10 x 15 iterations": (lambda r: W.c4_quadrotor(request=r), 4736, 2, 2),
    }
    out = {}
    for name, (make, count, dc, prec) in cfgs.items():
        base = [make(r) for r in range(8)]
        probs = [base[i % 8][0] for i in range(count)]
        opts = [base[i % 8][1] for i in range(count)]
        ms, trials = timed(probs, opts, prec)
        pb0, op0 = base[0]
        iters = op0.iters * max(op0.slr_iters, 1) if pb0.dyn_kind else op0.iters
        n = pb0.n
        flops = sum((pb.N + 1) * (t * fp64_flops_per_trial_state(n) + iters * fp64_flops_per_iter_state(n, dc))
                    for pb, t in zip(probs, trials))
        ach = flops * DF_EXPANSION / (ms / 1000.0) / 1e12
        form = "lane form (16 lanes per plan)" if n == 4 else "thread form (one thread per plan)"
        entry = {"batch": count, "form": form, "precision": DTYPES[prec], "ms": ms, "plans_per_s": count / (ms / 1000.0),
                 "roofline": {"bound": "alu", "achieved": ach, "peak": fp32_peak_tflops(), "unit": "TFLOP/s",
                              "frac": ach / fp32_peak_tflops(),
                              "note": "FP64-equivalent flops of the trials and updates x 9.29 FP32 flops each; "
                                      "the SLR linearisation and prior rebuilds are not counted"}}
        lat = {}
        for prec_l in (1, 2):
            lpb, lop = base[0]
            ms_l, _ = timed([lpb], [replace(lop, plan_threads=256)], prec_l)
            lat[DTYPES[prec_l]] = ms_l
        entry["single_plan_latency_ms_block_form_256"] = lat
        out[name] = entry
    return out


PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_df": 2}
DTYPES = {0: "f64", 1: "f32 quadrature + f64 recursions",
          2: "f32 quadrature + double-float (f32-pair, ~48-bit) recursions"}


def kernel_only(args):
    """One fused-iteration launch over a batch (an ncu target)."""
    from dataclasses import replace

    import torch

    import workloads as W
    from paper_2411_03416_b300 import _lib as L
    if args.kernel_workload == "dense":
        probs, opts = make_batch_problems(args.batch)
    else:
        make = {"arm": W.c3_arm, "quadrotor": W.c4_quadrotor}[args.kernel_workload]
        pairs = [make(request=r % 8) for r in range(args.batch)]
        probs, opts = [p for p, _ in pairs], [o for _, o in pairs]
    if args.kernel_n:
        # a shorter horizon of the same plans (a profiling case that fits a few GB at full occupancy)
        probs = [replace(p, N=args.kernel_n, T=p.T * args.kernel_n / p.N) for p in probs]
    iters = args.iters if args.kernel_workload == "dense" else opts[0].iters
    opts = [replace(o, iters=iters, plan_threads=args.plan_threads,
                    kl_eps=0.1 * (probs[0].N + 1) if args.kernel_n else o.kl_eps) for o in opts]
    b = L.Batch(probs, opts, PRECISIONS[args.precision])
    st = torch.cuda.Stream()
    sh = st.cuda_stream
    b.upload(sh)
    b.reset(sh)
    b.phase(L.PHASE_PRIOR, 0.0, sh)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    b.run(0, sh)
    e1.record(st)
    torch.cuda.synchronize()
    b.download_results(sh)
    torch.cuda.synchronize()
    trials = [sum(l["trials"] for l in b.result(i, full=False).logs) for i in range(args.batch)]
    ms = e0.elapsed_time(e1)
    flops = algorithmic_fp64_flops(probs, trials, iters)
    print(f"kernel-only: {args.kernel_workload}, batch {args.batch}, N {probs[0].N}, {iters} iterations, {args.precision}, "
          f"plan_threads {args.plan_threads}: {ms:.1f} ms, "
          f"{sum(trials)} trials, {flops / ms / 1e9:.4f} TFLOP/s-equivalent", flush=True)
    b.close()


DTYPES = {0: "f64", 1: "f32 quadrature + f64 recursions",
          2: "f32 quadrature + double-float (f32 pair) recursions"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)   # 2 x 38 s timed at the default batch
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=75776,
                    help="plans per GPU (75,776: one wave at 16 warps per SM in the thread form; eight waves of the "
                         "double-float lane form)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_df", "fp64"],
                    help="the batch's precision form: mixed (FP32 quadrature, FP64 recursions; the default, the form "
                         "the stated tolerances are for), mixed_df (double-float recursions) or fp64")
    ap.add_argument("--kernel-only", action="store_true",
                    help="profiling target: prior phase, then one fused-iteration launch; no JSON line")
    ap.add_argument("--iters", type=int, default=ITERS, help="proximal iterations (kernel-only mode)")
    ap.add_argument("--kernel-n", type=int, default=0, help="kernel-only mode: horizon N (0: the workload's 750)")
    ap.add_argument("--kernel-workload", default="dense", choices=["dense", "arm", "quadrotor"],
                    help="kernel-only mode: the dense-horizon batch (default), 7-DOF arm plans (N = 200, 25 "
                         "iterations) or quadrotor plans (their first linearisation's 15 iterations)")
    ap.add_argument("--plan-threads", type=int, default=0,
                    help="kernel-only mode: 0 default form, 1 thread form, 16 lane form, 32..256 block form")
    ap.add_argument("--serve-count", type=int, default=512, help="requests of the serving mix (0: skip serving)")
    ap.add_argument("--plain-count", type=int, default=32, help="requests of the plain per-request FP64 sample")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations' batch and latency runs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_only:
        return kernel_only(args)

    ws, rank, local = dist_init()
    cpu, samples = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, samples = cpu_baseline(samples=True)   # before any CUDA work: the pool is spawned, not forked

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    import paper_2411_03416_b300 as pg
    from paper_2411_03416_b300 import _lib as L

    probs, opts = make_batch_problems(args.batch, rank)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    def make(precision):
        b = L.Batch(probs, opts, precision)
        b.upload(sh)
        torch.cuda.synchronize()
        return b

    def time_steps(precision, steps):
        b = make(precision)
        plan_step(b)
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan_step(b)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        b.close()
        ms = statistics.median(times)
        return {"value": args.batch * ws / max_over_ranks(ws, ms / 1000.0), "unit": "plans/s", "ms_per_step": ms}

    def plan_step(b):
        b.reset(sh)
        b.run(0, sh)

    # ---- served form, device-resident inputs
    head = PRECISIONS[args.precision]
    bm = make(head)
    for _ in range(args.warmup):
        plan_step(bm)
    torch.cuda.synchronize()
    barrier(ws)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev_run = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for k in range(args.steps):
            ev[k][0].record(stream)
            bm.reset(sh)
            ev_run[k].record(stream)     # the run: prior, init, fused iterations, finalize
            bm.run(0, sh)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1000.0
    t_max = max_over_ranks(ws, t_dev)
    value = args.batch * ws * args.steps / t_max

    # ---- dominant kernel: the fused-iteration launch, timed inside the timed steps.  Each run's
    # interval also holds its prior, init and finalize launches (by the ncu launch lists 0.4% of it in the
    # thread form with FP64 recursions, 1.9% in the double-float lane form),
    # so the achieved rate below is a slight underestimate.  Trial counts come from the last step.
    run_ms = [a.elapsed_time(b[1]) for a, b in zip(ev_run, ev)]
    bm.download_results(sh)
    torch.cuda.synchronize()
    trials = []
    statuses = 0
    # invariants of every plan of the timed batch: all iterations ran, every
    # accepted step meets the KL bound and is a dyadic fraction of beta_max
    incomplete, kl_over, off_grid = 0, 0, 0
    for i in range(args.batch):
        r = bm.result(i, full=False)
        trials.append(sum(l["trials"] for l in r.logs))
        op = opts[i]
        incomplete += int(len(r.logs) != op.iters)
        for l in r.logs:
            if l["beta"] > 0:
                kl_over += int(l["kl"] > op.kl_eps * (1 + 1e-12))
                q = l["beta"] / op.beta_max * 2 ** op.max_bisect
                off_grid += int(abs(q - round(q)) > 1e-9)
    invariants = {"plans": args.batch, "incomplete": incomplete, "kl_above_bound": kl_over,
                  "step_not_dyadic": off_grid, "pass": incomplete == 0 and kl_over == 0 and off_grid == 0}
    state_trials = sum((pb.N + 1) * t for pb, t in zip(probs, trials))
    flops = algorithmic_fp64_flops(probs, trials)
    k_ms = sum(run_ms) / len(run_ms)
    traffic, traffic_note, executed = None, "no capture of this form's kernel", None
    lane = head == 2   # the default form of n = 4 plans: the lane form with double-float, the thread form otherwise
    if head == 1 and THREAD_F64_DRAM_BYTES_PER_STATE_TRIAL:
        traffic = THREAD_F64_DRAM_BYTES_PER_STATE_TRIAL * state_trials
        traffic_note = ("bytes per launch: ncu dram bytes per state-trial of a 2,368-plan, 30-iteration capture of "
                        f"this kernel x this launch's {state_trials} state-trials "
                        f"({traffic / (k_ms / 1000.0) / 1e9:.0f} GB/s over the launch)")
    if head == 2:
        flops32 = flops * DF_EXPANSION
        achieved = flops32 / (k_ms / 1000.0) / 1e12
        peak = fp32_peak_tflops()
        roof_kind = ("FP32 pipe (double-float recursions): counted FP64 flops x 9.29 FP32 flops each (the double-float "
                     "primitives' op counts); peak derived from unit counts and clock (measured FFMA loop: 68.2)")
        if lane:
            traffic = LANE_DF_DRAM_BYTES_PER_STATE_TRIAL * state_trials
            traffic_note = ("bytes per launch: ncu dram bytes per state-trial of a 2,368-plan, 30-iteration capture of "
                            f"this kernel x this launch's {state_trials} state-trials "
                            f"({traffic / (k_ms / 1000.0) / 1e9:.0f} GB/s over the launch)")
            ex = LANE_DF_EXECUTED_FP32_PER_STATE_TRIAL * state_trials / (k_ms / 1000.0) / 1e12
            executed = {"fp32_tflops": ex, "frac": ex / peak, "measured_df_expansion": LANE_DF_MEASURED_EXPANSION,
                        "note": ("FP32 flops the kernel executes (ncu counters per state-trial x state-trials), "
                                 "replicated lane work included")}
            kernel_name = "k_iterate_lane<float, df64> (fused iterations, lane form: 16 lanes per plan)"
        else:
            kernel_name = "k_iterate<4, float, df64> (fused iterations, thread form)"
    else:
        achieved = flops / (k_ms / 1000.0) / 1e12
        peak = fp64_peak_tflops()
        roof_kind = "FP64 derived from unit counts and clock (measured DFMA loop: 0.935)"
        kernel_name = (f"k_iterate_lane<{'float' if head == 1 else 'double'}, double> (lane form)" if lane else
                       f"k_iterate<4, {'float' if head == 1 else 'double'}, double> (fused iterations, thread form)")

    # ---- e2e through the C ABI with host buffers
    h2d, d2h_full, d2h = bm.io_bytes()
    torch.cuda.synchronize()
    e2e_ms = []
    e2e_steps = max(1, min(2, args.steps))
    for k in range(1 + e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        bm.upload(sh)
        plan_step(bm)
        bm.download_results(sh)
        stream.synchronize()
        if k:
            e2e_ms.append(1000.0 * (time.perf_counter() - t))
    e2e_max = max_over_ranks(ws, sum(e2e_ms) / 1000.0)
    e2e_value = args.batch * ws * e2e_steps / e2e_max
    bm.close()
    check = sample_check(samples, head) if samples else None
    check_df = sample_check(samples, 2) if (samples and head != 2) else None

    # ---- the other forms on the same batch
    others = {}
    if args.plain_steps > 0:
        others["plain_fp64"] = time_steps(L.PREC_PLAIN_FP64, args.plain_steps)
        if head != L.PREC_MIXED:
            others["served_fp64_recursions"] = time_steps(L.PREC_MIXED, args.plain_steps)
        if head != L.PREC_MIXED_DF:
            others["served_double_float_recursions"] = time_steps(L.PREC_MIXED_DF, args.plain_steps)

    serve = serving(args) if (args.serve_count > 0 and rank == 0) else None
    configs = other_configs(args) if (rank == 0 and not args.no_configs) else None

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "plans/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": config_dict(args.batch, ws),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "note": "batch latency: every plan of a step completes at the end of the step"},
        **others,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "fp64_equivalent": {"achieved": flops / (k_ms / 1000.0) / 1e12, "peak": fp64_peak_tflops(),
                                         "frac": flops / (k_ms / 1000.0) / 1e12 / fp64_peak_tflops(),
                                         "note": "the method's FP64 flops against the FP64 pipe's peak"},
                     "traffic": traffic, "traffic_note": traffic_note, "executed": executed,
                     "kernel": kernel_name, "kernel_ms": k_ms, "peak_kind": roof_kind,
                     "kernel_timing": ("CUDA events on the launching stream around the batch run of every timed "
                                       "step, averaged; the interval adds the prior, init and finalize launches "
                                       "(0.4% of it with FP64 recursions, 1.9% in the double-float lane form)"),
                     "algorithmic_fp64_equivalent_flops": flops},
        "cpu_baseline": cpu,
        "checks": {"invariants": invariants, "sample_vs_oracle": check,
                   "sample_vs_oracle_double_float_recursions": check_df},
        "e2e": {"value": e2e_value, "unit": "plans/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.median(e2e_ms)},
        "serving": serve,
        "configs": configs,
        "clocks": clk.summary(),
        "gpu_launches": 4 * args.steps,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
