#!/usr/bin/env python
"""Benchmark of the task-DAG executor on one B300 (or N replicas).

Headline: plain FP64 tiled Cholesky, N = 32768, tile 512 (64 x 64 tiles,
45,760 POTRF / TRSM / SYRK / GEMM tasks), A = B B^T / N + 0.1 I, seed 3,
submitted in right-looking order with R / RW modes and run as ONE
persistent-kernel launch per factorisation (the DAG is captured once into a
CUDA graph and replayed).  Metric: TFLOP/s = (N^3/3 + N^2/2 + N/6) / time.

Secondary (same JSON line, "secondary"): vector-scaling chains (n = 2^28
binary32, 256 blocks x 8 chained RW tasks) in task-level GB/s, scheduler
throughput in tasks/s on empty-bodied DAGs (1000 chains; fan-out / fan-in;
the Cholesky DAG at T = 64), the small Cholesky (N = 1024, tile 128, 120
tasks) in ms, time to solution with mixed precision and refinement, and
serving with continuous batching against the per-request path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --case serve_sweep | trace_headline | empty_dags | <kind>

--impl reference times the oracle (the sequential CPU executor) on the same
workload, a bounded sample of it per step, on the host cores.
Under torchrun every rank runs an independent replica (the DAG does not
shard); rank 0 prints one JSON line with the max time over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAK_FP64_FLOP_PER_CLK_SM = 4      # two DFMA per clock per SM on sm_103
NUM_SMS = 148
SM_MAX_MHZ = 2032.0
FALLBACK_HBM_GBS = 6400.0           # one earlier copy measurement on a B300


def hbm_peak():
    """Measured copy bandwidth of the B300s (GB/s) and its source."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Measured dense bf16 burst throughput (TFLOP/s) and its source."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1800.0, "fallback"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=32768)
    p.add_argument("--b", type=int, default=512)
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--nrhs", type=int, default=16)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-scipy", action="store_true", help="skip the LAPACK CPU baselines (scipy, all host cores)")
    p.add_argument("--no-sliced-resid", action="store_true",
                   help="time to solution: skip the refinement with the sliced FP64 residual (tensor cores)")
    p.add_argument("--mx-trsm", default="inv,sliced",
                   help="mixed panel solves to time, comma-separated: inv (TRTRI + TRMM_MX, FP64 DFMA), "
                        "sliced (TRTRI + TRMM_SL, the product on the tensor cores), subst (TRSM_MX); "
                        "both = inv,subst.  The traced case (--case trace_mixed) takes the first")
    p.add_argument("--serve-requests", type=int, default=2000,
                   help="requests served with continuous batching, per precision (serving sweep: per rate)")
    p.add_argument("--serve-distinct", type=int, default=128,
                   help="distinct client inputs (the first requests of the stream), cycled over the run")
    p.add_argument("--serve-plain-requests", type=int, default=256,
                   help="requests of the same stream served by the per-request path")
    p.add_argument("--prio", default="critical", choices=["critical", "upward", "depth"],
                   help="ready-queue order (b3t_config.prio_policy) of the headline context, the time to solution "
                        "and the profiling cases (--case); the vector chains and empty DAGs set their own")
    p.add_argument("--ctas-per-sm", type=int, default=0, help="grid of the profiling cases (0: occupancy)")
    p.add_argument("--item-chains", action="store_true",
                   help="profiling cases: run vector-scaling chains item by item (b3t_config.item_chains)")
    p.add_argument("--case", default=None, choices=["mx_gemm_bf16", "mx_gemm_e4m3", "scal", "resid", "resid_sl", "trmm_sl", "solve_f32", "trace_mixed",
                                                    "solve_f64", "empty_dags", "serve_sweep", "trace_headline", "batch",
                                                    "trace_solve"],
                   help="run one profiling case (a DAG of one task kind), or one secondary measurement alone "
                        "(empty_dags, serve_sweep, trace_headline, batch), and print its result")
    return p.parse_args()


def prio_of(args):
    import paper_1304_0878_b300 as b3t
    return {"upward": b3t.PRIO_UPWARD, "depth": b3t.PRIO_DEPTH, "critical": b3t.PRIO_CRITICAL}[args.prio]


def cholesky_flops(N):
    return float(N * (N + 1) * (2 * N + 1) // 6)


class Clocks:
    """nvidia-smi sampling during the timed region (every 200 ms)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def provenance():
    """What the line was measured on: host cores, the library sources'
    hash, and the git revision when the tree is a checkout."""
    out = {"host_cores": len(os.sched_getaffinity(0)), "source_hash": None, "git_rev": None}
    try:
        import paper_1304_0878_b300.build as pb
        out["source_hash"] = pb.source_hash()
    except Exception:
        pass
    try:
        top = subprocess.check_output(["git", "-C", ROOT, "rev-parse", "--show-toplevel"],
                                      stderr=subprocess.DEVNULL, text=True).strip()
        if os.path.realpath(top) == os.path.realpath(ROOT):
            out["git_rev"] = subprocess.check_output(["git", "-C", ROOT, "rev-parse", "HEAD"],
                                                     stderr=subprocess.DEVNULL, text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        pass
    return out


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def recorded_traffic(key):
    """DRAM bytes (read + write) per launch that an ncu capture recorded for
    this workload, or None when none exists or the kernel sources changed
    since (profiles/ncu_traffic.json holds the source hash)."""
    import paper_1304_0878_b300.build as pb
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[key]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_hash") != pb.source_hash():
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def max_over_ranks(ms, device=None):
    """Per-step time of the slowest rank (replicas run the same workload
    independently; the whole job is as slow as its slowest replica)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_replica, ms, world):
    """Whole-job value: the work of every replica over the slowest time."""
    return world * flops_per_replica / (ms / 1e3) / 1e12


def oracle_sample(get_tile, T, b, seconds):
    """The oracle on a bounded prefix of the submission order (1 core)."""
    import oracle
    from oracle import cholesky as och
    oracle.build()
    done, fl, sec = och.run_prefix(get_tile, T, b, seconds)
    return {"value": fl / sec / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": "first %d tasks (%.3g flop) of the N=%d, b=%d submission order in %.1f s"
                      % (done, fl, T * b, b, sec)}


def host_tile_getter(N, b, seed, shift):
    """Tiles of A = B B^T/N + shift I formed on the host in FP64 (no GPU)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((N, N))

    def get(i, j):
        blk = B[i * b:(i + 1) * b] @ B[j * b:(j + 1) * b].T / N
        if i == j:
            blk[np.diag_indices(b)] += shift
        return np.ascontiguousarray(blk.T)
    return get


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    N, b = args.n, args.b
    T = N // b
    get = None
    try:
        import torch
        if torch.cuda.is_available():
            import synth
            A0 = synth.spd_tiles_device(N, b, 3, 0.1, "cuda")
            from paper_1304_0878_b300.tiles import tile_index

            def get(i, j):
                return A0[tile_index(i, j, T)].cpu().numpy()
    except ImportError:
        pass
    if get is None:
        get = host_tile_getter(N, b, 3, 0.1)
    per = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    vals = []
    for s in range(args.warmup + args.steps):
        r = oracle_sample(get, T, b, per)
        if s >= args.warmup:
            vals.append(r)
    v = float(np.mean([r["value"] for r in vals]))
    flops = cholesky_flops(N)
    line = {"impl": "reference", "metric": "cholesky_fp64_tflops", "value": v, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": flops / (v * 1e12) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(N, b),
                       "execution": "the oracle: sequential CPU executor, C tile routines, one host core; "
                                    "a bounded prefix of the submission order per step"},
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "provenance": provenance()}
    print(json.dumps(line))


def workload_config(N, b):
    """The headline workload, named the same way by both arms."""
    return {"workload": "tiled Cholesky FP64 N=%d tile %d (%d POTRF/TRSM/SYRK/GEMM tasks), "
                        "A = B B^T/N + 0.1 I, B ~ N(0,1) seed 3" % (N, b, len_tasks(N // b)),
            "N": N, "tile": b, "tasks": len_tasks(N // b), "seed": 3, "shift": 0.1}


def len_tasks(T):
    return T + T * (T - 1) + T * (T - 1) * (T - 2) // 6


def sampled_residual(t, A0, N, b, nsamp=24, seed=0):
    """max |(L L^T - A)_ij| / max |A_ij| over sampled lower (i, j): rows of L
    gathered from the tiles, products formed on the device."""
    import torch
    from paper_1304_0878_b300.tiles import tile_index
    T = N // b
    rng = np.random.default_rng(seed)

    def row(M, i):
        I, r = divmod(i, b)
        return torch.cat([M[tile_index(I, J, T), :, r] for J in range(I + 1)])

    worst = 0.0
    for _ in range(nsamp):
        i = int(rng.integers(0, N))
        j = int(rng.integers(0, i + 1))
        li, lj = row(t, i)[: i + 1], row(t, j)[: j + 1]
        m = min(i, j) + 1
        v = float(torch.dot(li[:m], lj[:m]))
        a = float(row(A0, i)[j])
        worst = max(worst, abs(v - a))
    return worst / float(A0.abs().max())


def run_ours(args):
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    import paper_1304_0878_b300.build as pb

    ws, rank, local = dist()
    pb.build()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = b3t.Context(stream=stream.cuda_stream, timeout_ns=120_000_000_000, prio_policy=prio_of(args))
    N, b = args.n, args.b
    T = N // b
    flops = cholesky_flops(N)

    A0 = synth.spd_tiles_device(N, b, 3, 0.1, dev)
    a_bytes = A0.numel() * A0.element_size()
    t = torch.empty_like(A0)
    ptrs = dt.tile_ptrs(t)
    ctx.graph_capture_begin()
    ctx.cholesky_submit(ptrs, T, b)
    ctx_tasks = ctx.dag_stats()[0]
    g = ctx.graph_capture_end()

    def step():
        t.copy_(A0)
        ctx.graph_replay(g)
        ctx.task_wait()
        return ctx.last_launch()["kernel_ns"]

    for _ in range(args.warmup):
        step()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device())
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kns = []
    for _ in range(args.steps):
        kns.append(step())
    e1.record(stream)
    barrier()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    resid = sampled_residual(t, A0, N, b)
    kernel_s = float(np.mean(kns)) / 1e9
    achieved = flops / kernel_s / 1e12
    peak = NUM_SMS * PEAK_FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12

    # end to end through the public API: pinned host A in, L out, every step
    e2e = None
    if not args.no_e2e:
        hA = torch.empty(A0.shape, dtype=A0.dtype, pin_memory=True)
        hA.copy_(A0)
        hL = torch.empty_like(hA, pin_memory=True)
        ke = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(ke):
            t.copy_(hA, non_blocking=True)
            ctx.graph_replay(g)
            ctx.task_wait()
            hL.copy_(t, non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        mse = e2.elapsed_time(e3) / ke
        nbytes = A0.numel() * A0.element_size()
        e2e = {"value": ws * flops / (mse / 1e3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": mse,
               "note": "per step: pinned host A -> device, replay of the captured DAG (task table built once, "
                       "its host-side dependency derivation outside the timed region), L -> pinned host"}
        del hA, hL

    nctas = ctx.last_launch()["nctas"]
    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        from paper_1304_0878_b300.tiles import tile_index

        def get(i, j):
            return A0[tile_index(i, j, T)].cpu().numpy()
        cpu = oracle_sample(get, T, b, args.cpu_seconds)
        if not args.no_secondary:
            cpu["empty_dags"] = oracle_empty_dags(min(3.0, args.cpu_seconds / 5))
        if not args.no_serve:
            cpu["serving_scipy"] = scipy_serving_sample(min(10.0, args.cpu_seconds), args.serve_requests)
        if not args.no_scipy:
            cpu["library"] = scipy_baselines(A0.cpu().numpy(), N, b, args.nrhs)

    secondary = {}
    if not args.no_secondary:
        secondary = run_secondary(ctx, dev, stream)
    if not args.no_mixed:
        secondary["time_to_solution"] = run_time_to_solution(ctx, A0, t, g, N, b, dev, stream, args)
    if not args.no_serve:
        del A0, t
        torch.cuda.empty_cache()
        secondary["serving"] = run_serving(dev, args)

    ctx.graph_destroy(g)
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": "cholesky_fp64_tflops", "value": job_throughput(flops, ms, ws), "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {**workload_config(N, b),
                   "execution": "one persistent-kernel launch per factorisation, DAG captured once and replayed; "
                                "each diagonal POTRF runs as a panel DAG (%d device tasks)" % ctx_tasks,
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "inputs (%.2f GB of tiles) larger than L2" % (a_bytes / 1e9),
                   "input_reset": "A tiles restored by a device copy inside each step",
                   "persistent_ctas": nctas, "ready_queue": args.prio},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": recorded_traffic("cholesky_fp64_n%d_b%d" % (N, b)),
                     "note": "FP64 DFMA pipe: 148 SMs x 4 flop/clk x 2032 MHz; achieved = "
                             "N^3/3 flops / persistent-kernel time"},
        "check": {"sampled_rel_residual": resid},
        "clocks": ck,
        "gpu_launches": 2 * args.steps,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "secondary": secondary,
        "provenance": provenance(),
    }
    line["summary"] = summarise(line)
    print(json.dumps(line))


def summarise(line):
    """The figures a reader needs first, last on the line (a log tail keeps them)."""
    sec = line.get("secondary") or {}
    g = lambda d, *ks: _dig(d, ks)
    out = {"cholesky_fp64_tflops": line["value"], "roofline_frac": line["roofline"]["frac"],
           "e2e_tflops": g(line, "e2e", "value")}
    for k in ("vector_chains", "vector_chains_depth_first"):
        if k in sec:
            out[k] = {"ms": sec[k]["ms"], "hbm_frac": sec[k]["hbm_frac"]}
    if "vector_chains_item_chains" in sec:
        v = sec["vector_chains_item_chains"]
        out["vector_chains_item_chains"] = {"ms": v["ms"], "floor_ms": v["floor_ms"], "hbm_frac": v["hbm_frac"]}
    ed = sec.get("empty_dags") or {}
    tps = {k: v["tasks_per_s"] for k, v in ed.items()}
    if "tasks_per_s" in sec:
        tps["chains_100k"] = sec["tasks_per_s"]["value"]
    if tps:
        out["tasks_per_s"] = tps
    for k in ("cholesky_small", "cholesky_small_fifo"):
        if k in sec:
            out[k + "_ms"] = sec[k]["ms"]
    tts = sec.get("time_to_solution")
    if tts:
        out["time_to_solution"] = {"fp64_ms": tts["fp64"]["ms"]}
        for p in ("bf16", "e4m3", "bf16_sliced_panel", "e4m3_sliced_panel"):
            if p in tts:
                out["time_to_solution"][p] = {k: tts[p][k] for k in ("ms", "factor_ms", "speedup_vs_fp64", "eta",
                                                                      "host_sampled_eta", "iterations")}
                if "sliced_residual" in tts[p]:
                    out["time_to_solution"][p]["sliced_residual"] = {
                        k: tts[p]["sliced_residual"][k] for k in ("ms", "speedup_vs_fp64", "eta", "host_sampled_eta",
                                                                   "iterations")}
    sv = sec.get("serving")
    if sv:
        out["serving"] = {}
        for p in ("fp64", "bf16"):
            if p in sv:
                c, pl = sv[p]["continuous"], sv[p]["plain"]
                out["serving"][p] = {"requests": c["requests"], "p50_ms": c["p50_ms"], "p99_ms": c["p99_ms"],
                                     "solves_per_s": c["solves_per_s"], "max_queue": c.get("max_queue"),
                                     "plain_requests": pl["requests"], "plain_solves_per_s": pl["solves_per_s"],
                                     "plain_p99_ms": pl["p99_ms"]}
    cpu = line.get("cpu_baseline") or {}
    if cpu:
        out["cpu"] = {"oracle_tflops_1core": cpu.get("value"),
                      "scipy_cholesky_n32768_tflops": g(cpu, "library", "cholesky_n32768", "TFLOPs"),
                      "scipy_cholesky_n1024_ms": g(cpu, "library", "cholesky_n1024", "ms"),
                      "scipy_cores": g(cpu, "library", "cores")}
    return out


def _dig(d, ks):
    for k in ks:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def host_sym_row(tl, i, N, b):
    """Row i of the symmetric A from its packed lower tiles on the host
    (tl[t][c, r] = element (I*b + r, J*b + c) of tile t = (I, J))."""
    from paper_1304_0878_b300.tiles import tile_index
    T = N // b
    I, r = divmod(i, b)
    parts = [tl[tile_index(I, J, T)][:, r] for J in range(I + 1)]        # row r of tiles (I, J), J <= I
    parts[-1] = np.concatenate([parts[-1][: r + 1], tl[tile_index(I, I, T)][r, r + 1:]])
    parts += [tl[tile_index(J, I, T)][r, :] for J in range(I + 1, T)]    # column r of tiles (J, I), J > I
    return np.concatenate(parts)


def host_anorm(tl, N, b):
    """Exact ||A||_inf of the symmetric A from its lower tiles, in FP64 on the host."""
    from paper_1304_0878_b300.tiles import tile_index
    T = N // b
    rows = np.zeros(N)
    for j in range(T):
        for i in range(j, T):
            F = np.abs(tl[tile_index(i, j, T)].T)                        # F[r, c] = A(i*b + r, j*b + c)
            if i == j:
                F = np.tril(F) + np.tril(F, -1).T
                rows[i * b:(i + 1) * b] += F.sum(axis=1)
            else:
                rows[i * b:(i + 1) * b] += F.sum(axis=1)
                rows[j * b:(j + 1) * b] += F.sum(axis=0)
    return float(rows.max())


def sampled_host_eta(tl, anorm, X, Bh, N, b, nsamp=32, seed=1):
    """Normwise backward error of the device solution X (N x nrhs) on sampled
    rows: |b_i - A_i X| / (||A||_inf max|x_j| + max|b_j|), the residual rows
    formed in FP64 on the host from the stored A (the check the oracle's
    backward_error makes, restricted to rows it can afford at this size)."""
    rng = np.random.default_rng(seed)
    xn = np.abs(X).max(axis=0)
    bn = np.abs(Bh).max(axis=0)
    worst = 0.0
    for _ in range(nsamp):
        i = int(rng.integers(0, N))
        r = Bh[i] - host_sym_row(tl, i, N, b) @ X
        worst = max(worst, float(np.max(np.abs(r) / (anorm * xn + bn))))
    return worst


def scipy_baselines(tl, N, b, nrhs):
    """Library CPU baselines on all host cores (LAPACK through scipy): the
    FP64 Cholesky of the N = 1024 matrix (seed 0), and of the N = 32768
    matrix (the same bytes as the device's A, assembled from the tiles) with
    the FP64 solve of the 16 right-hand sides (seed 4)."""
    import scipy.linalg as sla
    import synth
    cores = len(os.sched_getaffinity(0))
    out = {"kind": "scipy.linalg (LAPACK) FP64 on the host", "cores": cores}
    A1 = synth.spd_host(1024, seed=0, shift=1.0)
    ts = []
    for _ in range(7):
        t0 = time.perf_counter()
        sla.cholesky(A1, lower=True, check_finite=False)
        ts.append(time.perf_counter() - t0)
    m1 = float(np.median(ts[2:]))
    out["cholesky_n1024"] = {"ms": 1e3 * m1, "TFLOPs": cholesky_flops(1024) / m1 / 1e12}
    from paper_1304_0878_b300.tiles import tile_index
    T = N // b
    A = np.zeros((N, N), order="F")
    for j in range(T):
        for i in range(j, T):
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = tl[tile_index(i, j, T)].T
    t0 = time.perf_counter()
    c = sla.cho_factor(A, lower=True, overwrite_a=True, check_finite=False)
    tf = time.perf_counter() - t0
    Bh = synth.rhs(N, nrhs, seed=4)
    t0 = time.perf_counter()
    sla.cho_solve(c, Bh, check_finite=False)
    tsv = time.perf_counter() - t0
    out["cholesky_n%d" % N] = {"s": tf, "TFLOPs": cholesky_flops(N) / tf / 1e12}
    out["solve_n%d" % N] = {"ms": 1e3 * tsv, "nrhs": nrhs, "time_to_solution_s": tf + tsv}
    del A, c
    return out


def rhs_parts(N, b, nrhs, seed, dev):
    """N(0,1) right-hand sides as T parts of b x nrhs (column-major)."""
    import torch
    import synth
    B = synth.rhs(N, nrhs, seed=seed)
    T = N // b
    return torch.from_numpy(np.ascontiguousarray(B.reshape(T, b, nrhs).transpose(0, 2, 1))).to(dev)


def mx_modes(args):
    m = args.mx_trsm.replace("both", "inv,subst").split(",")
    for x in m:
        if x not in ("inv", "sliced", "subst"):
            raise SystemExit("--mx-trsm: unknown panel solve %r" % x)
    return list(dict.fromkeys(m))


def run_time_to_solution(ctx, A0, t, g64, N, b, dev, stream, args):
    """Config 4: 16 right-hand sides to backward error <= 1e-12.
    FP64: FP64 factorisation (graph g64 on tiles t) + one FP64 solve step.
    Mixed: binary32 working tiles, bf16 / E4M3 tensor-core updates, FP64
    POTRF / TRSM, then iterative refinement (binary32 correction solves,
    FP64 residual) until eta <= 1e-12.  Times are device-event wall times of
    the whole solution, inputs resident."""
    import torch
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    import synth
    T = N // b
    nrhs = args.nrhs
    Bd = rhs_parts(N, b, nrhs, 4, dev)
    # per-result error against FP64, checked on the host: A's tiles, its exact
    # infinity norm, and the right-hand sides
    tl = A0.cpu().numpy()
    anorm = host_anorm(tl, N, b)
    Bh = synth.rhs(N, nrhs, seed=4)

    def host_eta(X):
        Xh = X.cpu().numpy().transpose(0, 2, 1).reshape(N, nrhs)
        return sampled_host_eta(tl, anorm, Xh, Bh, N, b)
    R = torch.zeros(b3t.ir_work_elems(T, b, nrhs), dtype=torch.float64, device=dev)
    eta = torch.zeros(nrhs + 1, dtype=torch.float64, device=dev)
    sliced = not args.no_sliced_resid and b % 128 == 0 and nrhs <= 16
    S = torch.empty(b3t.ir_slice_bytes(T, b) + 256, dtype=torch.uint8, device=dev) if sliced else None
    s_ptr = (S.data_ptr() + 255) // 256 * 256 if sliced else 0
    flops = cholesky_flops(N)
    out = {"workload": "N=%d tile %d, %d right-hand sides N(0,1) seed 4, target eta <= 1e-12" % (N, b, nrhs)}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def solve(Lp, X, flags, max_iter):
        return ctx.ir_solve(A0.data_ptr(), Lp, Bd.data_ptr(), X.data_ptr(), R.data_ptr(), eta.data_ptr(),
                            T, b, nrhs, flags, 1e-12, max_iter)

    # FP64 reference path
    X64 = torch.zeros_like(Bd)
    res = []
    for rep in range(2):
        t.copy_(A0)
        ev[0].record(stream)
        ctx.graph_replay(g64)
        ctx.task_wait()
        ev[1].record(stream)
        rc, its, e = solve(dt.tile_ptrs(t), X64, 0, 1)
        ev[2].record(stream)
        torch.cuda.synchronize()
        res.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), rc, its, e[nrhs]))
    f_ms, s_ms, rc, its, e64 = res[-1]
    out["fp64"] = {"ms": f_ms + s_ms, "factor_ms": f_ms, "solve_ms": s_ms, "eta": e64, "rc": rc,
                   "host_sampled_eta": host_eta(X64),
                   "effective_TFLOPs": flops / ((f_ms + s_ms) / 1e3) / 1e12}
    # mixed precision + refinement
    W = torch.empty(A0.shape, dtype=torch.float32, device=dev)
    Lm = torch.zeros_like(A0)
    U = torch.zeros((T, b, b), dtype=torch.float64, device=dev)
    up = dt.tile_ptrs(U)
    modes = mx_modes(args)
    suffix = {"inv": "", "sliced": "_sliced_panel", "subst": "_substitution"}
    variants = [(fmt, nm + suffix[m], m) for m in modes for fmt, nm in ((b3t.FMT_BF16, "bf16"), (b3t.FMT_E4M3, "e4m3"))]
    WS = US = None
    if "sliced" in modes:
        WS = torch.zeros((T * (T + 1) // 2, b3t.slice_w_bytes(b)), dtype=torch.uint8, device=dev)
        US = torch.zeros((T, b3t.slice_u_bytes(b)), dtype=torch.uint8, device=dev)
    for fmt, name, mode in variants:
        Q = dt.q_tiles(T, b, fmt, dev)
        wp, lp, qp = dt.tile_ptrs(W), dt.tile_ptrs(Lm), dt.tile_ptrs(Q)
        ctx.graph_capture_begin()
        if mode == "inv":
            ctx.cholesky_mx_inv_submit(wp, lp, qp, up, T, b, fmt)
        elif mode == "sliced":
            ctx.cholesky_mx_sliced_submit(wp, lp, qp, up, dt.tile_ptrs(WS), dt.tile_ptrs(US), T, b, fmt)
        else:
            ctx.cholesky_mx_submit(wp, lp, qp, T, b, fmt)
        gm = ctx.graph_capture_end()
        Xm = torch.zeros_like(Bd)
        res = []
        for rep in range(3):
            ev[0].record(stream)
            W.copy_(A0)
            ctx.graph_replay(gm)
            ctx.task_wait()
            ev[1].record(stream)
            rc, its, e = solve(lp, Xm, b3t.VEC_F32, 30)
            ev[2].record(stream)
            torch.cuda.synchronize()
            res.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), rc, its, e[nrhs]))
        f_ms, s_ms, rc, its, em = res[-1]
        diff = float((Xm - X64).abs().max() / X64.abs().max())
        sl = None
        if sliced:
            # the same factor refined with the sliced FP64 residual (SLICE_A
            # once, then SLICE_X + RESID_SL every step, on the tensor cores)
            Xs = torch.zeros_like(Bd)
            sres = []
            for rep in range(2):
                Xs.zero_()
                ev[2].record(stream)
                rc2, its2, e2 = ctx.ir_solve_sliced(A0.data_ptr(), lp, Bd.data_ptr(), Xs.data_ptr(), R.data_ptr(),
                                                    s_ptr, eta.data_ptr(), T, b, nrhs, b3t.VEC_F32, 1e-12, 30)
                ev[3].record(stream)
                torch.cuda.synchronize()
                sres.append((ev[2].elapsed_time(ev[3]), rc2, its2, e2[nrhs]))
            r_ms, rc2, its2, e2m = sres[-1]
            sl = {"ms": f_ms + r_ms, "refine_ms": r_ms, "iterations": its2, "eta": e2m, "converged": rc2 == 0,
                  "host_sampled_eta": host_eta(Xs),
                  "max_rel_diff_vs_fp64_solution": float((Xs - X64).abs().max() / X64.abs().max()),
                  "speedup_vs_fp64": out["fp64"]["ms"] / (f_ms + r_ms)}
            del Xs
        panel = {"inv": "TRTRI + TRMM_MX (inverted diagonal tile, FP64 DFMA)",
                 "sliced": "TRTRI + TRMM_SL (inverted diagonal tile, the product sliced onto the tensor cores)",
                 "subst": "TRSM_MX (substitution)"}[mode]
        out[name] = {"panel_solve": panel,
                     "ms": f_ms + s_ms, "factor_ms": f_ms, "refine_ms": s_ms, "iterations": its, "eta": em,
                     "host_sampled_eta": host_eta(Xm),
                     "converged": rc == 0, "max_rel_diff_vs_fp64_solution": diff,
                     "effective_TFLOPs": flops / ((f_ms + s_ms) / 1e3) / 1e12,
                     "speedup_vs_fp64": (out["fp64"]["ms"]) / (f_ms + s_ms)}
        if sl is not None:
            out[name]["sliced_residual"] = sl
        ctx.graph_destroy(gm)
        ctx.tiles_unregister(qp, T)
        # the panel forms partition the diagonal tiles differently (64- or
        # 128-wide panels): the next variant registers the tiles anew
        ctx.tiles_unregister(wp, T)
        ctx.tiles_unregister(lp, T)
        del Q
    for p in up:
        ctx.data_unregister(ctx.data_lookup(p))
    out["host_check"] = ("host_sampled_eta: 32 sampled rows of b - A x formed in FP64 on the host from the "
                         "stored A and B, with the exact ||A||_inf")
    return out


def run_serving(dev, args):
    """Config 5 (bounded window): the first requests of the seed-5 stream
    (Poisson 2000/s, N log-uniform in [256, 8192], 1..32 right-hand sides),
    served with continuous batching (one resident executor) and, on a prefix
    of the same stream, one at a time (plain per-request path).  Each
    request's A and B are uploaded from pinned host memory at admission and
    its X downloaded at completion, both inside the latency."""
    import torch
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import serve as sv
    n, P, n_plain = args.serve_requests, args.serve_distinct, min(args.serve_plain_requests, args.serve_requests)
    out = {"workload": "first %d requests of the 100k-request Poisson 2000/s stream (seed 5), N log-uniform "
                       "[256, 8192], 1-32 rhs, A = B B^T/N + I; client inputs of the first %d requests held in "
                       "pinned host memory and cycled (request i carries the inputs of request i mod %d); "
                       "latency = arrival -> X in host memory, upload of A and B and download of X included; "
                       "plain per-request path on the first %d requests" % (n, P, P, n_plain)}
    for prec in ("fp64", "bf16"):
        pool = {}
        sstream = torch.cuda.Stream(device=dev)
        # an FP64-only stream runs the resident kernel without the tensor-memory
        # path (two CTAs per SM)
        ctx = b3t.Context(stream=sstream.cuda_stream, timeout_ns=60_000_000_000, stream_no_mx=prec == "fp64")
        reqs = sv.make_requests(n, 2000.0, 5, prec=prec, distinct=P)
        gen_s, pinned = sv.prepare(reqs, pool=pool)
        cont = sv.serve(ctx, reqs, prec=prec, budget_bytes=64 << 30, max_inflight=48, time_limit=600.0)
        cont["input_generation_s"] = gen_s
        cont["pinned_input_bytes"] = pinned
        ctx.close()
        ctx2 = b3t.Context(stream=torch.cuda.current_stream(dev).cuda_stream, timeout_ns=60_000_000_000)
        reqs2 = sv.make_requests(n_plain, 2000.0, 5, prec=prec, distinct=P)
        sv.prepare(reqs2, pool=pool)
        plain = sv.serve_plain(ctx2, reqs2, prec=prec, time_limit=600.0)
        ctx2.close()
        out[prec] = {"continuous": cont, "plain": plain}
        del reqs, reqs2, pool
        torch.cuda.empty_cache()
    return out


EMPTY_DAGS = (("chains", "1000 chains x 1000 RW tasks, submitted level by level (1M tasks)"),
              ("fan", "1000 rounds of one writer of a shared buffer and 999 readers of it that each "
                      "update a buffer of their own (fan-out, then a 999-way fan-in; 1M tasks)"),
              ("cholesky", "the tiled Cholesky DAG at T = 64 with empty bodies (45,760 tasks)"))


def empty_dag(shape):
    """An empty-bodied DAG for scheduler throughput: the codelets' access
    modes, the number of buffers, the task count and a generator of
    (codelet, buffers) in submission order (the runtime derives the edges)."""
    R_, RW_ = 1, 3
    if shape == "chains":
        def gen():
            for _ in range(1000):
                for h in range(1000):
                    yield 0, (h,)
        return [[RW_]], 1000, 10 ** 6, gen
    if shape == "fan":
        def gen():
            for _ in range(1000):
                yield 0, (0,)
                for i in range(1, 1000):
                    yield 1, (0, i)
        return [[RW_], [R_, RW_]], 1000, 10 ** 6, gen
    T = 64

    def ix(i, j):
        return i * (i + 1) // 2 + j

    def gen():
        # POTRF(kk); TRSM(kk, ik); SYRK(ik, ii); GEMM(ik, jk, ij) in
        # right-looking order (Section 5.2's tiled factorisation)
        for k in range(T):
            yield 0, (ix(k, k),)
            for i in range(k + 1, T):
                yield 1, (ix(k, k), ix(i, k))
            for i in range(k + 1, T):
                yield 1, (ix(i, k), ix(i, i))
                for j in range(k + 1, i):
                    yield 2, (ix(i, k), ix(j, k), ix(i, j))
    return [[RW_], [R_, RW_], [R_, R_, RW_]], T * (T + 1) // 2, len_tasks(T), gen


def run_empty_dags(dev, stream):
    """Tasks/s of the persistent executor on the three empty-bodied DAGs
    (device time of one launch; the host's submission time apart)."""
    import torch
    import paper_1304_0878_b300 as b3t
    out = {}
    runs = [(shape, desc, 0) for shape, desc in EMPTY_DAGS]
    # the Cholesky shape again with one ready-queue level: FIFO order instead
    # of upward-rank priorities (Section 5.3's hint)
    runs.append(("cholesky", EMPTY_DAGS[2][1] + ", one ready-queue level (FIFO)", 1))
    for shape, desc, levels in runs:
        modes, nh, nt, gen = empty_dag(shape)
        ctx = b3t.Context(stream=stream.cuda_stream, timeout_ns=60_000_000_000, prio_levels=levels)
        buf = torch.zeros(nh * 16, device=dev)
        hs = [ctx.data_register(buf[i * 16:(i + 1) * 16].data_ptr(), 16, 4) for i in range(nh)]
        cls = [ctx.task_decl("empty", b3t.NOOP, m) for m in modes]
        t0 = time.perf_counter()
        ctx.graph_capture_begin()
        for c, bs in gen():
            ctx.task_submit(cls[c], [hs[h] for h in bs])
        ntasks, nedges = ctx.dag_stats()
        g = ctx.graph_capture_end()
        host_s = time.perf_counter() - t0
        ts = []
        for r in range(7):
            ctx.graph_replay(g)
            ctx.task_wait()
            if r >= 2:
                ts.append(ctx.last_launch()["kernel_ns"] / 1e9)
        med = float(np.median(ts))
        out[shape + ("_fifo" if levels == 1 else "")] = {
                      "workload": desc, "tasks": ntasks, "edges": nedges, "ms": 1e3 * med,
                      "tasks_per_s": ntasks / med, "host_submit_s": host_s,
                      "host_submit_tasks_per_s": ntasks / host_s}
        ctx.graph_destroy(g)
        ctx.close()
        del buf
    return out


def oracle_empty_dags(seconds):
    """The oracle executor (each task run at submission, empty bodies) on a
    bounded prefix of each empty-bodied DAG, one core: tasks/s."""
    from oracle import executor as oex
    out = {}
    for shape, _ in EMPTY_DAGS:
        modes, nh, nt, gen = empty_dag(shape)
        ex = oex.Executor()
        hs = [ex.data_register(np.zeros(16, np.float32)) for _ in range(nh)]
        cls = [ex.task_decl("empty", oex.noop_body, m) for m in modes]
        n = 0
        t0 = time.perf_counter()
        for c, bs in gen():
            ex.task_submit(cls[c], [hs[h] for h in bs])
            n += 1
            if (n & 1023) == 0 and time.perf_counter() - t0 > seconds:
                break
        sec = time.perf_counter() - t0
        out[shape] = {"tasks_per_s": n / sec, "cores": 1, "kind": "oracle",
                      "sample": "first %d of %d tasks in %.2f s" % (n, nt, sec)}
    return out


def scipy_serving_sample(seconds, n_max=96):
    """Library CPU baseline of the serving workload: the first requests of
    the seed-5 stream solved one at a time on the host (scipy Cholesky
    factor and solve, all host cores), until `seconds` of solve time.  Each
    A is a diagonally dominant symmetric matrix of the request's size (the
    factorisation's cost does not depend on the values); building it is not
    timed."""
    import scipy.linalg as sla
    import synth
    _, Ns, nrhs, seeds = synth.serve_requests(n_max, rate=2000.0, seed=5)
    lat, total, done = [], 0.0, 0
    for N, r, sd in zip(Ns, nrhs, seeds):
        rng = np.random.default_rng(sd % (2 ** 62))
        A = rng.random((int(N), int(N)))
        A += A.T
        A[np.diag_indices(int(N))] += 2.0 * N
        Bm = rng.standard_normal((int(N), int(r)))
        t0 = time.perf_counter()
        c = sla.cho_factor(A, lower=True, check_finite=False)
        sla.cho_solve(c, Bm, check_finite=False)
        dt = time.perf_counter() - t0
        lat.append(dt)
        total += dt
        done += 1
        if total > seconds:
            break
    return {"solves_per_s": done / total, "p50_solve_ms": 1e3 * float(np.median(lat)),
            "cores": len(os.sched_getaffinity(0)), "kind": "scipy (LAPACK) on the host, one request at a time",
            "sample": "first %d of the %d served requests, %.1f s of factor + solve time" % (done, n_max, total)}


SWEEP_RATES = {"fp64": (10.0, 20.0, 40.0, 80.0, 160.0, 2000.0), "bf16": (20.0, 40.0, 80.0, 160.0, 320.0, 2000.0)}


def run_serve_sweep(dev, args):
    """Continuous batching at a range of offered rates (the same requests:
    the generator draws arrival gaps as unit exponentials over the rate, so
    sizes and seeds do not depend on it).  The largest sustainable rate is
    the highest offered rate whose p99 latency stays within twice the p99 at
    the lowest rate of the sweep (the queue does not build up)."""
    import torch
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import serve as sv
    n = min(args.serve_requests, 500) if args.serve_requests == 2000 else args.serve_requests
    out = {"workload": "first %d requests of the seed-5 stream, N log-uniform [256, 8192], 1-32 rhs, "
                       "at each offered rate; client inputs of the first %d requests cycled, uploads and "
                       "downloads inside the latency" % (n, args.serve_distinct)}
    for prec, rates in SWEEP_RATES.items():
        rows = []
        pool = {}
        for rate in rates:
            sstream = torch.cuda.Stream(device=dev)
            ctx = b3t.Context(stream=sstream.cuda_stream, timeout_ns=60_000_000_000, stream_no_mx=prec == "fp64")
            reqs = sv.make_requests(n, rate, 5, prec=prec, distinct=args.serve_distinct)
            sv.prepare(reqs, pool=pool)
            st = sv.serve(ctx, reqs, prec=prec, budget_bytes=64 << 30, max_inflight=48, time_limit=600.0)
            ctx.close()
            rows.append({"offered_per_s": rate, "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"],
                         "p99_ms": st["p99_ms"], "failed": st["failed"], "max_eta": st["max_eta"]})
            del reqs
            torch.cuda.empty_cache()
        slo = 2.0 * rows[0]["p99_ms"]
        ok = [r["offered_per_s"] for r in rows if r["p99_ms"] <= slo and r["failed"] == 0]
        out[prec] = {"rates": rows, "p99_bound_ms": slo, "max_sustainable_rate_per_s": max(ok) if ok else None}
    return out


def run_secondary(ctx, dev, stream):
    """Vector chains (config 2), tasks/s on empty-bodied DAGs, small Cholesky."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    out = {}
    # vector-scaling chains: n = 2^28 f32, 256 blocks x 8 tasks, under both
    # ready-queue orders (upward rank = breadth first here; depth = each
    # chain's next task first, its block still in L2)
    nb, nk, n = 256, 8, 1 << 20
    x = torch.from_numpy(synth.vector_f32(nb * n, seed=1)).to(dev)
    f = synth.chain_factors(nb, nk, seed=2)
    tbytes = 8.0 * nb * nk * n
    # item chains: a block's 8 tasks run item by item on one CTA (one load,
    # 8 multiplies, one store per chunk): the floor is 2 GiB of HBM traffic
    floor_bytes = 8.0 * nb * n
    for name, pol, chained in (("vector_chains", b3t.PRIO_UPWARD, False),
                               ("vector_chains_depth_first", b3t.PRIO_DEPTH, False),
                               ("vector_chains_item_chains", b3t.PRIO_UPWARD, True)):
        c2 = b3t.Context(stream=stream.cuda_stream, timeout_ns=60_000_000_000, prio_policy=pol,
                         item_chains=chained)
        hs = [c2.data_register(x[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
        cl = c2.task_decl("scale_vector", b3t.SCAL_F32, [b3t.RW], 4)
        c2.graph_capture_begin()
        for k in range(nk):
            for i in range(nb):
                c2.task_submit(cl, [hs[i]], b3t.pack_f32(float(f[i, k])))
        g = c2.graph_capture_end()
        ts = []
        for r in range(8):
            c2.graph_replay(g)
            c2.task_wait()
            if r >= 3:
                ts.append(c2.last_launch()["kernel_ns"] / 1e9)
        med = float(np.median(ts))
        out[name] = {"workload": "n=2^28 f32, 256 blocks x 8 chained RW tasks (2048 tasks)",
                     "ms": 1e3 * med, "task_level_GBps": tbytes / med / 1e9, "task_bytes": tbytes,
                     "hbm_frac": tbytes / med / 1e9 / hbm_peak()[0], "hbm_peak_GBps": hbm_peak()[0],
                     "hbm_peak_source": hbm_peak()[1]}
        if chained:
            # each element read and written once: the HBM floor of the DAG
            out[name].update({"execution": "item chains (each block's 8 tasks item by item on one CTA)",
                              "floor_bytes": floor_bytes,
                              "floor_ms": 1e3 * floor_bytes / (hbm_peak()[0] * 1e9),
                              "hbm_frac": floor_bytes / med / 1e9 / hbm_peak()[0]})
        c2.graph_destroy(g)
        c2.close()
    del x
    # scheduler throughput: 1000 chains x 100 empty tasks
    y = torch.zeros(1000 * 64, device=dev)
    hy = [ctx.data_register(y[i * 64:(i + 1) * 64].data_ptr(), 64, 4) for i in range(1000)]
    cn = ctx.task_decl("noop", b3t.NOOP, [b3t.RW])
    ctx.graph_capture_begin()
    for k in range(100):
        for h in hy:
            ctx.task_submit(cn, [h])
    g = ctx.graph_capture_end()
    ts = []
    for r in range(6):
        ctx.graph_replay(g)
        ctx.task_wait()
        if r >= 2:
            ts.append(ctx.last_launch()["kernel_ns"] / 1e9)
    out["tasks_per_s"] = {"workload": "1000 chains x 100 empty tasks (100k tasks)",
                          "value": 1e5 / float(np.median(ts))}
    ctx.graph_destroy(g)
    for h in hy:
        ctx.data_unregister(h)
    del y
    out["empty_dags"] = run_empty_dags(dev, stream)
    # small Cholesky, N = 1024, tile 128 (config 1): latency of one launch,
    # with upward-rank priorities and with one level (FIFO)
    N1, b1 = 1024, 128
    A1 = dt.to_tiles(torch.from_numpy(synth.spd_host(N1, seed=0, shift=1.0)).to(dev), b1)
    t1 = torch.empty_like(A1)
    p1 = dt.tile_ptrs(t1)
    for name, levels in (("cholesky_small", 0), ("cholesky_small_fifo", 1)):
        c1 = b3t.Context(stream=stream.cuda_stream, timeout_ns=60_000_000_000, prio_levels=levels)
        c1.graph_capture_begin()
        c1.cholesky_submit(p1, N1 // b1, b1)
        ntasks = c1.dag_stats()[0]
        g = c1.graph_capture_end()
        ts = []
        for r in range(13):
            t1.copy_(A1)
            c1.graph_replay(g)
            c1.task_wait()
            if r >= 3:
                ts.append(c1.last_launch()["kernel_ns"] / 1e9)
        med = float(np.median(ts))
        out[name] = {"workload": "FP64 N=1024 tile 128 (120 tile tasks, %d device tasks)%s"
                                 % (ntasks, ", one ready-queue level (FIFO)" if levels == 1 else ""),
                     "ms": 1e3 * med, "TFLOPs": cholesky_flops(N1) / med / 1e12,
                     "tasks_per_s": ntasks / med}
        c1.graph_destroy(g)
        c1.tiles_unregister(p1, N1 // b1)
        c1.close()
    return out


def run_case(args):
    """Single-kind DAGs sized for a short profiler capture (inputs > L2)."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    import paper_1304_0878_b300.build as pb
    pb.build()
    dev = torch.device("cuda", 0)
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=60_000_000_000,
                      ctas_per_sm=args.ctas_per_sm,
                      prio_policy=prio_of(args),
                      item_chains=args.item_chains)
    b = 512
    if args.case.startswith("mx_gemm"):
        # 64 independent GEMM_MX updates W_i -= Q_a Q_b^T (b = 512): 64 x 2 b^3 flop
        fmt = b3t.FMT_BF16 if args.case.endswith("bf16") else b3t.FMT_E4M3
        nW = 64
        L = torch.randn((8, b, b), dtype=torch.float64, device=dev) * 0.1
        Q = torch.empty((8, b3t.q_bytes(b, fmt)), dtype=torch.uint8, device=dev)
        W = torch.randn((nW, b, b), dtype=torch.float32, device=dev)
        hl = [ctx.data_register(p, b * b, 8, b) for p in dt.tile_ptrs(L)]
        hq = [ctx.data_register(p, Q.shape[1], 1, b) for p in dt.tile_ptrs(Q)]
        hw = [ctx.data_register(p, b * b, 4, b) for p in dt.tile_ptrs(W)]
        cq = ctx.task_decl("quant", b3t.QUANT, [1, 2], 4)
        for i in range(8):
            ctx.task_submit(cq, [hl[i], hq[i]], b3t.pack_i32(fmt))
        ctx.task_wait()
        cg = ctx.task_decl("gemm_mx", b3t.GEMM_MX, [1, 1, 3], 4)
        ctx.graph_capture_begin()
        for i in range(nW):
            ctx.task_submit(cg, [hq[i % 8], hq[(i * 3 + 1) % 8], hw[i]], b3t.pack_i32(fmt))
        g = ctx.graph_capture_end()
        work, unit = nW * 2.0 * b ** 3, "TFLOP/s"
    elif args.case == "scal":
        n, nb, nk = 1 << 20, 256, 8
        x = torch.from_numpy(synth.vector_f32(nb * n, seed=1)).to(dev)
        hs = [ctx.data_register(x[i * n:(i + 1) * n].data_ptr(), n, 4) for i in range(nb)]
        cl = ctx.task_decl("scale_vector", b3t.SCAL_F32, [3], 4)
        ctx.graph_capture_begin()
        for k in range(nk):
            for h in hs:
                ctx.task_submit(cl, [h], b3t.pack_f32(1.0000001))
        g = ctx.graph_capture_end()
        work, unit = 8.0 * n * nb * nk, "GB/s"
    elif args.case.startswith("solve"):
        # forward + backward solve with a tiled factor and its inverted
        # diagonal tiles (the refinement's solve), N = 16384, 16 rhs
        N, nrhs = 16384, 16
        T = N // b
        L = synth.spd_tiles_device(N, b, 3, 0.1, dev)
        ctx.graph_capture_begin()
        ctx.cholesky_submit(dt.tile_ptrs(L), T, b)
        gl = ctx.graph_capture_end()
        ctx.graph_replay(gl)
        ctx.task_wait()
        ctx.graph_destroy(gl)
        Y = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
        Z = torch.zeros_like(Y)
        U = torch.empty((T, b, b), dtype=torch.float64, device=dev)
        ctx.chol_inv_submit(dt.tile_ptrs(L), dt.tile_ptrs(U), T, b)     # once per factor, not timed
        ctx.task_wait()
        flags = b3t.VEC_F32 if args.case.endswith("f32") else 0
        ctx.graph_capture_begin()
        ctx.chol_solve_inv_submit(dt.tile_ptrs(L), dt.tile_ptrs(U), Y.data_ptr(), Z.data_ptr(), T, b, nrhs,
                                  b * nrhs, flags)
        g = ctx.graph_capture_end()
        work, unit = 2.0 * N * N * nrhs, "TFLOP/s"
    elif args.case == "resid_sl":
        return run_resid_sliced(ctx, dev, args)
    elif args.case == "trmm_sl":
        return run_trmm_sliced(ctx, dev, args)
    else:  # resid: one refinement residual over N = 16384, 16 rhs (FP64)
        N, nrhs = 16384, 16
        T = N // b
        A = synth.spd_tiles_device(N, b, 3, 0.1, dev)
        X = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
        B = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
        PR = b3t.resid_part_elems(b, nrhs)             # residual part: values, then per-item maxima
        R = torch.zeros(T * PR, dtype=torch.float64, device=dev)
        ha = ctx.data_register(A.data_ptr(), A.numel(), 8)
        hx = ctx.data_register(X.data_ptr(), X.numel(), 8)
        hb = ctx.data_register(B.data_ptr(), B.numel(), 8)
        hr = ctx.data_register(R.data_ptr(), R.numel(), 8)
        pr = ctx.data_partition(hr, T, PR)
        cr = ctx.task_decl("resid", b3t.RESID, [1, 1, 1, 2], 20)
        ctx.graph_capture_begin()
        for i in range(T):
            ctx.task_submit(cr, [ha, hx, hb, pr[i]], b3t.vec_args(nrhs, 0, i, T, b))
        g = ctx.graph_capture_end()
        work, unit = 2.0 * N * N * nrhs, "TFLOP/s"
    ts = []
    for r in range(args.warmup + args.steps):
        ctx.graph_replay(g)
        ctx.task_wait()
        if r >= args.warmup:
            ts.append(ctx.last_launch()["kernel_ns"] / 1e9)
    med = float(np.median(ts))
    scale = 1e12 if unit == "TFLOP/s" else 1e9
    print(json.dumps({"case": args.case, "kernel_ms": med * 1e3, "value": work / med / scale, "unit": unit,
                      "nctas": ctx.last_launch()["nctas"], "prio": args.prio}))
    ctx.graph_destroy(g)
    ctx.close()


def run_resid_sliced(ctx, dev, args):
    """The refinement residual at N = 32768, tile 512, 16 rhs: the sliced
    FP64 residual (SLICE_X + RESID_SL, one launch per step; SLICE_A once per
    solve) against the FP64 RESID on the same inputs.  Kernel times of the
    persistent launches (CUDA events), inputs larger than L2."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    N, b, nrhs = (args.n if args.n != 32768 else 32768), 512, 16
    T = N // b
    A = synth.spd_tiles_device(N, b, 3, 0.1, dev)
    X = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
    B = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
    PR = b3t.resid_part_elems(b, nrhs)
    PB, XB = b3t.slice_a_part_bytes(b), b3t.slice_x_part_bytes(b)
    R = torch.zeros(T * PR, dtype=torch.float64, device=dev)
    AS = torch.empty(T * T * PB, dtype=torch.uint8, device=dev)
    XS = torch.empty(T * XB, dtype=torch.uint8, device=dev)
    ha = ctx.data_register(A.data_ptr(), A.numel(), 8)
    hx = ctx.data_register(X.data_ptr(), X.numel(), 8)
    px = ctx.data_partition(hx, T, b * nrhs)
    hb = ctx.data_register(B.data_ptr(), B.numel(), 8)
    hr = ctx.data_register(R.data_ptr(), R.numel(), 8)
    pr = ctx.data_partition(hr, T, PR)
    has = ctx.data_register(AS.data_ptr(), AS.numel(), 1)
    pas = ctx.data_partition(has, T * T, PB)
    hxs = ctx.data_register(XS.data_ptr(), XS.numel(), 1)
    pxs = ctx.data_partition(hxs, T, XB)
    ca = ctx.task_decl("slice_a", b3t.SLICE_A, [1, 2, 2], 20)
    cx = ctx.task_decl("slice_x", b3t.SLICE_X, [1, 2], 20)
    cs = ctx.task_decl("resid_sl", b3t.RESID_SL, [1, 1, 1, 2], 20)
    cr = ctx.task_decl("resid", b3t.RESID, [1, 1, 1, 2], 20)
    graphs = {}
    ctx.graph_capture_begin()
    for j in range(T):
        for i in range(j, T):
            ctx.task_submit(ca, [ha, pas[i * T + j], pas[j * T + i]], b3t.slice_args(i, j, T, b, 0))
    graphs["slice_a"] = ctx.graph_capture_end()
    ctx.graph_capture_begin()
    for J in range(T):
        ctx.task_submit(cx, [px[J], pxs[J]], b3t.slice_args(J, 0, T, b, nrhs))
    for i in range(T):
        ctx.task_submit(cs, [has, hxs, hb, pr[i]], b3t.slice_args(i, 0, T, b, nrhs))
    graphs["sliced_step"] = ctx.graph_capture_end()
    ctx.graph_capture_begin()
    for i in range(T):
        ctx.task_submit(cr, [ha, hx, hb, pr[i]], b3t.vec_args(nrhs, 0, i, T, b))
    graphs["fp64_resid"] = ctx.graph_capture_end()
    ms = {}
    for name in ("slice_a", "sliced_step", "fp64_resid"):
        ts = []
        for r in range(args.warmup + args.steps):
            ctx.graph_replay(graphs[name])
            ctx.task_wait()
            if r >= args.warmup:
                ts.append(ctx.last_launch()["kernel_ns"] / 1e6)
        ms[name] = float(np.median(ts))
        ctx.graph_destroy(graphs[name])
    flops = 2.0 * N * N * nrhs
    slice_bytes = T * T * (PB - 8 * b - 16)
    hbm, src = hbm_peak()
    out = {"case": "resid_sl", "workload": "r = b - A x, N=%d tile %d, %d rhs" % (N, b, nrhs),
           "fp64_resid_ms": ms["fp64_resid"], "fp64_resid_TFLOPs": flops / ms["fp64_resid"] / 1e9,
           "sliced_step_ms": ms["sliced_step"], "sliced_effective_TFLOPs": flops / ms["sliced_step"] / 1e9,
           "slice_a_ms": ms["slice_a"], "speedup_per_step": ms["fp64_resid"] / ms["sliced_step"],
           "slice_bytes_per_step": slice_bytes,
           "roofline": {"bound": "hbm", "achieved": slice_bytes / ms["sliced_step"] / 1e6, "peak": hbm,
                        "unit": "GB/s", "frac": slice_bytes / ms["sliced_step"] / 1e6 / hbm, "peak_source": src},
           "nctas": ctx.last_launch()["nctas"]}
    print(json.dumps(out))
    ctx.close()


def run_trmm_sliced(ctx, dev, args):
    """64 panel products L_i = fp64(W_i) U (b = 512) in one launch: TRMM_SL
    from slices (SLICE_W / SLICE_U once, untimed) against TRMM_MX (FP64
    DFMA) on the same inputs.  Work: b^3 FP64-equivalent flop per product
    (U triangular); the tensor-core flops of the kept slice pairs for the
    roofline (E4M3 peak = the measured bf16 peak x 2)."""
    import torch
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    b, n = 512, 64
    U = torch.triu(torch.randn((b, b), dtype=torch.float64, device=dev)).T.contiguous()   # tile: upper
    W = torch.randn((n, b, b), dtype=torch.float32, device=dev)
    L = torch.zeros((n, b, b), dtype=torch.float64, device=dev)
    WS = torch.empty((n, b3t.slice_w_bytes(b)), dtype=torch.uint8, device=dev)
    US = torch.empty(b3t.slice_u_bytes(b), dtype=torch.uint8, device=dev)
    hu = ctx.data_register(U.data_ptr(), b * b, 8, b)
    hus = ctx.data_register(US.data_ptr(), US.numel(), 1)
    hw = [ctx.data_register(p, b * b, 4, b) for p in dt.tile_ptrs(W)]
    hl = [ctx.data_register(p, b * b, 8, b) for p in dt.tile_ptrs(L)]
    hws = [ctx.data_register(p, WS.shape[1], 1) for p in dt.tile_ptrs(WS)]
    cu = ctx.task_decl("slice_u", b3t.SLICE_U, [1, 2])
    cw = ctx.task_decl("slice_w", b3t.SLICE_W, [1, 2])
    cm = ctx.task_decl("trmm_sl", b3t.TRMM_SL, [1, 1, 2])
    cf = ctx.task_decl("trmm_mx", b3t.TRMM_MX, [1, 1, 2])
    ctx.task_submit(cu, [hu, hus])
    for i in range(n):
        ctx.task_submit(cw, [hw[i], hws[i]])
    ctx.task_wait()
    graphs = {}
    ctx.graph_capture_begin()
    for i in range(n):
        ctx.task_submit(cm, [hus, hws[i], hl[i]])
    graphs["trmm_sl"] = ctx.graph_capture_end()
    ctx.graph_capture_begin()
    for i in range(n):
        ctx.task_submit(cf, [hu, hw[i], hl[i]])
    graphs["trmm_mx"] = ctx.graph_capture_end()
    ms = {}
    for name, g in graphs.items():
        ts = []
        for r in range(args.warmup + args.steps):
            ctx.graph_replay(g)
            ctx.task_wait()
            if r >= args.warmup:
                ts.append(ctx.last_launch()["kernel_ns"] / 1e6)
        ms[name] = float(np.median(ts))
        ctx.graph_destroy(g)
    fp64_flops = n * float(b) ** 3
    # tensor work: per 128 x 32 block, K = 32 (cb + 1), 78 kept pairs of E4M3 products
    kc = sum(32 * (cb + 1) for cb in range(b // 32)) * (b // 128)
    tensor_flops = n * 78 * 2.0 * 128 * 32 * kc
    peak = 2.0 * bf16_peak()[0]
    out = {"case": "trmm_sl", "workload": "%d panel products L = fp64(W) U, b = %d, U upper triangular" % (n, b),
           "trmm_sl_ms": ms["trmm_sl"], "trmm_mx_fp64_ms": ms["trmm_mx"], "speedup": ms["trmm_mx"] / ms["trmm_sl"],
           "fp64_equivalent_TFLOPs": fp64_flops / ms["trmm_sl"] / 1e9,
           "fp64_dfma_TFLOPs": fp64_flops / ms["trmm_mx"] / 1e9,
           "roofline": {"bound": "tensor", "achieved": tensor_flops / ms["trmm_sl"] / 1e9, "peak": peak,
                        "unit": "TFLOP/s", "frac": tensor_flops / ms["trmm_sl"] / 1e9 / peak,
                        "peak_source": "measured bf16 burst x 2 (E4M3)"}}
    print(json.dumps(out))
    ctx.close()


def run_trace_headline(dev, args):
    """One traced factorisation of the headline workload: how busy the CTAs
    were, each task kind's share of the CTA time, and the longest chain of
    task spans (first item's start to last item's end) through the DAG, its
    critical path, against the launch's makespan."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    N, b = args.n, args.b
    T = N // b
    ctx = b3t.Context(stream=torch.cuda.current_stream(dev).cuda_stream, timeout_ns=120_000_000_000,
                      prio_policy=prio_of(args))
    t = synth.spd_tiles_device(N, b, 3, 0.1, dev)
    ctx.trace_start(1 << 22)
    ctx.cholesky_submit(dt.tile_ptrs(t), T, b)
    ntasks, nedges = ctx.dag_stats()
    ed = np.array(ctx.dag_edges(), dtype=np.int64).reshape(-1, 2)
    ctx.task_wait()
    tr = ctx.trace_read()
    ctx.trace_stop()
    ll = ctx.last_launch()
    ctx.close()
    assert len(tr) == ll["nitems"], "trace buffer too small"
    out = {"workload": "FP64 Cholesky N=%d tile %d, one traced launch" % (N, b), "tasks": ntasks,
           "edges": nedges, "items": int(len(tr)), "ctas": ll["nctas"], "traced_kernel_ms": ll["kernel_ns"] / 1e6}
    from paper_1304_0878_b300 import trace
    out.update(trace.summary(tr, ntasks, ed, ll["nctas"]))
    return out


def run_trace_mixed(dev, args):
    """One traced mixed-precision factorisation (bf16 updates, FP64 panel),
    N = --n, tile --b, the panel solve by --mx-trsm: CTA busy fraction, the
    per-kind share of CTA time and the critical path."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt
    N, b = args.n, args.b
    T = N // b
    ctx = b3t.Context(stream=torch.cuda.current_stream(dev).cuda_stream, timeout_ns=120_000_000_000,
                      prio_policy=prio_of(args))
    A0 = synth.spd_tiles_device(N, b, 3, 0.1, dev)
    W = A0.float()
    del A0
    Lm = torch.zeros(W.shape, dtype=torch.float64, device=dev)
    Q = dt.q_tiles(T, b, b3t.FMT_BF16, dev)
    U = torch.zeros((T, b, b), dtype=torch.float64, device=dev)
    mode = mx_modes(args)[0]
    if mode == "sliced":
        WS = torch.zeros((T * (T + 1) // 2, b3t.slice_w_bytes(b)), dtype=torch.uint8, device=dev)
        US = torch.zeros((T, b3t.slice_u_bytes(b)), dtype=torch.uint8, device=dev)
    ctx.trace_start(1 << 23)
    if mode == "subst":
        ctx.cholesky_mx_submit(dt.tile_ptrs(W), dt.tile_ptrs(Lm), dt.tile_ptrs(Q), T, b, b3t.FMT_BF16)
    elif mode == "sliced":
        ctx.cholesky_mx_sliced_submit(dt.tile_ptrs(W), dt.tile_ptrs(Lm), dt.tile_ptrs(Q), dt.tile_ptrs(U),
                                      dt.tile_ptrs(WS), dt.tile_ptrs(US), T, b, b3t.FMT_BF16)
    else:
        ctx.cholesky_mx_inv_submit(dt.tile_ptrs(W), dt.tile_ptrs(Lm), dt.tile_ptrs(Q), dt.tile_ptrs(U), T, b,
                                   b3t.FMT_BF16)
    ntasks, nedges = ctx.dag_stats()
    ed = np.array(ctx.dag_edges(), dtype=np.int64).reshape(-1, 2)
    ctx.task_wait()
    tr = ctx.trace_read()
    ctx.trace_stop()
    ll = ctx.last_launch()
    ctx.close()
    assert len(tr) == ll["nitems"], "trace buffer too small"
    out = {"workload": "mixed bf16 Cholesky N=%d tile %d (%s), one traced launch" % (N, b, mode),
           "tasks": ntasks, "edges": nedges, "items": int(len(tr)), "ctas": ll["nctas"],
           "traced_kernel_ms": ll["kernel_ns"] / 1e6}
    from paper_1304_0878_b300 import trace
    out.update(trace.summary(tr, ntasks, ed, ll["nctas"]))
    # busy fraction over time: tenths of the makespan
    st = tr["t_start_ns"].astype(np.int64)
    en = tr["t_end_ns"].astype(np.int64)
    t0, t1 = int(st.min()), int(en.max())
    edges_t = np.linspace(t0, t1, 11)
    busy = []
    for i in range(10):
        lo, hi = edges_t[i], edges_t[i + 1]
        ov = np.clip(np.minimum(en, hi) - np.maximum(st, lo), 0, None)
        busy.append(round(float(ov.sum()) / (ll["nctas"] * (hi - lo)), 3))
    out["busy_by_tenth"] = busy
    return out


def run_batch(dev, args):
    """Batching: 24 uneven FP64 factorisations (N log-uniform in [256, 4096],
    the serving stream's sizes, seed 5; tiles from the tuner, ragged sizes
    padded with identity) in ONE persistent launch, against one launch per
    matrix.  Each way is timed end to end (padding into tiles included) on
    the device with CUDA events, after one untimed pass."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import batch as bt
    _, Ns, _, seeds = synth.serve_requests(24, rate=2000.0, seed=5, nmin=256, nmax=4096)
    mats = []
    for N, sd in zip(Ns, seeds):
        g = torch.Generator(device=dev)
        g.manual_seed(int(sd % (2 ** 62)))
        Bm = torch.randn((int(N), int(N)), generator=g, device=dev, dtype=torch.float64)
        mats.append(Bm @ Bm.T / int(N) + torch.eye(int(N), dtype=torch.float64, device=dev))
    del Bm
    stream = torch.cuda.current_stream(dev)
    ctx = b3t.Context(stream=stream.cuda_stream, timeout_ns=60_000_000_000)
    flops = float(sum(cholesky_flops(int(N)) for N in Ns))
    res = {}
    for name in ("one_launch", "launch_per_matrix"):
        ts = []
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            if name == "one_launch":
                bt.cholesky_many(ctx, mats)
            else:
                for A in mats:
                    bt.cholesky_many(ctx, [A])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        res[name] = {"ms": ts[-1], "TFLOPs": flops / (ts[-1] / 1e3) / 1e12}
    ctx.close()
    res["speedup"] = res["launch_per_matrix"]["ms"] / res["one_launch"]["ms"]
    res["sizes"] = [int(N) for N in Ns]
    return res


def run_trace_solve(dev, args):
    """The refinement's correction solve traced: forward and backward
    substitution in binary32 with the inverted diagonal tiles of a sliced bf16
    factor, N = --n, tile --b, 16 right-hand sides (two untraced runs, then one
    traced): the critical path through the 2T dependent GEMV steps and the
    time its tasks waited for a CTA."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from paper_1304_0878_b300 import tiles as dt, trace
    N, b, nrhs = args.n, args.b, 16
    T = N // b
    ctx = b3t.Context(stream=torch.cuda.current_stream(dev).cuda_stream, timeout_ns=120_000_000_000,
                      prio_policy=prio_of(args))
    A0 = synth.spd_tiles_device(N, b, 3, 0.1, dev)
    W = A0.float()
    del A0
    L = torch.zeros(W.shape, dtype=torch.float64, device=dev)
    Q = dt.q_tiles(T, b, b3t.FMT_BF16, dev)
    U = torch.zeros((T, b, b), dtype=torch.float64, device=dev)
    WS = torch.zeros((T * (T + 1) // 2, b3t.slice_w_bytes(b)), dtype=torch.uint8, device=dev)
    US = torch.zeros((T, b3t.slice_u_bytes(b)), dtype=torch.uint8, device=dev)
    ctx.cholesky_mx_sliced_submit(dt.tile_ptrs(W), dt.tile_ptrs(L), dt.tile_ptrs(Q), dt.tile_ptrs(U),
                                  dt.tile_ptrs(WS), dt.tile_ptrs(US), T, b, b3t.FMT_BF16)
    ctx.task_wait()
    del W, WS, US, Q
    Y = torch.randn((T, nrhs, b), dtype=torch.float64, device=dev)
    Z = torch.zeros_like(Y)
    out = {"workload": "binary32 forward + backward solve, N=%d tile %d, %d rhs, inverted diagonal tiles"
                       % (N, b, nrhs)}
    kms = []
    for rep in range(3):
        if rep == 2:
            ctx.trace_start(1 << 20)
        ctx.chol_solve_inv_submit(dt.tile_ptrs(L), dt.tile_ptrs(U), Y.data_ptr(), Z.data_ptr(), T, b, nrhs,
                                  b * nrhs, b3t.VEC_F32)
        ntasks, nedges = ctx.dag_stats()
        ed = np.array(ctx.dag_edges(), dtype=np.int64).reshape(-1, 2)
        ctx.task_wait()
        kms.append(ctx.last_launch()["kernel_ns"] / 1e6)
    tr = ctx.trace_read()
    ctx.trace_stop()
    ll = ctx.last_launch()
    ctx.close()
    out.update({"tasks": ntasks, "edges": nedges, "kernel_ms_untraced": kms[:2], "traced_kernel_ms": kms[2]})
    out.update(trace.summary(tr, ntasks, ed, ll["nctas"]))
    return out


def run_part(args):
    """One secondary measurement alone, printed as one JSON line."""
    import torch
    import paper_1304_0878_b300.build as pb
    pb.build()
    dev = torch.device("cuda", 0)
    if args.case == "empty_dags":
        res = run_empty_dags(dev, torch.cuda.current_stream(dev))
    elif args.case == "trace_headline":
        res = run_trace_headline(dev, args)
    elif args.case == "trace_mixed":
        res = run_trace_mixed(dev, args)
    elif args.case == "batch":
        res = run_batch(dev, args)
    elif args.case == "trace_solve":
        res = run_trace_solve(dev, args)
    else:
        res = run_serve_sweep(dev, args)
    print(json.dumps({"case": args.case, "result": res}))


if __name__ == "__main__":
    a = parse()
    if a.case in ("empty_dags", "serve_sweep", "trace_headline", "trace_mixed", "batch", "trace_solve"):
        run_part(a)
    elif a.case:
        run_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
