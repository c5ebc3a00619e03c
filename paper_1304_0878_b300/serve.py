"""Serving loop: Cholesky-solve requests with continuous batching.

Requests (N x N SPD matrix, nrhs right-hand sides) arrive as a Poisson
process.  The loop admits them in arrival order while their device
footprint fits an HBM budget and a slot is free, generates each request's
matrix on the device (a side stream), and hands its work to ONE resident
executor (stream mode): every request stage is a task graph submitted while
the others run, so requests that arrive while others are on the GPU join
them as slots and memory free up, and their tasks share the SMs.

Stages per request:
  * fp64: factorisation + one solve step (x = (L L^T)^{-1} b, residual, eta);
  * bf16 / e4m3: mixed-precision factorisation + first refinement step, then
    one refinement step per stage until eta <= tol (FP64 residual).
Factors stay on the device until the request completes.  Latency is
measured from arrival to the completion of the last stage.

`serve_plain` is the per-request path for comparison: one request at a time,
one launch per stage, no overlap.

Request inputs (the matrix and right-hand sides, as a client would send
them) are built on the device before serving starts (`prepare`, timed
separately): that step uses library GEMMs, which may be persistent kernels
that need the whole GPU and so cannot run next to the resident executor.
Admission then only allocates the working buffers and copies into them.
"""
import math
import time

import numpy as np
import torch

from . import tiles as dt
from . import tune
from . import _lib

U64 = 8


def footprint(Np, nrhs, b, prec):
    """Device bytes of one request (packed lower tiles + vectors)."""
    T = Np // b
    tile = T * (T + 1) // 2 * b * b
    vec = T * b * nrhs * 8
    work = _lib.ir_work_elems(T, b, nrhs) * 8             # residual parts, scratch, inverted tiles
    if prec == "fp64":
        mats = tile * 16                                   # A + factor
    else:
        mats = tile * (8 + 4 + 8 + (2 if prec == "bf16" else 1))   # A, W, L, Q
    return mats + 2 * vec + work + 4096


class Request:
    __slots__ = ("rid", "arrival", "N", "nrhs", "seed", "b", "Np", "T", "state", "bufs", "ptrs",
                 "batch", "gen_ev", "t_admit", "t_ready", "t_done", "iters", "eta", "info", "bytes", "x",
                 "inputs")

    def __init__(self, rid, arrival, N, nrhs, seed):
        self.rid, self.arrival, self.N, self.nrhs, self.seed = rid, arrival, int(N), int(nrhs), int(seed)
        self.state = "queued"
        self.iters = 0
        self.eta = float("nan")
        self.info = 0
        self.batch = -1


def make_inputs(req, device, stream):
    """Request inputs on the device: A = B B^T / N + I with B ~ N(0, 1)
    binary32 from torch's CUDA generator seeded with req.seed (binary32
    product, TF32 off), padded to diag(A, I), as packed lower FP64 tiles; the
    right-hand sides N(0, 1) as T parts of b x nrhs.  Built before serving
    starts: library GEMMs may be persistent kernels that need the whole GPU,
    so they must not run next to the resident executor."""
    N, b, Np, T, nrhs = req.N, req.b, req.Np, req.T, req.nrhs
    with torch.cuda.stream(stream):
        g = torch.Generator(device=device)
        g.manual_seed(req.seed)
        B = torch.randn((N, N), generator=g, device=device, dtype=torch.float32)
        C = torch.zeros((Np, Np), dtype=torch.float32, device=device)
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        C[:N, :N] = B @ B.T
        torch.backends.cuda.matmul.allow_tf32 = prev
        A = dt.pack_lower(C, b).double()
        A.div_(N)
        d = torch.arange(b, device=device)
        ii, jj = dt.packed_index(T, device)
        diag = (ii == jj).nonzero().flatten()
        A[diag[:, None], d[None, :], d[None, :]] += 1.0
        rv = torch.randn((nrhs, N), generator=g, device=device, dtype=torch.float64)
        flat = torch.zeros((nrhs, Np), dtype=torch.float64, device=device)
        flat[:, :N] = rv
        rhs = flat.view(nrhs, T, b).permute(1, 0, 2).contiguous()     # T parts of b x nrhs
        del B, C
    req.inputs = (A, rhs)


def generate(req, prec, device, stream):
    """Admission: the request's working buffers, filled from its inputs with
    elementwise copies on `stream` (safe next to the resident executor)."""
    import paper_1304_0878_b300 as b3t
    T, b, nrhs = req.T, req.b, req.nrhs
    A, rhs = req.inputs
    with torch.cuda.stream(stream):
        X = torch.zeros_like(rhs)
        R = torch.zeros(b3t.ir_work_elems(T, b, nrhs), dtype=torch.float64, device=device)
        eta = torch.zeros(nrhs + 1, dtype=torch.float64, device=device)
        bufs = {"A": A, "B": rhs, "X": X, "R": R, "eta": eta}
        if prec == "fp64":
            bufs["F"] = A.clone()
        else:
            fmt = b3t.FMT_BF16 if prec == "bf16" else b3t.FMT_E4M3
            bufs["W"] = A.float()
            bufs["L"] = torch.empty_like(A)
            bufs["Q"] = dt.q_tiles(T, b, fmt, device)
        ev = torch.cuda.Event()
        ev.record(stream)
    req.bufs = bufs
    req.gen_ev = ev
    req.ptrs = {k: dt.tile_ptrs(v) for k, v in bufs.items() if k in ("F", "W", "L", "Q")}


def prepare(reqs, device="cuda"):
    """Build every request's inputs (before serving); returns seconds."""
    t0 = time.perf_counter()
    s = torch.cuda.current_stream(device)
    for r in reqs:
        make_inputs(r, device, s)
    torch.cuda.synchronize(device)
    return time.perf_counter() - t0


def submit_stage(ctx, req, prec, first, tol):
    """Submit the request's next stage into the current batch (caller flushes
    or stream-submits)."""
    import paper_1304_0878_b300 as b3t
    bf = req.bufs
    T, b, nrhs = req.T, req.b, req.nrhs
    if prec == "fp64":
        ctx.cholesky_submit(req.ptrs["F"], T, b, 0)
        Lp = req.ptrs["F"]
        flags = 0
    else:
        fmt = b3t.FMT_BF16 if prec == "bf16" else b3t.FMT_E4M3
        if first:
            ctx.cholesky_mx_submit(req.ptrs["W"], req.ptrs["L"], req.ptrs["Q"], T, b, fmt, 0)
        Lp = req.ptrs["L"]
        flags = b3t.VEC_F32
    ctx.ir_step_submit(bf["A"].data_ptr(), Lp, bf["B"].data_ptr(), bf["X"].data_ptr(), bf["R"].data_ptr(),
                       bf["eta"].data_ptr(), T, b, nrhs, flags, first)


def release(ctx, req, keep_x=False, stream=None):
    """Forget the request's registrations (its batches are done); keep_x
    copies the solution (T parts of b x nrhs) to the host first."""
    if keep_x:
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            req.x = req.bufs["X"].to("cpu", non_blocking=False)
    for p in req.ptrs.values():
        ctx.tiles_unregister(p, req.T)
    ctx.ir_release(req.bufs["R"].data_ptr(), req.T, req.b, req.nrhs)
    for k in ("A", "B", "X", "eta"):
        try:
            h = ctx.data_lookup(req.bufs[k].data_ptr())
            ctx.data_unregister(h)
        except Exception:
            pass
    req.bufs = None
    req.ptrs = None
    req.inputs = None


def make_requests(n, rate, seed, nmin=256, nmax=8192, rmax=32, prec="fp64", tile=None):
    """n requests (Poisson arrivals at `rate` per second); the tile size is
    the tuner's choice for each N unless `tile` fixes it."""
    import synth
    arr, Ns, nrhs, seeds = synth.serve_requests(n, rate=rate, seed=seed, nmin=nmin, nmax=nmax, rmax=rmax)
    out = []
    for i in range(n):
        r = Request(i, float(arr[i]), Ns[i], nrhs[i], seeds[i] % (2 ** 62))
        r.b = tile or tune.choose_tile(r.N, prec)
        r.Np = dt.pad_size(r.N, r.b)
        r.T = r.Np // r.b
        r.bytes = footprint(r.Np, r.nrhs, r.b, prec)
        out.append(r)
    return out


def _stats(reqs, t_first, t_last, prec, mode):
    lat = np.array([r.t_done - r.arrival for r in reqs]) * 1e3
    qd = np.array([r.t_admit - r.arrival for r in reqs]) * 1e3
    ok = [r for r in reqs if r.info == 0]
    return {
        "mode": mode, "precision": prec, "requests": len(reqs),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "admission_wait_p50_ms": float(np.percentile(qd, 50)),
        "solves_per_s": len(reqs) / max(t_last - t_first, 1e-9),
        "max_eta": float(max(r.eta for r in ok)) if ok else None,
        "mean_iterations": float(np.mean([r.iters for r in reqs])),
        "failed": len(reqs) - len(ok),
        "flop_per_s": float(sum(r.N ** 3 / 3.0 for r in reqs) / max(t_last - t_first, 1e-9)),
    }


def warm_up(prec, device, gen_stream, side, host, reserve_bytes):
    """Initialise, before the resident kernel starts, everything that is set up
    lazily on first use and may synchronise the whole device: cuBLAS handles
    and workspaces of the generation stream, the random generator, and the
    caching allocator's pools (one large reservation, freed into torch's
    cache so that later allocations on that stream reuse it)."""
    r = Request(-1, 0.0, 300, 2, 1)
    r.b = tune.choose_tile(r.N, prec)
    r.Np = dt.pad_size(r.N, r.b)
    r.T = r.Np // r.b
    make_inputs(r, device, gen_stream)
    generate(r, prec, device, gen_stream)
    gen_stream.synchronize()
    with torch.cuda.stream(side):
        host[:3].copy_(r.bufs["eta"][:3], non_blocking=True)
    side.synchronize()
    with torch.cuda.stream(gen_stream):
        free = torch.cuda.mem_get_info(device)[0]
        pool = torch.empty(int(min(reserve_bytes, 0.8 * free)), dtype=torch.uint8, device=device)
        del pool
    r.bufs = None
    torch.cuda.synchronize(device)


def serve(ctx, reqs, prec="fp64", budget_bytes=48 << 30, max_inflight=64, tol=1e-12, max_iter=30,
          device="cuda", time_limit=600.0, max_tasks=1 << 22, max_edges=1 << 24, keep_x=False):
    """Continuous batching with the resident executor.  Arrival times in
    `reqs` are seconds from the start of the run; the requests' inputs must
    have been built (prepare).  `ctx` must be bound to a stream of its own:
    the resident kernel occupies it for the whole run (admission copies and
    read-backs use other streams)."""
    gen_stream = torch.cuda.Stream(device=device)
    side = torch.cuda.Stream(device=device)
    host = torch.empty(64, dtype=torch.float64, pin_memory=True)
    warm_up(prec, device, gen_stream, side, host, budget_bytes)
    nb = sum(1 for _ in reqs) * (max_iter + 1) + 16
    # from here until stream_close nothing may synchronise the whole device
    ctx.stream_open(max_tasks, max_edges, nb, int(time_limit * 1e9))
    pending = list(reqs)            # not yet arrived (arrival order)
    queue, gen, run, done = [], [], [], []
    used = 0
    t0 = time.perf_counter()
    pi = 0
    try:
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            if now > time_limit:
                raise TimeoutError("serving run exceeded its time limit")
            while pi < len(pending) and pending[pi].arrival <= now:
                queue.append(pending[pi])
                pi += 1
            while queue and len(gen) + len(run) < max_inflight and used + queue[0].bytes <= budget_bytes:
                r = queue.pop(0)
                r.t_admit = time.perf_counter() - t0
                used += r.bytes
                generate(r, prec, device, gen_stream)
                gen.append(r)
            for r in list(gen):
                if r.gen_ev.query():
                    submit_stage(ctx, r, prec, True, tol)
                    r.batch = ctx.stream_submit()
                    r.t_ready = time.perf_counter() - t0
                    r.iters = 1
                    gen.remove(r)
                    run.append(r)
            for r in list(run):
                fin, info = ctx.stream_query(r.batch)
                if not fin:
                    continue
                r.info = r.info or info
                with torch.cuda.stream(side):
                    host[: r.nrhs + 1].copy_(r.bufs["eta"], non_blocking=True)
                side.synchronize()
                r.eta = float(host[r.nrhs])
                if prec != "fp64" and r.info == 0 and r.eta > tol and r.iters < max_iter:
                    submit_stage(ctx, r, prec, False, tol)
                    r.batch = ctx.stream_submit()
                    r.iters += 1
                    continue
                r.t_done = time.perf_counter() - t0
                run.remove(r)
                release(ctx, r, keep_x, side)
                used -= r.bytes
                done.append(r)
            if not gen and not run and not queue and pi < len(pending):
                time.sleep(max(0.0, min(pending[pi].arrival - (time.perf_counter() - t0), 0.001)))
    finally:
        ctx.stream_close()
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.t_done for r in done)
    return _stats(done, t_first, t_last, prec, "continuous")


def serve_plain(ctx, reqs, prec="fp64", tol=1e-12, max_iter=30, device="cuda", time_limit=600.0,
                keep_x=False):
    """Per-request path: requests one at a time in arrival order, one launch
    per stage, nothing overlapped."""
    stream = torch.cuda.current_stream(device)
    done = []
    host = torch.empty(64, dtype=torch.float64, pin_memory=True)
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if now > time_limit:
            raise TimeoutError("plain serving run exceeded its time limit")
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.t_admit = time.perf_counter() - t0
        generate(r, prec, device, stream)
        r.gen_ev.synchronize()
        first = True
        while True:
            submit_stage(ctx, r, prec, first, tol)
            try:
                ctx.task_wait()
            except Exception as e:   # non-SPD request: report and continue
                import paper_1304_0878_b300 as b3t
                if isinstance(e, b3t.B3TError) and e.code == b3t._lib.EDOM:
                    r.info = ctx.last_error()[1]
                    break
                raise
            host[: r.nrhs + 1].copy_(r.bufs["eta"])
            r.eta = float(host[r.nrhs])
            r.iters += 1
            first = False
            if prec == "fp64" or r.eta <= tol or r.iters >= max_iter:
                break
        r.t_done = time.perf_counter() - t0
        release(ctx, r, keep_x)
        done.append(r)
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.t_done for r in done)
    return _stats(done, t_first, t_last, prec, "plain per-request")
