"""Serving loop: Cholesky-solve requests with continuous batching.

Requests (N x N SPD matrix, nrhs right-hand sides) arrive as a Poisson
process.  The loop admits them in arrival order while their device
footprint fits an HBM budget and a slot is free, uploads each request's
inputs from the client's (pinned) host memory on a side stream, and hands
its work to ONE resident executor (stream mode): every request stage is a
task graph submitted while the others run, so requests that arrive while
others are on the GPU join them as slots and memory free up, and their
tasks share the SMs.

Stages per request:
  * fp64: factorisation + one solve step (x = (L L^T)^{-1} b, residual, eta);
  * bf16 / e4m3: mixed-precision factorisation + first refinement step, then
    one refinement step per stage until eta <= tol (FP64 residual).
Factors stay on the device until the request completes.  Latency is
measured from arrival to the moment the solution is back in host memory:
it includes the upload of A and B (host -> device) at admission and the
download of X (device -> host) at the end.

`serve_plain` is the per-request path for comparison: one request at a time,
one launch per stage, no overlap, with the same uploads and downloads.

Client inputs.  A request's matrix and right-hand sides live in pinned host
memory, as a client would hold them: packed lower FP64 tiles of the padded
matrix diag(A, I) and T parts of b x nrhs.  They are built before serving
(`prepare`, timed separately) on the device, where building them uses library
GEMMs, then copied to the host.  Host memory bounds how many distinct inputs
can be held, so a run of n requests uses the first P requests of the stream
as the input sources: request i arrives at the i-th arrival time of the
stream and carries the size, right-hand-side count and contents of request
i mod P.
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
                 "inputs", "src", "host", "slot")

    def __init__(self, rid, arrival, N, nrhs, seed, src=None):
        self.rid, self.arrival, self.N, self.nrhs, self.seed = rid, arrival, int(N), int(nrhs), int(seed)
        self.src = rid if src is None else src
        self.state = "queued"
        self.iters = 0
        self.eta = float("nan")
        self.info = 0
        self.batch = -1
        self.host = None
        self.slot = None
        self.x = None


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
    """Admission: the client's inputs are uploaded from pinned host memory
    (host -> device copies on `stream`), then the request's working buffers
    are filled from them with elementwise copies (safe next to the resident
    executor)."""
    import paper_1304_0878_b300 as b3t
    T, b, nrhs = req.T, req.b, req.nrhs
    A_h, rhs_h = req.host
    with torch.cuda.stream(stream):
        A = torch.empty(A_h.shape, dtype=A_h.dtype, device=device)
        A.copy_(A_h, non_blocking=True)
        rhs = torch.empty(rhs_h.shape, dtype=rhs_h.dtype, device=device)
        rhs.copy_(rhs_h, non_blocking=True)
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


def prepare(reqs, device="cuda", pool=None):
    """Build the client inputs of every distinct source of `reqs` on the
    device and keep them in pinned host memory (before serving); returns
    (seconds, pinned bytes of the sources built).  `pool` (a dict, source ->
    host tensors) is reused and filled, so that runs over the same stream
    share one set of client inputs."""
    t0 = time.perf_counter()
    s = torch.cuda.current_stream(device)
    pool = {} if pool is None else pool
    nbytes = 0
    for r in reqs:
        if r.src not in pool:
            make_inputs(r, device, s)
            A, rhs = r.inputs
            A_h = torch.empty(A.shape, dtype=A.dtype, pin_memory=True)
            rhs_h = torch.empty(rhs.shape, dtype=rhs.dtype, pin_memory=True)
            A_h.copy_(A)
            rhs_h.copy_(rhs)
            pool[r.src] = (A_h, rhs_h)
            nbytes += A_h.numel() * 8 + rhs_h.numel() * 8
            r.inputs = None
        r.host = pool[r.src]
        if r.host[0].shape[0] != r.T * (r.T + 1) // 2 or r.host[0].shape[1] != r.b or r.host[1].shape != (r.T, r.nrhs, r.b):
            raise ValueError("client input of source %d does not fit request %d (pool built for another stream)"
                             % (r.src, r.rid))
    torch.cuda.synchronize(device)
    return time.perf_counter() - t0, nbytes


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


def download(req, slot, stream, keep_x=False):
    """The solution back to the client: X (T parts of b x nrhs) into pinned
    host memory `slot` (device -> host on `stream`), waited for; keep_x also
    keeps a copy of it on the request."""
    X = req.bufs["X"]
    n = X.numel()
    with torch.cuda.stream(stream):
        slot[:n].copy_(X.view(-1), non_blocking=True)
    stream.synchronize()
    if keep_x:
        req.x = slot[:n].clone().view(X.shape)


def release(ctx, req):
    """Forget the request's registrations (its batches are done)."""
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


def make_requests(n, rate, seed, nmin=256, nmax=8192, rmax=32, prec="fp64", tile=None, distinct=None):
    """n requests (Poisson arrivals at `rate` per second); the tile size is
    the tuner's choice for each N unless `tile` fixes it.  With `distinct`
    = P < n, request i takes the size, right-hand sides and seed of request
    i mod P of the stream (the input sources) and its own arrival time."""
    import synth
    arr, Ns, nrhs, seeds = synth.serve_requests(n, rate=rate, seed=seed, nmin=nmin, nmax=nmax, rmax=rmax)
    P = n if distinct is None else max(1, min(n, distinct))
    out = []
    for i in range(n):
        j = i % P
        r = Request(i, float(arr[i]), Ns[j], nrhs[j], seeds[j] % (2 ** 62), src=j)
        r.b = tile or tune.choose_tile(r.N, prec)
        r.Np = dt.pad_size(r.N, r.b)
        r.T = r.Np // r.b
        r.bytes = footprint(r.Np, r.nrhs, r.b, prec)
        out.append(r)
    return out


def _timeline(samples, t_end, bins=24):
    """Queue length and admission over time: per time bin, requests that
    arrived, were admitted and completed, and the largest queue seen."""
    if not samples:
        return []
    w = max(t_end, 1e-6) / bins
    out = []
    k = 0
    prev = (0, 0, 0)
    for i in range(bins):
        hi = (i + 1) * w
        mq = 0
        last = None
        while k < len(samples) and samples[k][0] <= hi:
            mq = max(mq, samples[k][1])
            last = samples[k]
            k += 1
        if last is None:
            continue
        arrived, admitted, completed = last[3], last[4], last[5]
        out.append({"t_s": round(hi, 3), "arrived": arrived - prev[0], "admitted": admitted - prev[1],
                    "completed": completed - prev[2], "max_queue": mq, "in_flight": last[2]})
        prev = (arrived, admitted, completed)
    return out


def _stats(reqs, t_first, t_last, prec, mode):
    lat = np.array([r.t_done - r.arrival for r in reqs]) * 1e3
    qd = np.array([r.t_admit - r.arrival for r in reqs]) * 1e3
    ok = [r for r in reqs if r.info == 0]
    h2d = sum(r.host[0].numel() * 8 + r.host[1].numel() * 8 for r in reqs)
    d2h = sum(r.host[1].numel() * 8 for r in reqs)
    return {
        "mode": mode, "precision": prec, "requests": len(reqs),
        "distinct_inputs": len({r.src for r in reqs}),
        "h2d_bytes": h2d, "d2h_bytes": d2h,
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
    and workspaces of the generation stream, the random generator, pinned
    staging, and the caching allocator's pools (one large reservation, freed
    into torch's cache so that later allocations on that stream reuse it)."""
    r = Request(-1, 0.0, 300, 2, 1)
    r.b = tune.choose_tile(r.N, prec)
    r.Np = dt.pad_size(r.N, r.b)
    r.T = r.Np // r.b
    prepare([r], device)
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


def stream_capacity(reqs, prec, iters):
    """Upper bounds on the tasks and edges the stream executor's fixed
    arenas must hold for `reqs` (stream mode does not reuse the slots of
    retired batches): per request the factorisation (POTRF / TRSM (+ QUANT)
    / SYRK / GEMM tasks, the diagonal-panel tasks) and `iters` solve or
    refinement steps (each about T^2 + 4T + 4 vector tasks), with three edges
    per task and a quarter of slack."""
    tasks = 0
    for r in reqs:
        T = r.T
        pan = (r.b // 64) ** 2 if r.b >= 256 else 1
        fac = T * pan + T * (T - 1) + T * (T - 1) // 2 + T * (T - 1) * (T - 2) // 6 + 2 * T
        step = T * T + 4 * T + 4
        tasks += fac + iters * step
    tasks = int(tasks * 1.25) + 4096
    return tasks, 3 * tasks


def _result_slots(reqs, k):
    """k pinned host buffers, each large enough for any request's X."""
    n = max(r.Np * r.nrhs for r in reqs)
    return [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(k)]


def serve(ctx, reqs, prec="fp64", budget_bytes=48 << 30, max_inflight=64, tol=1e-12, max_iter=30,
          device="cuda", time_limit=600.0, max_tasks=None, max_edges=None, keep_x=False):
    """Continuous batching with the resident executor.  Arrival times in
    `reqs` are seconds from the start of the run; the requests' client inputs
    must be in host memory (prepare).  `ctx` must be bound to a stream of its
    own: the resident kernel occupies it for the whole run (uploads,
    admission copies and read-backs use other streams).  The stream's
    arenas are sized by stream_capacity (12 refinement steps per mixed
    request) unless max_tasks / max_edges are given."""
    if max_tasks is None or max_edges is None:
        mt, me = stream_capacity(reqs, prec, 1 if prec == "fp64" else 12)
        max_tasks = max_tasks or mt
        max_edges = max_edges or me
    gen_stream = torch.cuda.Stream(device=device)
    side = torch.cuda.Stream(device=device)
    host = torch.empty(64, dtype=torch.float64, pin_memory=True)
    warm_up(prec, device, gen_stream, side, host, budget_bytes)
    free_slots = _result_slots(reqs, max_inflight)
    nb = sum(1 for _ in reqs) * (max_iter + 1) + 16
    # from here until stream_close nothing may synchronise the whole device
    ctx.stream_open(max_tasks, max_edges, nb, int(time_limit * 1e9))
    pending = list(reqs)            # not yet arrived (arrival order)
    queue, gen, run, done = [], [], [], []
    used = 0
    samples = []
    t_sample = -1.0
    admitted = 0
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
                r.slot = free_slots.pop()
                generate(r, prec, device, gen_stream)
                gen.append(r)
                admitted += 1
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
                download(r, r.slot, side, keep_x)
                r.t_done = time.perf_counter() - t0
                run.remove(r)
                release(ctx, r)
                free_slots.append(r.slot)
                r.slot = None
                used -= r.bytes
                done.append(r)
            if now - t_sample >= 0.02:
                samples.append((now, len(queue), len(gen) + len(run), pi, admitted, len(done)))
                t_sample = now
            if not gen and not run and not queue and pi < len(pending):
                time.sleep(max(0.0, min(pending[pi].arrival - (time.perf_counter() - t0), 0.001)))
    finally:
        ctx.stream_close()
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.t_done for r in done)
    st = _stats(done, t_first, t_last, prec, "continuous")
    samples.append((t_last, 0, 0, pi, admitted, len(done)))
    st["max_queue"] = max(x[1] for x in samples)
    st["timeline"] = _timeline(samples, t_last)
    return st


def serve_plain(ctx, reqs, prec="fp64", tol=1e-12, max_iter=30, device="cuda", time_limit=600.0,
                keep_x=False):
    """Per-request path: requests one at a time in arrival order, one launch
    per stage, nothing overlapped (uploads and downloads as in serve)."""
    stream = torch.cuda.current_stream(device)
    done = []
    host = torch.empty(64, dtype=torch.float64, pin_memory=True)
    slot = _result_slots(reqs, 1)[0]
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
        download(r, slot, stream, keep_x)
        r.t_done = time.perf_counter() - t0
        release(ctx, r)
        done.append(r)
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.t_done for r in done)
    return _stats(done, t_first, t_last, prec, "plain per-request")
