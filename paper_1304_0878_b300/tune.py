"""Tile-size autotuner for the tiled Cholesky DAG.

The best tile size depends on N and on the precision: small tiles give more
parallel tasks (and a shorter critical path per step), large tiles give
fewer, more efficient tasks.  `sweep` measures one factorisation per
(precision, N, b) on the device (the DAG captured once, replayed), and
`choose_tile` answers from the measured table, falling back to a rule of
thumb for sizes outside it.

    python -m paper_1304_0878_b300.tune [--out PATH]   # on the GPU

writes the table next to this file (tune_table.json).
"""
import json
import os
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(PKG, "tune_table.json")
TILES = {"fp64": (64, 128, 256, 512), "bf16": (128, 256, 512), "e4m3": (128, 256, 512)}
SIZES = (256, 512, 1024, 2048, 4096, 8192)

_table = None


def default_tile(N, prec="fp64"):
    """Rule of thumb: about 8-32 tiles per side, tiles of 128..512."""
    if prec == "fp64":
        return 64 if N <= 512 else 128 if N <= 2048 else 256 if N <= 8192 else 512
    return 128 if N <= 2048 else 256 if N <= 8192 else 512


def load(path=TABLE):
    global _table
    if os.path.exists(path):
        with open(path) as f:
            _table = json.load(f)
    else:
        _table = {}
    return _table


def choose_tile(N, prec="fp64"):
    """Tile size for an N x N factorisation: the measured best at the
    nearest tuned size (in log scale), else the rule of thumb."""
    if _table is None:
        load()
    rows = _table.get(prec, {})
    if not rows:
        return default_tile(N, prec)
    import math
    best_n = min(rows, key=lambda k: abs(math.log(int(k)) - math.log(max(N, 1))))
    b = int(rows[best_n]["best"])
    while b > 64 and b >= 2 * N:      # never more than one mostly-padded tile
        b //= 2
    if prec != "fp64":
        b = max(b, 128)
    return b


def sweep(ctx, sizes=SIZES, precs=("fp64", "bf16"), reps=3, device="cuda"):
    """Measure factorisation time for every (precision, N, tile)."""
    import torch
    import synth
    import paper_1304_0878_b300 as b3t
    from . import tiles as dt
    out = {}
    for prec in precs:
        out[prec] = {}
        for N in sizes:
            res = {}
            for b in TILES[prec]:
                if b > N or N % b:
                    continue
                T = N // b
                A = dt.to_tiles(torch.from_numpy(synth.spd_host(N, seed=N, shift=1.0)).to(device), b)
                t = torch.empty_like(A)
                ctx.graph_capture_begin()
                if prec == "fp64":
                    ptrs = [dt.tile_ptrs(t)]
                    ctx.cholesky_submit(ptrs[0], T, b)
                else:
                    fmt = b3t.FMT_BF16 if prec == "bf16" else b3t.FMT_E4M3
                    W = A.float()
                    L = torch.empty_like(A)
                    Q = dt.q_tiles(T, b, fmt, device)
                    ptrs = [dt.tile_ptrs(W), dt.tile_ptrs(L), dt.tile_ptrs(Q)]
                    ctx.cholesky_mx_submit(*ptrs, T, b, fmt)
                g = ctx.graph_capture_end()
                ts = []
                for r in range(reps + 1):
                    if prec == "fp64":
                        t.copy_(A)
                    else:
                        W.copy_(A)
                    ctx.graph_replay(g)
                    ctx.task_wait()
                    if r:
                        ts.append(ctx.last_launch()["kernel_ns"] / 1e6)
                ctx.graph_destroy(g)
                for p in ptrs:
                    ctx.tiles_unregister(p, T)
                res[str(b)] = min(ts)
            best = min(res, key=res.get)
            out[prec][str(N)] = {"ms": res, "best": int(best)}
            print(prec, N, res, "best", best, file=sys.stderr)
    return out


def main():
    import torch
    import paper_1304_0878_b300 as b3t
    path = TABLE
    if "--out" in sys.argv:
        path = sys.argv[sys.argv.index("--out") + 1]
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=60_000_000_000)
    t0 = time.time()
    table = sweep(ctx)
    table["meta"] = {"device": torch.cuda.get_device_name(0), "seconds": time.time() - t0}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    ctx.close()
    print(path)


if __name__ == "__main__":
    main()
