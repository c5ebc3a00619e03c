"""Batched factorisations: many uneven Cholesky factorisations in ONE
persistent-kernel launch, each with its own tile size.

Each matrix gets a tile size from the autotuner (tune.choose_tile); a size
that is not a multiple of it is padded with an identity block (the Cholesky
factor of diag(A, I) is diag(L, I), so the padding changes nothing in L).
All task graphs are submitted before one wait, so the executor runs their
union: tasks of different factorisations fill each other's idle SMs.
"""
import torch

from . import tiles as dt
from . import tune


def padded_tiles(A, b):
    """Dense (N, N) FP64 device tensor -> packed lower tiles of diag(A, I)
    padded to a multiple of b."""
    N = A.shape[0]
    Np = dt.pad_size(N, b)
    if Np != N:
        C = torch.zeros((Np, Np), dtype=A.dtype, device=A.device)
        C[:N, :N] = A
        idx = torch.arange(N, Np, device=A.device)
        C[idx, idx] = 1.0
    else:
        C = A
    return dt.pack_lower(C, b), Np


def cholesky_many(ctx, mats, prec="fp64", tiles=None):
    """Factor every dense FP64 device matrix of `mats` in one launch.
    Returns a list of (L tiles, N, Np, b); the L tiles are packed lower tiles
    of the padded factor.  prec: "fp64" (in place on the tiles) or "bf16" /
    "e4m3" (mixed precision; returns the FP64 L tiles)."""
    import paper_1304_0878_b300 as b3t
    out, keep = [], []
    for k, A in enumerate(mats):
        N = A.shape[0]
        b = tiles[k] if tiles else tune.choose_tile(N, prec)
        t, Np = padded_tiles(A, b)
        T = Np // b
        if prec == "fp64":
            p = dt.tile_ptrs(t)
            ctx.cholesky_submit(p, T, b, 0)
            keep.append((p, T))
            out.append((t, N, Np, b))
        else:
            fmt = b3t.FMT_BF16 if prec == "bf16" else b3t.FMT_E4M3
            W = t.float()
            L = torch.empty_like(t)
            Q = dt.q_tiles(T, b, fmt, A.device)
            ps = [dt.tile_ptrs(W), dt.tile_ptrs(L), dt.tile_ptrs(Q)]
            ctx.cholesky_mx_submit(*ps, T, b, fmt, 0)
            keep.extend((p, T) for p in ps)
            out.append((L, N, Np, b))
            keep.append(("hold", (W, Q)))
    ctx.task_wait()
    for p, T in keep:
        if p != "hold":
            ctx.tiles_unregister(p, T)
    return out
