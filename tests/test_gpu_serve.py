"""Serving with continuous batching (GPU): every served solution is checked
against the oracle (its sequential tiled Cholesky and substitutions on the
request's own matrix and right-hand sides, as the client uploaded them), the
backward error is recomputed on the host, and each request's solution
computed in the mix (stream mode, overlapping with other requests) is
bit-for-bit the solution of the same request served alone (one request at a
time)."""
import copy
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import serve as sv
from paper_1304_0878_b300 import batch as bt
import serve_oracle
import synth
from oracle import cholesky as och, ir as oir

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


def requests(n, rate, prec, nmin=200, nmax=1536):
    tile = 256 if nmin > 2048 else None
    return sv.make_requests(n, rate, seed=5, nmin=nmin, nmax=nmax, rmax=8, prec=prec, tile=tile)


# the large cases use tiles of 256 (diagonal tiles split into column panels)
# and, with two requests in flight, reuse freed buffers' addresses
@pytest.mark.parametrize("prec,tol,n,nmin,nmax,inflight", [
    ("fp64", 1e-14, 10, 200, 1536, 6), ("bf16", 1e-12, 10, 200, 1536, 6),
    ("fp64", 1e-14, 6, 2100, 3500, 2), ("bf16", 1e-12, 6, 2100, 3500, 2)])
def test_serve_mix_equals_alone(orc, prec, tol, n, nmin, nmax, inflight):
    reqs = requests(n, 400.0, prec, nmin, nmax)
    sv.prepare(reqs)
    # the oracle's solutions, computed on the host cores while the GPU serves
    # (worker processes started with spawn: they never touch CUDA)
    pool = ProcessPoolExecutor(max_workers=min(n, 8), mp_context=mp.get_context("spawn"))
    futs = [pool.submit(serve_oracle.solve, (r.host[0].numpy().copy(), r.host[1].numpy().copy(), r.Np, r.b))
            for r in reqs]
    side = torch.cuda.Stream()
    # FP64 requests are served by the resident kernel without the
    # tensor-memory path (two CTAs per SM)
    ctx = b3t.Context(stream=side.cuda_stream, timeout_ns=20_000_000_000, stream_no_mx=prec == "fp64")
    st = sv.serve(ctx, reqs, prec=prec, budget_bytes=2 << 30, max_inflight=inflight, time_limit=120.0,
                  max_tasks=1 << 20, max_edges=1 << 22, keep_x=True)
    ctx.close()
    assert st["requests"] == n and st["failed"] == 0
    assert all(r.eta <= tol for r in reqs)
    alone = [copy.copy(r) for r in requests(n, 1e9, prec, nmin, nmax)]     # same requests, served one by one
    sv.prepare(alone)
    c2 = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    sv.serve_plain(c2, alone, prec=prec, keep_x=True)
    c2.close()
    for r, a in zip(reqs, alone):
        assert r.N == a.N and r.iters == a.iters
        assert torch.equal(r.x, a.x)
    # against the oracle: FP64 to the oracle's own rounding level; mixed
    # precision refined to eta <= 1e-12 agrees to about kappa(A) * 1e-12
    # (kappa <= 5 for A = B B^T / N + I), and the backward error recomputed
    # on the host from the uploaded A and B and the downloaded X meets the
    # target (the FP64 residual of an N <= 3584 system adds at most ~1e-13)
    xtol = 1e-13 if prec == "fp64" else 1e-10
    for r, f in zip(reqs, futs):
        Xo, A, Bm = f.result()
        X = serve_oracle.dense_rhs(r.x.numpy())
        assert np.max(np.abs(X - Xo)) / np.max(np.abs(Xo)) <= xtol
        assert oir.backward_error(A, X, Bm) <= 2e-12
    pool.shutdown()


def test_batch_uneven_sizes_one_launch(orc):
    # many uneven factorisations in one launch, tile sizes from the tuner,
    # ragged sizes padded with identity: each equals its own factorisation
    sizes = [300, 1000, 513, 2048, 77, 1500]
    mats = [synth.spd_host(N, seed=N, shift=1.0) for N in sizes]
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    out = bt.cholesky_many(ctx, [torch.from_numpy(A).cuda() for A in mats])
    ctx.close()
    for A, (t, N, Np, b) in zip(mats, out):
        L = np.tril(och.from_tiles(t.cpu().numpy(), Np, b))
        assert np.array_equal(L[N:, N:], np.eye(Np - N))      # identity padding
        assert np.all(L[N:, :N] == 0)
        Lo, info = och.dense_potrf(A)
        Lo = np.tril(Lo)
        assert info == 0
        assert np.max(np.abs(L[:N, :N] - Lo)) / np.max(np.abs(Lo)) <= 1e-12


@pytest.mark.parametrize("prec", ["bf16", "e4m3"])
def test_batch_mixed_precision_one_launch(orc, prec):
    # cholesky_many in mixed precision: uneven sizes in one launch, tiles from
    # the tuner, ragged sizes padded with identity.  Each factor is bitwise
    # the one its matrix gets factored alone with the same tile (the order of
    # every element's operations does not depend on the other requests), and
    # its residual is that of the mixed oracle's factor of the padded matrix
    # (the same low-precision factor up to the order of the binary32 sums)
    from oracle import mixed as omx
    sizes = [300, 1000, 513, 640]
    mats = [synth.spd_host(N, seed=N + 1, shift=1.0) for N in sizes]
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=20_000_000_000)
    out = bt.cholesky_many(ctx, [torch.from_numpy(A).cuda() for A in mats], prec=prec)
    for A, (t, N, Np, b) in zip(mats, out):
        L = np.tril(och.from_tiles(t.cpu().numpy(), Np, b))
        assert np.array_equal(L[N:, N:], np.eye(Np - N)) and np.all(L[N:, :N] == 0)
        (t1, _, _, _), = bt.cholesky_many(ctx, [torch.from_numpy(A).cuda()], prec=prec, tiles=[b])
        assert np.array_equal(np.tril(och.from_tiles(t1.cpu().numpy(), Np, b)), L)
        Ap = np.eye(Np)
        Ap[:N, :N] = A
        Lt, info = omx.factor(och.to_tiles(Ap, b), Np // b, b, prec)
        assert info == 0
        Lo = np.tril(och.from_tiles(Lt, Np, b))
        r_dev, r_orc = och.rel_residual(L[:N, :N], A), och.rel_residual(Lo[:N, :N], A)
        assert r_dev <= 2.0 * r_orc and r_orc <= 2.0 * r_dev
    ctx.close()
