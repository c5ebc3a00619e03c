"""Seeded synthetic inputs shared by the oracle and the device path.

This module holds no arithmetic of the method (no tile kernel, no
dependency rule, no factorisation step): only random draws and the
construction of the input matrices.  Both sides consume the identical bytes.

Recipes (numpy PCG64 ``default_rng(seed)`` unless stated):
  * vector chains: x ~ U[-1, 1) drawn in float64 then rounded to float32;
    factors f[blk][k] ~ U[0.5, 2) drawn block-major (blk outer, k inner),
    rounded to float32.
  * SPD matrices: A = B B^T / N + shift * I with B_ij ~ N(0, 1) (float64).
    Division by N is exact for N a power of two.  Large N (spd_tiles_device)
    is formed on the GPU in binary32 and widened to FP64.
  * integer SPD matrices: A = L0 L0^T with L0 lower triangular, small
    integer entries and a positive integer diagonal, formed in int64 (exact
    below 2^53), so every Cholesky step on it is exact.
  * right-hand sides: N(0, 1) float64, column-major N x nrhs.
  * random task sets for dependency fuzzing: handles and modes uniform.
  * serving requests: Poisson arrivals, log-uniform sizes, per-request seeds
    from SeedSequence(seed).spawn(n).
"""
import math

import numpy as np


def vector_f32(n, seed=1, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    out = np.empty(n, dtype=np.float32)
    step = 1 << 24
    for s in range(0, n, step):
        m = min(step, n - s)
        out[s:s + m] = rng.uniform(lo, hi, m).astype(np.float32)
    return out


def chain_factors(nblocks, nchain, seed=2, lo=0.5, hi=2.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (nblocks, nchain)).astype(np.float32)


def gaussian(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def spd_host(N, seed=0, shift=1.0):
    """A = B B^T / N + shift I, FP64, formed on the host (small N)."""
    B = gaussian((N, N), seed)
    A = (B @ B.T) / N
    A[np.diag_indices(N)] += shift
    return A


def spd_tiles_device(N, b, seed, shift, device):
    """Packed lower tiles (column-major inside a tile) of an SPD matrix
    A = B B^T / N + shift I formed on `device`, for sizes too large to form on
    the host: B ~ N(0, 1) is drawn in binary32 by torch's CUDA generator
    seeded with `seed`, B B^T is formed by a binary32 matmul (no TF32) one
    row block of tiles at a time, then widened to FP64, divided by N (exact)
    and shifted.  The bytes returned are the input's definition.  Returns a
    tensor of shape (T(T+1)/2, b, b) with out[t, c, r] = A[i*b + r, j*b + c]
    for tile t = (i, j) in packed column order."""
    import torch
    assert N % b == 0
    T = N // b
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    B = torch.randn((N, N), generator=g, device=device, dtype=torch.float32)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        nt = T * (T + 1) // 2
        out = torch.empty((nt, b, b), dtype=torch.float64, device=device)
        for i in range(T):
            blk = (B[i * b:(i + 1) * b] @ B[:(i + 1) * b].T).double() / N   # b x (i+1)b
            for j in range(i + 1):
                t = j * T - j * (j - 1) // 2 + (i - j)
                out[t] = blk[:, j * b:(j + 1) * b].T
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del B
    idx = torch.arange(b, device=device)
    for k in range(T):
        t = k * T - k * (k - 1) // 2
        out[t, idx, idx] += shift
    return out


def integer_lower(N, seed, lo=-3, hi=3, dlo=1, dhi=4):
    """Lower-triangular int64 L0 with entries in [lo, hi] and diagonal in
    [dlo, dhi] (positive)."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.integers(lo, hi + 1, (N, N)), -1)
    L0[np.diag_indices(N)] = rng.integers(dlo, dhi + 1, N)
    return L0.astype(np.int64)


def integer_spd(N, seed, **kw):
    """(A, L0) with A = L0 L0^T computed exactly in int64, returned as float64."""
    L0 = integer_lower(N, seed, **kw)
    A = L0 @ L0.T
    assert np.max(np.abs(A)) < 2 ** 53
    return A.astype(np.float64), L0.astype(np.float64)


def rhs(N, nrhs, seed=4):
    return np.asfortranarray(gaussian((N, nrhs), seed))


def random_accesses(ntasks, nhandles, maxbuf, seed):
    """Random task sets: each task names 1..maxbuf distinct handles with
    modes drawn from {R=1, W=2, RW=3}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ntasks):
        k = int(rng.integers(1, maxbuf + 1))
        hs = rng.choice(nhandles, size=min(k, nhandles), replace=False)
        out.append([(int(h), int(rng.integers(1, 4))) for h in hs])
    return out


def serve_requests(n, rate=2000.0, seed=5, nmin=256, nmax=8192, rmin=1, rmax=32, total=100000):
    """The first n of a stream of `total` Cholesky-solve requests: arrival
    times (s) of a Poisson process of the given rate, N log-uniform on
    [nmin, nmax], nrhs uniform on {rmin..rmax}, and an independent seed per
    request.  The whole stream is drawn (gaps, then sizes, then right-hand
    side counts, each for `total` requests) and its prefix returned, so the
    first k requests are the same whatever n >= k is asked for."""
    m = max(n, total)
    root = np.random.SeedSequence(seed)
    rng = np.random.default_rng(root)
    gaps = rng.exponential(1.0 / rate, m)[:n]
    arrival = np.cumsum(gaps)
    N = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), m))).astype(np.int64)[:n]
    nrhs = rng.integers(rmin, rmax + 1, m)[:n]
    seeds = [int(s.generate_state(1)[0]) for s in root.spawn(n)]
    return arrival, N, nrhs, seeds
