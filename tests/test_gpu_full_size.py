"""Parity at the full sizes of the headline workloads (GPU), in the launch
configuration the benchmark times (the DAG captured once, replayed), on
outputs the oracle can check one by one:

  * tiled Cholesky, FP64, N = 32768, tile 512: the leading 2048 x 2048 block
    of L equals the oracle's unblocked factorisation of A's leading block (a
    leading principal submatrix factors to the leading block of L); sampled
    entries of L L^T equal A; a second replay is bitwise identical;
  * mixed precision (bf16, E4M3 updates) + FP64 refinement at the same size,
    16 right-hand sides: the refinement converges, and sampled rows of the
    residual b - A x, formed in FP64 on the host, meet the backward-error
    target with the exact infinity norm of A.
"""
import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt
from oracle import cholesky as och

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

N, B = 32768, 512
T = N // B
NRHS = 16


@pytest.fixture(scope="module")
def a0():
    A = synth.spd_tiles_device(N, B, 3, 0.1, "cuda")
    yield A
    del A
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def anorm(a0):
    """Exact infinity norm of the symmetric A, one tile at a time on the host."""
    rows = np.zeros(N)
    for j in range(T):
        for i in range(j, T):
            F = np.abs(tile(a0, i, j))
            if i == j:
                F = np.tril(F) + np.tril(F, -1).T
                rows[i * B:(i + 1) * B] += F.sum(axis=1)
            else:
                rows[i * B:(i + 1) * B] += F.sum(axis=1)
                rows[j * B:(j + 1) * B] += F.sum(axis=0)
    return float(rows.max())


def tile(tl, i, j):
    """Host copy of tile (i, j): F[r, c] = element (i*B + r, j*B + c)."""
    return tl[dt.tile_index(i, j, T)].cpu().numpy().T


def lower_row(tl, i):
    """Row i of the lower triangle (entries k <= i), from the tiles."""
    I, r = divmod(i, B)
    parts = [tl[dt.tile_index(I, J, T), :, r] for J in range(I + 1)]
    return torch.cat(parts).cpu().numpy()[: i + 1]


def sym_row(tl, i):
    """Row i of the symmetric matrix whose lower triangle the tiles hold."""
    I, r = divmod(i, B)
    out = np.empty(N)
    for J in range(T):
        if J < I:
            out[J * B:(J + 1) * B] = tl[dt.tile_index(I, J, T), :, r].cpu().numpy()
        elif J > I:
            out[J * B:(J + 1) * B] = tl[dt.tile_index(J, I, T), r, :].cpu().numpy()
        else:
            F = tile(tl, I, I)
            c = np.arange(B)
            out[I * B:(I + 1) * B] = np.where(c <= r, F[r, c], F[c, r])
    return out


def test_cholesky_full_size_sampled(orc, a0):
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=120_000_000_000)
    t = torch.empty_like(a0)
    ptrs = dt.tile_ptrs(t)
    ctx.graph_capture_begin()
    ctx.cholesky_submit(ptrs, T, B)
    g = ctx.graph_capture_end()
    t.copy_(a0)
    ctx.graph_replay(g)
    ctx.task_wait()
    first = t.clone()
    t.copy_(a0)
    ctx.graph_replay(g)
    ctx.task_wait()
    assert torch.equal(t, first)                                    # bitwise deterministic
    del first
    ctx.graph_destroy(g)
    ctx.tiles_unregister(ptrs, T)
    ctx.close()
    # leading block: 4 x 4 tiles against the oracle's dense factorisation
    k = 4
    Ak = np.zeros((k * B, k * B))
    Lk = np.zeros((k * B, k * B))
    for i in range(k):
        for j in range(i + 1):
            Ak[i * B:(i + 1) * B, j * B:(j + 1) * B] = tile(a0, i, j)
            Lk[i * B:(i + 1) * B, j * B:(j + 1) * B] = tile(t, i, j)
    Ak = np.tril(Ak) + np.tril(Ak, -1).T
    Lo, info = och.dense_potrf(Ak)
    assert info == 0
    Lo = np.tril(Lo)
    assert np.max(np.abs(np.tril(Lk) - Lo)) / np.max(np.abs(Lo)) <= 1e-12
    # sampled entries of L L^T, FP64 dot products on the host
    rng = np.random.default_rng(0)
    amax = float(a0.abs().max())
    worst = 0.0
    for _ in range(48):
        i = int(rng.integers(0, N))
        j = int(rng.integers(0, i + 1))
        li, lj = lower_row(t, i), lower_row(t, j)
        m = j + 1
        v = float(np.dot(li[:m], lj[:m]))
        worst = max(worst, abs(v - sym_row(a0, i)[j]) / amax)
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("fmt", [b3t.FMT_BF16, b3t.FMT_E4M3])
def test_mixed_refinement_full_size_sampled(orc, a0, anorm, fmt):
    ctx = b3t.Context(stream=torch.cuda.current_stream().cuda_stream, timeout_ns=120_000_000_000)
    Bh = synth.rhs(N, NRHS, seed=4)                                   # N x NRHS, column-major
    Bd = torch.from_numpy(np.ascontiguousarray(Bh.reshape(T, B, NRHS).transpose(0, 2, 1))).cuda()
    X = torch.zeros_like(Bd)
    R = torch.zeros(b3t.ir_work_elems(T, B, NRHS), dtype=torch.float64, device="cuda")
    eta = torch.zeros(NRHS + 1, dtype=torch.float64, device="cuda")
    W = torch.empty(a0.shape, dtype=torch.float32, device="cuda")
    L = torch.zeros_like(a0)
    Q = dt.q_tiles(T, B, fmt, "cuda")
    wp, lp, qp = dt.tile_ptrs(W), dt.tile_ptrs(L), dt.tile_ptrs(Q)
    ctx.graph_capture_begin()
    ctx.cholesky_mx_submit(wp, lp, qp, T, B, fmt)
    g = ctx.graph_capture_end()
    W.copy_(a0)
    ctx.graph_replay(g)
    ctx.task_wait()
    rc, its, e = ctx.ir_solve(a0.data_ptr(), lp, Bd.data_ptr(), X.data_ptr(), R.data_ptr(), eta.data_ptr(),
                              T, B, NRHS, b3t.VEC_F32, 1e-12, 30)
    ctx.graph_destroy(g)
    for p in (qp, wp, lp):
        ctx.tiles_unregister(p, T)
    ctx.close()
    assert rc == 0 and 1 <= its <= 30 and e[NRHS] <= 1e-12
    Xh = X.cpu().numpy().transpose(0, 2, 1).reshape(N, NRHS)        # back to N x NRHS
    xn = np.abs(Xh).max(axis=0)
    bn = np.abs(Bh).max(axis=0)
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(32):
        i = int(rng.integers(0, N))
        r = Bh[i] - sym_row(a0, i) @ Xh
        worst = max(worst, float(np.max(np.abs(r) / (anorm * xn + bn))))
    assert worst <= 1e-12, worst
