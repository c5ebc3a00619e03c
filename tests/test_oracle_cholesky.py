"""Pins for the oracle's tiled Cholesky (FP64 tile bodies + right-looking
submission order of the partitioned-matrix idiom, Section 5.1)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import cholesky as ch, tiles as tl


def factor_tiled(A, b):
    N = A.shape[0]
    t = ch.to_tiles(A, b)
    info = ch.run(t, N // b, b)
    return np.tril(ch.from_tiles(t, N, b)), info


@pytest.mark.parametrize("N,b", [(8, 4), (32, 8), (64, 16), (1024, 128)])
def test_integer_matrix_factors_exactly(orc, N, b):
    # A = L0 L0^T in integers: every product, sum, sqrt and quotient of the
    # factorisation is exact, so L must equal L0 bit for bit.
    A, L0 = synth.integer_spd(N, seed=N + b)
    L, info = factor_tiled(A, b)
    assert info == 0
    assert np.array_equal(L, L0)


def test_single_tile_equals_unblocked(orc):
    A = synth.spd_host(96, seed=7, shift=1.0)
    L1, info = factor_tiled(A, 96)
    Ld, infod = ch.dense_potrf(A)
    assert info == infod == 0
    assert np.array_equal(L1, np.tril(Ld))


@pytest.mark.parametrize("N,b", [(16, 4), (32, 8), (64, 16), (64, 8)])
def test_tiled_matches_unblocked(orc, N, b):
    A = synth.spd_host(N, seed=N * b, shift=1.0)
    L, info = factor_tiled(A, b)
    Ld, _ = ch.dense_potrf(A)
    Ld = np.tril(Ld)
    assert np.max(np.abs(L - Ld)) / np.max(np.abs(Ld)) <= 1e-14


def test_config1_residual_and_library_crosscheck(orc):
    # N = 1024, tile 128, A = B B^T / N + I, seed 0
    A = synth.spd_host(1024, seed=0, shift=1.0)
    L, info = factor_tiled(A, 128)
    assert info == 0
    assert ch.rel_residual(L, A) <= 1e-13
    assert np.all(np.diag(L) > 0)
    Ls = sla.cholesky(A, lower=True)
    assert np.max(np.abs(L - Ls)) / np.max(np.abs(Ls)) <= 1e-12


def test_closed_forms(orc):
    I = np.eye(32)
    L, _ = factor_tiled(I, 8)
    assert np.array_equal(L, I)
    d = np.arange(1.0, 33.0) ** 2
    L, _ = factor_tiled(np.diag(d), 8)
    assert np.array_equal(L, np.diag(np.arange(1.0, 33.0)))
    a, bb, c = 4.0, 2.0, 5.0
    L, _ = ch.dense_potrf(np.array([[a, bb], [bb, c]]))
    assert np.allclose(np.tril(L), [[2.0, 0.0], [1.0, 2.0]], rtol=0, atol=0)


def test_not_spd_reports_global_column(orc):
    A = synth.spd_host(32, seed=3, shift=1.0)
    A[20, 20] = -50.0
    _, info = factor_tiled(A, 8)
    assert info == 21
    A = np.eye(16)
    A[5, 5] = np.nan
    _, info = factor_tiled(A, 4)
    assert info == 6


def test_tile_bodies_against_definitions(orc):
    rng = np.random.default_rng(5)
    b = 24
    M = rng.standard_normal((b, b))
    Lk = np.tril(M) + b * np.eye(b)
    A = rng.standard_normal((b, b))
    X = np.asfortranarray(A.copy())
    tl.trsm(np.asfortranarray(Lk), X)
    assert np.allclose(X @ Lk.T, A, rtol=0, atol=1e-13)
    B = rng.standard_normal((b, b))
    C = rng.standard_normal((b, b))
    Cg = np.asfortranarray(C.copy())
    tl.gemm(np.asfortranarray(A), np.asfortranarray(B), Cg)
    assert np.allclose(Cg, C - A @ B.T, rtol=0, atol=1e-12)
    Cs = np.asfortranarray(C.copy())
    tl.syrk(np.asfortranarray(A), Cs)
    ref = C - A @ A.T
    assert np.allclose(np.tril(Cs), np.tril(ref), rtol=0, atol=1e-12)
    assert np.array_equal(np.triu(Cs, 1), np.triu(C, 1))   # upper untouched


def test_layout_roundtrip_and_indexing():
    T, b = 5, 3
    N = T * b
    A = np.arange(N * N, dtype=np.float64).reshape(N, N)
    t = ch.to_tiles(A, b)
    assert t.shape == (ch.ntiles(T), b, b)
    # tile (3, 1): element (r, c) of the tile lives at tiles[t][c, r]
    k = ch.tile_index(3, 1, T)
    assert t[k][2, 1] == A[3 * b + 1, 1 * b + 2]
    B = ch.from_tiles(t, N, b)
    for j in range(T):
        for i in range(j, T):
            assert np.array_equal(B[i*b:(i+1)*b, j*b:(j+1)*b], A[i*b:(i+1)*b, j*b:(j+1)*b])
    idx = [ch.tile_index(i, j, T) for j in range(T) for i in range(j, T)]
    assert idx == list(range(ch.ntiles(T)))


def test_flop_count():
    assert ch.flops(1) == 1.0
    # sum of tile-task flops equals the dense count for any T, b
    # (lower-order terms differ: tiles count b^2 (b+1) per SYRK)
    for T, b in [(4, 8), (8, 128), (64, 512)]:
        tot = sum(ch.task_flops(k, b) for k, _ in ch.task_list(T))
        assert tot == pytest.approx(ch.flops(T * b), rel=2.0 / b)


def test_spd_stream_is_row_block_invariant():
    # drawing B in row blocks consumes the same stream as one draw
    rng = np.random.default_rng(9)
    a = rng.standard_normal((6, 10))
    rng = np.random.default_rng(9)
    b = np.concatenate([rng.standard_normal((2, 10)), rng.standard_normal((4, 10))])
    assert np.array_equal(a, b)
