"""Pins for the oracle's low-precision pieces: rounding to bfloat16 / E4M3,
the power-of-two per-tile scale, the binary32-accumulated update and the
mixed-precision factorisation.

The quantisation of a panel tile is one rounding, q = RN_fmt(x / 2^e),
straight from FP64.  It is pinned here against an independent exact
computation in rational arithmetic (fractions.Fraction), including FP64
values just off a midpoint of the format's grid, where rounding through
binary32 first would land on the midpoint and then round the other way."""
import math

import numpy as np
import pytest
import torch

import synth
from fpgrid import chain_round, exact_round, grid_midpoints, ulp32
from oracle import cholesky as ch, mixed, tiles as tl


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3e38, -3.4e38, 1e-40]]).astype(np.float32)
    ours = tl.round_format(x, "bf16")
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: rounds to 1 (even)
    assert tl.round_format(np.float32(1 + 2 ** -8), "bf16") == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: rounds up (even)
    assert tl.round_format(np.float32(1 + 3 * 2 ** -8), "bf16") == 1 + 2 ** -6


def test_e4m3_rounding_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = (rng.uniform(-440, 440, 5000) * 2.0 ** rng.integers(-12, 0, 5000)).astype(np.float32)
    ours = tl.round_format(x, "e4m3")
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_e4m3_saturates_and_grid():
    assert tl.round_format(np.float32(1000.0), "e4m3") == 448.0
    assert tl.round_format(np.float32(-470.0), "e4m3") == -448.0
    assert tl.round_format(np.float32(17.0), "e4m3") == 16.0     # 4 significant bits
    assert tl.round_format(np.float32(2 ** -9), "e4m3") == 2 ** -9   # smallest subnormal
    assert tl.round_format(np.float32(2 ** -11), "e4m3") == 0.0


def test_scale_exponent():
    assert tl.scale_exponent(448.0, "e4m3") == 0
    assert tl.scale_exponent(448.0001, "e4m3") == 1
    assert tl.scale_exponent(224.0, "e4m3") == -1
    assert tl.scale_exponent(16.0, "e4m3") == -4
    assert tl.scale_exponent(0.0, "e4m3") == 0
    assert tl.scale_exponent(123.0, "bf16") == 0
    for a in np.random.default_rng(2).uniform(1e-6, 1e6, 200):
        e = tl.scale_exponent(a, "e4m3")
        assert a <= 448 * 2.0 ** e and a > 448 * 2.0 ** (e - 1)


def test_lowp_update_exact_on_integers():
    rng = np.random.default_rng(3)
    A = np.asfortranarray(rng.integers(-16, 17, (64, 96)).astype(np.float64))
    B = np.asfortranarray(rng.integers(-16, 17, (32, 96)).astype(np.float64))
    C0 = rng.integers(-1000, 1000, (64, 32)).astype(np.float32)
    C = np.asfortranarray(C0.copy())
    tl.gemm_lowp(A, B, 1.0, C)
    assert np.array_equal(C, (C0 - A @ B.T).astype(np.float32))
    C = np.asfortranarray(C0[:32, :32].copy())
    A32 = np.asfortranarray(A[:32])
    tl.gemm_lowp(A32, A32, 4.0, C, lower=True)
    ref = C0[:32, :32] - 4.0 * A[:32] @ A[:32].T
    assert np.array_equal(np.tril(C), np.tril(ref).astype(np.float32))
    assert np.array_equal(np.triu(C, 1), np.triu(C0[:32, :32], 1))


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_mixed_factor_exact_on_integer_matrix(fmt):
    # entries of L0 in [-3, 3], diagonal in [1, 4]: representable in both
    # formats after a power-of-two scale, products and sums exact
    N, b = 64, 16
    A, L0 = synth.integer_spd(N, seed=21)
    Lt, info = mixed.factor(ch.to_tiles(A, b), N // b, b, fmt)
    assert info == 0
    assert np.array_equal(np.tril(ch.from_tiles(Lt, N, b)), L0)


@pytest.mark.parametrize("fmt,lo,hi", [("bf16", 1e-6, 5e-2), ("e4m3", 1e-4, 1.0)])
def test_mixed_factor_is_low_precision(fmt, lo, hi):
    N, b = 256, 64
    A = synth.spd_host(N, seed=4, shift=1.0)
    Lt, info = mixed.factor(ch.to_tiles(A, b), N // b, b, fmt)
    assert info == 0
    r = ch.rel_residual(np.tril(ch.from_tiles(Lt, N, b)), A)
    assert lo < r < hi


# ---- quantisation pinned to its definition in exact arithmetic

@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_quantise_is_one_rounding_from_fp64(fmt):
    rng = np.random.default_rng(11)
    p, emin, maxval, _ = tl.FORMATS[fmt]
    # random FP64 values over the format's whole range and beyond it
    mags = rng.uniform(-1, 1, 3000) * 2.0 ** rng.uniform(emin - p - 3, math.log2(maxval) + 2, 3000)
    # values just off midpoints: below half a binary32 ulp, so binary32
    # rounds them onto the midpoint and the chain breaks the tie instead
    mids = grid_midpoints(fmt, rng, 600)
    u = ulp32(mids)
    crafted = np.concatenate([mids + u * 2.0 ** -8, mids - u * 2.0 ** -8, mids, -mids])
    x = np.concatenate([mags, crafted, [0.0, -0.0, 2.0 ** (emin - p), 2.0 ** (emin - p) * 1.0000001,
                                        maxval, -maxval]])
    X = np.asfortranarray(x.reshape(1, -1))
    ref = np.array([exact_round(float(v), fmt) for v in x])
    if fmt == "e4m3":
        # unit scale: the tile maximum would pick e > 0, so quantise with e = 0
        got = np.array([tl.round_format(float(v), fmt) for v in x])
    else:
        got, e = tl.quantise(X, fmt)
        assert e == 0
        got = got.ravel()
    assert np.array_equal(got, ref)
    # the crafted values tell one rounding from the binary32 chain: a slip
    # to double rounding would fail the comparison above on these
    n = len(mids)
    chain = chain_round(crafted[:2 * n], fmt)
    assert np.sum(chain != ref[len(mags):len(mags) + 2 * n]) >= n // 2


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_quantise_tile_against_exact(fmt):
    # a whole tile with its scale: every element is RN_fmt(x / 2^e); the tile
    # maximum is 448 * 2^3, so E4M3 takes e = 3, and the first 8 columns are
    # grid midpoints (after the scale) nudged below half a binary32 ulp
    rng = np.random.default_rng(12)
    X = rng.standard_normal((64, 64))
    X = np.asfortranarray(X / np.max(np.abs(X)) * 448.0 * 8.0 * 0.99)
    X[5, 40] = 448.0 * 8.0
    mids = grid_midpoints(fmt, rng, 64 * 8)
    if fmt == "e4m3":
        mids = mids * 8.0
    X[:, :8] = (mids + ulp32(mids) * 2.0 ** -10).reshape(64, 8)
    Q, e = tl.quantise(X, fmt)
    assert e == (3 if fmt == "e4m3" else 0)
    ref = np.array([exact_round(float(v) * 2.0 ** -e, fmt) for v in X.ravel(order="F")])
    assert np.array_equal(Q.ravel(order="F"), ref)
    chain = chain_round(X[:, :8].ravel(order="F") * 2.0 ** -e, fmt)
    assert np.sum(chain != ref[:64 * 8]) >= 64
