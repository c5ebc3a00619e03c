"""The host restatement of the sliced FP64 residual (tests/sliced_ref.py)
pinned to the mathematics: the digits represent each value to within
2^(e-60), the sliced residual stays within its a-priori bound of the exact
residual (error-free products + math.fsum), and planted mistakes -- a
transposed use of an off-diagonal tile, a dropped tile, a wrong scale, a
wrong digit sign -- break the bound."""
from fractions import Fraction

import numpy as np
import pytest

import synth
import sliced_ref as sr

N, B_, NRHS = 512, 128, 16
T = N // B_


def test_digits_represent_values():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((64, 64)) * 10.0 ** rng.integers(-20, 20, (64, 64))
    M[0, 0] = 0.0
    M[1, 1] = 5e-324
    e = sr.scale_exp(float(np.max(np.abs(M))))
    assert np.max(np.abs(M)) < 2.0 ** (e - 2) <= 2 * np.max(np.abs(M)) * 4
    V = sr.to_int(M, e)
    D = sr.digits(V)
    assert D.min() >= -16 and D.max() <= 15
    assert np.array_equal(sr.from_digits(D), V)
    # trunc(v 2^(60-e)) exactly, against rational arithmetic
    for (r, c) in [(0, 0), (1, 1), (2, 3), (10, 20), (63, 63)]:
        want = int(Fraction(float(M[r, c])) * Fraction(2) ** (60 - e)) if abs(M[r, c]) >= 2.0 ** -1022 else 0
        assert V[r, c] == want
    err = np.abs(M - np.ldexp(V.astype(np.float64), e - 60))
    assert np.all(err < 2.0 ** (e - 60))


@pytest.fixture(scope="module")
def problem():
    A = synth.spd_host(N, seed=3, shift=0.1)
    X = synth.rhs(N, NRHS, seed=5) * 0.3
    Bm = A @ X + 1e-3 * synth.rhs(N, NRHS, seed=6)    # residual of order 1e-3
    rows = list(range(0, N, 37)) + [N - 1]
    Rex = sr.exact_resid_rows(A, X, Bm, rows, B_)
    return A, X, Bm, rows, Rex


def test_sliced_residual_within_bound(problem):
    A, X, Bm, rows, Rex = problem
    R, eA, eX = sr.resid_sliced(A, X, Bm, B_, NRHS)
    bound = sr.resid_bound(eA, eX, rows, Rex, B_, T, NRHS)
    err = np.abs(R[rows] - Rex)
    assert np.all(err <= bound)
    # an FP64 residual formed the plain way agrees to its own rounding
    plain = Bm - np.tril(A) @ X - np.tril(A, -1).T @ X
    assert np.max(np.abs(plain[rows] - Rex)) <= 1e-12


def _mutated(A, X, Bm, how):
    """resid_sliced with one planted mistake."""
    orig_use, orig_exp = sr.use_tile, sr.scale_exp
    try:
        if how == "transposed":
            sr.use_tile = lambda A_, i, J, b: (orig_use(A_, i, J, b).T if i != J else orig_use(A_, i, J, b))
        elif how == "dropped_tile":
            sr.use_tile = lambda A_, i, J, b: (orig_use(A_, i, J, b) * (0.0 if (i, J) == (2, 1) else 1.0))
        elif how == "scale":
            return sr.resid_sliced(A, X, Bm, B_, NRHS, h_shift=34)
        return sr.resid_sliced(A, X, Bm, B_, NRHS)
    finally:
        sr.use_tile, sr.scale_exp = orig_use, orig_exp


@pytest.mark.parametrize("how", ["transposed", "dropped_tile", "scale"])
def test_planted_mistakes_break_the_bound(problem, how):
    A, X, Bm, rows, Rex = problem
    R, eA, eX = _mutated(A, X, Bm, how)
    _, eA0, eX0 = sr.resid_sliced(A, X, Bm, B_, NRHS)
    bound = sr.resid_bound(eA0, eX0, rows, Rex, B_, T, NRHS)
    assert np.any(np.abs(R[rows] - Rex) > bound)


def test_wrong_digit_sign_breaks_the_bound(problem):
    A, X, Bm, rows, Rex = problem
    orig = sr.digits
    try:
        sr.digits = lambda V: (lambda D: np.concatenate([D[:3], -D[3:4], D[4:]]))(orig(V))
        R, eA, eX = sr.resid_sliced(A, X, Bm, B_, NRHS)
    finally:
        sr.digits = orig
    bound = sr.resid_bound(eA, eX, rows, Rex, B_, T, NRHS)
    assert np.any(np.abs(R[rows] - Rex) > bound)


def test_any_consistent_exponent_gives_the_same_sum(problem):
    # the exponent rule only has to keep |v| < 2^(e-2): a larger exponent
    # represents the same values (fewer low digits), within the same bound
    A, X, Bm, rows, Rex = problem
    orig = sr.scale_exp
    try:
        sr.scale_exp = lambda amax: orig(amax) + (1 if amax > 0 else 0)
        R, eA, eX = sr.resid_sliced(A, X, Bm, B_, NRHS)
    finally:
        sr.scale_exp = orig
    assert np.all(np.abs(R[rows] - Rex) <= sr.resid_bound(eA, eX, rows, Rex, B_, T, NRHS))


def test_column_sums_follow_the_warp_order():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((128, 5))
    s = sr.warp_col_sums(M)
    assert np.allclose(s, np.sum(np.abs(M), axis=0), rtol=1e-14)
