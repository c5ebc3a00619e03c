"""Pins for the oracle's solves, refinement and backward error."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import cholesky as ch, ir, mixed


def test_substitutions_against_library():
    A = synth.spd_host(128, seed=1)
    L = sla.cholesky(A, lower=True)
    Bv = synth.rhs(128, 5, seed=2)
    Y = ir.forward_sub(L, Bv)
    assert np.allclose(Y, sla.solve_triangular(L, Bv, lower=True), rtol=1e-13, atol=1e-13)
    X = ir.back_sub_t(L, Y)
    assert np.allclose(X, sla.solve_triangular(L.T, Y, lower=False), rtol=1e-13, atol=1e-13)


def test_backward_error_definition():
    A = np.array([[2.0, 1.0], [1.0, 3.0]])
    x = np.array([[1.0], [1.0]])
    b = np.array([[3.0], [5.0]])           # residual (0, 1)
    # ||r|| = 1, ||A||_inf = 4, ||x|| = 1, ||b|| = 5  ->  1 / 9
    assert ir.backward_error(A, x, b) == pytest.approx(1.0 / 9.0, rel=1e-15)
    assert ir.backward_error(A, np.array([[0.8], [1.4]]), np.array([[3.0], [5.0]])) < 1e-15


def test_exact_integer_system():
    A, L0 = synth.integer_spd(48, seed=3)
    X0 = np.random.default_rng(4).integers(-5, 6, (48, 3)).astype(np.float64)
    B = A @ X0
    X = ir.chol_solve(L0, B)
    assert np.max(np.abs(X - X0)) < 1e-9
    assert ir.backward_error(A, X, B) < 1e-15


@pytest.mark.parametrize("fmt", ["bf16"])
def test_refinement_reaches_fp64_accuracy(fmt):
    N, b = 256, 64
    A = synth.spd_host(N, seed=6, shift=1.0)
    B = synth.rhs(N, 4, seed=7)
    Lt, info = mixed.factor(ch.to_tiles(A, b), N // b, b, fmt)
    L = np.tril(ch.from_tiles(Lt, N, b))
    X, its, hist = ir.refine(ir.symmetric_from_lower(A), L, B, tol=1e-12)
    assert hist[-1] <= 1e-12 and its < 30
    Xs = sla.cho_solve(sla.cho_factor(A, lower=True), B)
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(X - Xs)) / np.max(np.abs(Xs)) <= kappa * 1e-12
