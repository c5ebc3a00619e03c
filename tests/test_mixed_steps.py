"""The per-task bound checker of the mixed-precision factorisation
(tests/mixed_steps.py), pinned on the oracle's own factorisation: it accepts
the oracle's state and rejects each planted mistake (a flipped quantised
value, a perturbed or transposed or missing update, a perturbed diagonal or
panel factor, a wrong inverse or product)."""
import numpy as np
import pytest

import synth
from mixed_steps import (check_factor, potrf_ratio, trmm_ratio, trmm_sliced_ratio, trsm_ratio,
                         trtri_ratio, update_ratio)
from oracle import cholesky as och, ir as oir, mixed as omx, tiles as otl
from oracle.cholesky import tile_index

N, B = 384, 128
T = N // B


@pytest.fixture(scope="module", params=["bf16", "e4m3"])
def state(request):
    fmt = request.param
    A = synth.spd_host(N, seed=11, shift=1.0)
    Lt, info, Wt, Q = omx.factor(och.to_tiles(A, B), T, B, fmt, state=True)
    assert info == 0
    Qd = {k: (np.asarray(q), e) for k, (q, e) in Q.items()}
    return fmt, A, Lt, Wt, Qd


def test_oracle_state_within_bounds(state):
    fmt, A, Lt, Wt, Q = state
    r = check_factor(A, Wt, Lt, Q, T, B, fmt)
    assert r["quant"] == 0.0
    assert r["update"] <= 1.0 and r["potrf"] <= 1.0 and r["panel"] <= 1.0, r
    # the bounds are not vacuous: the updates use a visible share of theirs
    assert r["update"] > 1e-4 and r["potrf"] > 1e-4 and r["panel"] > 1e-4, r


def test_flipped_quantised_value_fails(state):
    fmt, A, Lt, Wt, Q = state
    Q2 = dict(Q)
    q, e = Q[(2, 0)]
    q = q.copy()
    x = q[5, 7]
    step = 2.0 ** -6 if fmt == "bf16" else 2.0 ** -2   # above half the format's spacing
    q[5, 7] = otl.round_format(x * (1.0 + step), fmt) if x != 0 else 2.0 ** -6
    assert q[5, 7] != x
    Q2[(2, 0)] = (q, e)
    assert check_factor(A, Wt, Lt, Q2, T, B, fmt)["quant"] == np.inf


def _terms(Q, i, j):
    return [(Q[(i, k)][0], Q[(i, k)][1], Q[(j, k)][0], Q[(j, k)][1]) for k in range(j)]


def _tile(tl, i, j):
    return tl[tile_index(i, j, T)].T


def test_update_mistakes_fail(state):
    fmt, A, Lt, Wt, Q = state
    i, j = 2, 1
    A32 = A[i * B:(i + 1) * B, j * B:(j + 1) * B].astype(np.float32)
    W = _tile(Wt, i, j)
    assert update_ratio(A32, W, _terms(Q, i, j), B, False) <= 1.0
    W2 = W.copy()
    W2[3, 9] += np.float32(1e-4) * max(abs(W2[3, 9]), np.float32(1e-3))
    assert update_ratio(A32, W2, _terms(Q, i, j), B, False) > 1.0
    # transposed operands, a dropped update, a sign error
    swapped = [(qb, eb, qa, ea) for qa, ea, qb, eb in _terms(Q, i, j)]
    assert update_ratio(A32, W, swapped, B, False) > 1.0
    assert update_ratio(A32, W, _terms(Q, i, j)[:-1], B, False) > 1.0
    neg = [(-qa, ea, qb, eb) for qa, ea, qb, eb in _terms(Q, i, j)]
    assert update_ratio(A32, W, neg, B, False) > 1.0
    # a diagonal tile whose strict upper part was written
    Ad = A[i * B:(i + 1) * B, i * B:(i + 1) * B].astype(np.float32)
    Wd = _tile(Wt, i, i)
    assert update_ratio(Ad, Wd, _terms(Q, i, i), B, True) <= 1.0
    Wd2 = Wd.copy()
    Wd2[0, 5] += np.float32(1.0)
    assert update_ratio(Ad, Wd2, _terms(Q, i, i), B, True) == np.inf


def test_factor_mistakes_fail(state):
    fmt, A, Lt, Wt, Q = state
    Lkk, Wkk = _tile(Lt, 1, 1), _tile(Wt, 1, 1)
    assert potrf_ratio(Wkk, Lkk) <= 1.0
    L2 = Lkk.copy()
    L2[40, 17] *= 1.0 + 1e-12
    assert potrf_ratio(Wkk, L2) > 1.0
    Lik, Wik = _tile(Lt, 2, 1), _tile(Wt, 2, 1)
    assert trsm_ratio(Wik, Lik, Lkk) <= 1.0
    X2 = Lik.copy()
    X2[100, 3] *= 1.0 + 1e-12
    assert trsm_ratio(Wik, X2, Lkk) > 1.0
    assert trsm_ratio(Wik, Lik, Lkk.T) > 1.0


def test_inverse_and_product_checks(state):
    fmt, A, Lt, Wt, Q = state
    Lkk, Wik = np.tril(_tile(Lt, 0, 0)), _tile(Wt, 1, 0)
    U = oir.forward_sub(Lkk, np.eye(B)).T              # L_kk^{-T}, upper
    U = np.triu(U)
    assert trtri_ratio(U, Lkk) <= 1.0
    U2 = U.copy()
    U2[10, 50] *= 1.0 + 1e-11
    assert trtri_ratio(U2, Lkk) > 1.0
    U3 = U.copy()
    U3[50, 10] = 1e-30
    assert trtri_ratio(U3, Lkk) == np.inf
    X = Wik.astype(np.float64) @ U
    assert trmm_ratio(Wik, X, U) <= 1.0
    X2 = X.copy()
    X2[7, 90] *= 1.0 + 1e-12
    assert trmm_ratio(Wik, X2, U) > 1.0


def test_sliced_product_check(state):
    # the host restatement of TRMM_SL passes its bound; a perturbation of
    # 1e-11 relative does not
    import sliced_ref as sr
    fmt, A, Lt, Wt, Q = state
    Lkk, Wik = np.tril(_tile(Lt, 0, 0)), _tile(Wt, 1, 0)
    U = np.triu(oir.forward_sub(Lkk, np.eye(B)).T)
    X, _, _ = sr.trmm_sliced(Wik, U)
    assert trmm_sliced_ratio(Wik, X, U) <= 1.0
    X2 = X.copy()
    X2[7, 90] *= 1.0 + 1e-11
    assert trmm_sliced_ratio(Wik, X2, U) > 1.0
