"""Per-task rounding bounds for the mixed-precision factorisation (test helper).

Given the state a factorisation leaves behind -- the updated binary32 tiles
W, the FP64 factor tiles L, the quantised panel tiles Q (format values and
scale exponents) and, for the product form of the panel solve, the inverted
diagonal tiles U -- every task's output is checked against that task's own
inputs, each with an a-priori bound (Higham, Accuracy and Stability of
Numerical Algorithms, 2nd ed.: gamma_n = n u / (1 - n u); Lemma 8.4 and
Theorem 8.5 for substitution in any summation order, Theorem 10.3 for
Cholesky, Section 3.5 for inner products and matrix products):

  QUANT    Q_ik = quantise(L_ik) bit for bit (one rounding from FP64)
  updates  W_ij = fl32(A_ij) - sum_{k<j} 2^(e_ik + e_jk) Q_ik Q_jk^T, k
           ascending; an update adds b exact products to the binary32 tile,
           so it errs by at most gamma_b(2^-23) (|W before| + 2^e |Q_ik||Q_jk|^T)
           (2^-23: faithful rounding of every addition, to nearest or not);
           the bound is carried through the updates of a tile
  POTRF    |L_kk L_kk^T - fp64(W_kk)| <= gamma_{b+1}(2^-53) |L_kk||L_kk^T|
  TRSM     |L_ik L_kk^T - fp64(W_ik)| <= gamma_b(2^-53) |L_ik||L_kk^T|
  TRTRI    |U_k L_kk^T - I| <= gamma_b(2^-53) |U_k||L_kk^T|, U_k upper
  TRMM     |L_ik - fp64(W_ik) U_k| <= gamma_b(2^-53) |W_ik||U_k|
  TRMM_SL  |L_ik - fp64(W_ik) U_k| <= b 2^(eW[r]+eU[c]-58.3) + 2u|L_ik|
           (the product from slices: row exponents of W, column ones of U)

Residuals are formed in numpy's extended precision and the rounding of that
evaluation is added to each bound.  Each check returns the largest ratio of
error to bound (at most 1 passes; an error where the bound is 0 is inf).
"""
import numpy as np

from oracle import tiles as otl
from oracle.cholesky import tile_index

U64 = 2.0 ** -53
UACC = 2.0 ** -23
ULD = float(np.finfo(np.longdouble).eps) / 2.0


def gamma(n, u):
    return n * u / (1.0 - n * u)


def _ld(x):
    return np.asarray(x, dtype=np.longdouble)


def _ratio(err, bound, mask=None):
    err, bound = np.abs(_ld(err)), _ld(bound)
    if mask is not None:
        err, bound = err[mask], bound[mask]
    if err.size == 0:
        return 0.0
    if np.any((bound == 0) & (err > 0)):
        return float("inf")
    pos = bound > 0
    return float(np.max(err[pos] / bound[pos])) if np.any(pos) else 0.0


def _product(A, B):
    """(A B, |A||B|) in extended precision."""
    A, B = _ld(A), _ld(B)
    return A @ B, np.abs(A) @ np.abs(B)


def quant_equal(Lik, q, e, fmt):
    """QUANT: the stored tile is the oracle's quantisation of L_ik."""
    qo, eo = otl.quantise(np.asfortranarray(Lik), fmt)
    return e == eo and np.array_equal(q, qo)


def update_ratio(A32, W, terms, b, lower):
    """W (binary32, after the updates) against fl32(A) minus the exact sum
    of the scaled products; terms = [(qa, ea, qb, eb), ...] in update order.
    lower: a diagonal tile (SYRK updates, lower triangle; the strict upper
    part must be untouched)."""
    E = _ld(np.asarray(A32, dtype=np.float64))
    bnd = np.zeros_like(E)
    for qa, ea, qb, eb in terms:
        s = 2.0 ** (ea + eb)
        P, Pabs = _product(qa, np.transpose(qb))
        P, Pabs = P * s, Pabs * s
        bnd = bnd + gamma(b, UACC) * (np.abs(E) + bnd + Pabs) + gamma(b, ULD) * Pabs
        E = E - P
    bnd = bnd + ULD * np.abs(E)
    err = _ld(np.asarray(W, dtype=np.float64)) - E
    if not lower:
        return _ratio(err, bnd)
    n = W.shape[0]
    low = np.tril(np.ones((n, n), dtype=bool))
    r = _ratio(err, bnd, low)
    if not np.array_equal(np.triu(np.asarray(W), 1), np.triu(np.asarray(A32), 1)):
        return float("inf")
    return r


def potrf_ratio(W32, L):
    """POTRF: L (lower part used) is a Cholesky factor of fp64(W) (lower)."""
    n = L.shape[0]
    Lt = np.tril(L)
    Wd = np.tril(np.asarray(W32, dtype=np.float64))
    R, Rabs = _product(Lt, Lt.T)
    err = R - _ld(Wd)
    bnd = gamma(n + 1, U64) * Rabs + gamma(n + 1, ULD) * (Rabs + np.abs(_ld(Wd)))
    if not np.all(np.diag(Lt) > 0):
        return float("inf")
    return _ratio(err, bnd, np.tril(np.ones((n, n), dtype=bool)))


def trsm_ratio(W32, X, Lkk):
    """TRSM: X L_kk^T = fp64(W) by substitution."""
    n = Lkk.shape[0]
    Lt = np.tril(Lkk)
    R, Rabs = _product(X, Lt.T)
    Wd = _ld(np.asarray(W32, dtype=np.float64))
    err = R - Wd
    bnd = gamma(n, U64) * Rabs + gamma(n, ULD) * (Rabs + np.abs(Wd))
    return _ratio(err, bnd)


def trtri_ratio(U, Lkk):
    """TRTRI: U = L_kk^{-T}, exactly zero below the diagonal."""
    n = Lkk.shape[0]
    if np.any(np.tril(U, -1) != 0.0):
        return float("inf")
    Lt = np.tril(Lkk)
    R, Rabs = _product(U, Lt.T)
    I = _ld(np.eye(n))
    err = R - I
    bnd = gamma(n, U64) * Rabs + gamma(n, ULD) * (Rabs + 1.0)
    return _ratio(err, bnd)


def trmm_sliced_ratio(W32, X, U):
    """TRMM_SL: X = fp64(W) U from the slices (row exponents eW of W,
    column exponents eU of U): per term the truncation bound
    2^(eW[r]+eU[c]-58.3) (tests/sliced_ref.py), b terms, one rounding."""
    import sliced_ref as sr
    n = U.shape[0]
    Wd = np.asarray(W32, dtype=np.float64)
    eW, eU = sr.row_exps(Wd), sr.col_exps(U)
    R, Rabs = _product(Wd, U)
    err = _ld(X) - R
    scale = np.ldexp(1.0, (eW[:, None] + eU[None, :]).astype(np.int64))
    bnd = _ld(n * sr.term_error() * scale) + (2 * U64 + gamma(n, ULD)) * (np.abs(R) + Rabs * ULD)
    return _ratio(err, bnd)


def trmm_ratio(W32, X, U):
    """TRMM: X = fp64(W) U as a product."""
    n = U.shape[0]
    R, Rabs = _product(np.asarray(W32, dtype=np.float64), U)
    err = _ld(X) - R
    bnd = gamma(n, U64) * Rabs + gamma(n, ULD) * Rabs
    return _ratio(err, bnd)


def check_factor(A, Wt, Lt, Q, T, b, fmt, Ut=None, sliced=False):
    """Every task of the factorisation against its bound.

    A: the input (N x N FP64, lower used); Wt, Lt: packed tiles in the
    layout of oracle.cholesky.to_tiles (binary32 and FP64); Q: {(i, k):
    (values [r, c], e)} for i > k; Ut: (T, b, b) inverted diagonal tiles
    (element (r, c) at [k][c, r]) for the product form, else None;
    sliced: the product formed from slices (TRMM_SL), checked against its
    own bound.  Returns {check name: worst ratio} (quant: 0 equal, inf not)."""
    F = lambda t: t.T                                  # tile -> [r, c]
    A32 = {}
    for j in range(T):
        for i in range(j, T):
            A32[(i, j)] = A[i * b:(i + 1) * b, j * b:(j + 1) * b].astype(np.float32)
    W = {(i, j): F(Wt[tile_index(i, j, T)]) for (i, j) in A32}
    L = {(i, j): F(Lt[tile_index(i, j, T)]) for (i, j) in A32}
    out = {"quant": 0.0, "update": 0.0, "potrf": 0.0, "panel": 0.0}
    if Ut is not None:
        out["trtri"] = 0.0
    for (i, k), (q, e) in Q.items():
        if not quant_equal(L[(i, k)], q, e, fmt):
            out["quant"] = float("inf")
    for (i, j) in A32:
        terms = []
        for k in range(j):
            qa, ea = Q[(i, k)]
            qb, eb = Q[(j, k)]
            terms.append((qa, ea, qb, eb))
        out["update"] = max(out["update"], update_ratio(A32[(i, j)], W[(i, j)], terms, b, i == j))
    for k in range(T):
        out["potrf"] = max(out["potrf"], potrf_ratio(W[(k, k)], L[(k, k)]))
        if k + 1 < T and Ut is not None:
            out["trtri"] = max(out["trtri"], trtri_ratio(F(Ut[k]), L[(k, k)]))
        for i in range(k + 1, T):
            if Ut is None:
                r = trsm_ratio(W[(i, k)], L[(i, k)], L[(k, k)])
            elif sliced:
                r = trmm_sliced_ratio(W[(i, k)], L[(i, k)], F(Ut[k]))
            else:
                r = trmm_ratio(W[(i, k)], L[(i, k)], F(Ut[k]))
            out["panel"] = max(out["panel"], r)
    return out
