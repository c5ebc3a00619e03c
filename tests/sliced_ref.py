"""Host restatement of the sliced FP64 residual (test helper).

The residual r = b - A x (A symmetric, only its lower tiles stored) computed
the way the sliced kinds define it (include/b3t.h, B3T_SLICE_A / B3T_SLICE_X /
B3T_RESID_SL; the Ozaki scheme): every value v of a block with scale
exponent e (e = ilogb(max|block|) + 3) becomes V = trunc(v 2^(60-e)) in
twelve balanced base-32 digits; per tile and part the slice pairs with
s + t <= 11 are multiplied exactly and summed per group m = s + t; the
groups are combined in integers, H = sum_{m<6} G_m 32^(5-m),
L = sum_{m>=6} G_m 32^(11-m), and added to the FP64 accumulator as
H 2^(eA+eX-35), then L 2^(eA+eX-65), tile after tile; r = b - acc.  Every
step is integer arithmetic except those two additions per tile and the final
subtraction, taken here in the same order, so the result is the device's bit
for bit.  Also: the exact residual (error-free products and math.fsum) and
the a-priori bound of the sliced result against it.
"""
import math

import numpy as np

DIGITS = 12
BIAS = 16 * (32 ** 12 - 1) // 31
NP = 16                       # right-hand sides as B-operand rows (zero padded)
U64 = 2.0 ** -53


def scale_exp(amax):
    """Smallest e = ilogb(amax) + 3 (so |v| < 2^(e-2)); 0 for amax = 0."""
    if not amax > 0.0:
        return 0
    _, ex = math.frexp(amax)          # amax = m 2^ex, m in [0.5, 1): ilogb = ex - 1
    return ex + 2


def to_int(M, e):
    """V = trunc(v 2^(60-e)) elementwise (int64); zeros and subnormals -> 0.
    e may be an array broadcasting against M (one exponent per column)."""
    M = np.asarray(M, dtype=np.float64)
    V = np.trunc(np.ldexp(M, 60 - np.asarray(e)))
    V[np.abs(M) < 2.0 ** -1022] = 0.0
    return V.astype(np.int64)


def digits(V):
    """(12, ...) balanced base-32 digits, most significant first."""
    u = V + BIAS
    return np.stack([((u >> (5 * (DIGITS - 1 - s))) & 31) - 16 for s in range(DIGITS)])


def from_digits(D):
    V = np.zeros(D.shape[1:], dtype=np.int64)
    for s in range(DIGITS):
        V = V * 32 + D[s]
    return V


def use_tile(A, i, J, b):
    """Tile (i, J) of the symmetric matrix from the lower triangle of A."""
    if J < i:
        return A[i * b:(i + 1) * b, J * b:(J + 1) * b]
    if J > i:
        return A[J * b:(J + 1) * b, i * b:(i + 1) * b].T
    D = np.tril(A[i * b:(i + 1) * b, i * b:(i + 1) * b])
    return D + np.tril(D, -1).T


def seq_row_sums(M):
    """Row sums of |M| with the columns added in order (as the device does)."""
    return np.cumsum(np.abs(M), axis=1)[:, -1]


def warp_col_sums(M):
    """Column sums of |M| as a warp forms them: lane l adds rows l, l + 32,
    ... in order, then the lanes are combined by the xor tree 16, 8, 4, 2, 1."""
    n = M.shape[0]
    s = np.zeros((32, M.shape[1]))
    for l in range(32):
        for r in range(l, n, 32):
            s[l] = s[l] + np.abs(M[r])
    for o in (16, 8, 4, 2, 1):
        s = s + s[np.arange(32) ^ o]
    return s[0]


def row_sums_of_use(A, i, J, b):
    """The row sums of |A_use(i, J)| the slice part of that use holds."""
    if J < i:
        return seq_row_sums(A[i * b:(i + 1) * b, J * b:(J + 1) * b])
    if J > i:
        return warp_col_sums(A[J * b:(J + 1) * b, i * b:(i + 1) * b])
    return seq_row_sums(use_tile(A, i, i, b))


def x_exps(Xj, nrhs):
    """Per right-hand side exponents of a part (NP entries, padding 0)."""
    ex = np.zeros(NP, dtype=np.int64)
    for c in range(nrhs):
        ex[c] = scale_exp(float(np.max(np.abs(Xj[:, c]))))
    return ex


def group_sums(DA, DX):
    """G_m = sum_{s+t=m} A_s X_t (exact: integers below 2^24, float64 BLAS)."""
    G = np.zeros((DIGITS,) + (DA.shape[1], DX.shape[2]))
    A = DA.astype(np.float64)
    X = DX.astype(np.float64)
    for s in range(DIGITS):
        for t in range(DIGITS - s):
            G[s + t] += A[s] @ X[t]
    return G.astype(np.int64)


def resid_sliced(A, X, B, b, nrhs, pairs=DIGITS - 1, h_shift=35):
    """R = B - A X the sliced way (A: N x N, lower triangle used; X, B:
    N x nrhs).  Returns (R, eA (T x T), eX (T x NP)).  pairs: the largest
    s + t kept (11 in the library); h_shift: the scale of H (35; another
    value plants a mistake)."""
    N = A.shape[0]
    T = N // b
    eA = np.zeros((T, T), dtype=np.int64)
    eX = np.zeros((T, NP), dtype=np.int64)
    DX = []
    for J in range(T):
        Xj = np.zeros((b, NP))
        Xj[:, :nrhs] = X[J * b:(J + 1) * b]
        eX[J] = x_exps(Xj, nrhs)
        DX.append(digits(to_int(Xj, eX[J][None, :])))
    R = np.zeros((N, nrhs))
    for i in range(T):
        acc = np.zeros((b, NP))
        for J in range(T):
            Au = use_tile(A, i, J, b)
            e = scale_exp(float(np.max(np.abs(Au))))
            eA[i, J] = e
            G = group_sums(digits(to_int(Au, e)), DX[J])
            H = np.zeros((b, NP), dtype=np.int64)
            L = np.zeros((b, NP), dtype=np.int64)
            for m in range(min(pairs, DIGITS - 1) + 1):
                if m < 6:
                    H += G[m] << (5 * (5 - m))
                else:
                    L += G[m] << (5 * (11 - m))
            sc = e + eX[J]
            acc = acc + np.ldexp(H.astype(np.float64), sc - h_shift)
            acc = acc + np.ldexp(L.astype(np.float64), sc - 65)
        R[i * b:(i + 1) * b] = B[i * b:(i + 1) * b] - acc[:, :nrhs]
    return R, eA, eX


def _split(x):
    c = 134217729.0 * x                 # 2^27 + 1 (Veltkamp)
    hi = c - (c - x)
    return hi, x - hi


def exact_resid_rows(A, X, B, rows, b):
    """r = b - A x, correctly rounded, for the given rows (Dekker's exact
    products, then math.fsum)."""
    N = A.shape[0]
    out = np.zeros((len(rows), X.shape[1]))
    for k, r in enumerate(rows):
        i = r // b
        arow = np.concatenate([use_tile(A, i, J, b)[r - i * b] for J in range(N // b)])
        ah, al = _split(arow)
        for c in range(X.shape[1]):
            x = X[:, c]
            p = arow * x
            xh, xl = _split(x)
            e = ((ah * xh - p) + ah * xl + al * xh) + al * xl
            out[k, c] = math.fsum([B[r, c]] + list(-p) + list(-e))
    return out


def gamma(n, u=U64):
    return n * u / (1.0 - n * u)


def term_error():
    """Bound on |a x - kept pairs| per product term, over 2^(eA+eX): both
    truncations (|v - V 2^(e-60)| < 2^(e-60), |v| < 2^(e-2)) and the pairs
    with s + t >= 12 (23 - m of them, digit products <= 256)."""
    drop = sum((23 - m) * 256.0 * 2.0 ** (-5 * m - 10) for m in range(12, 23))
    return 2.0 ** -62 * (2.0 + 2.0 ** -58) + drop


def resid_bound(eA, eX, rows, Rex, b, T, nrhs):
    """|R_sliced - r| bound for the given rows: per tile b terms of
    term_error(), the FP64 accumulation (2T additions of terms whose digit
    products sum to at most b (16/31)^2 2^(eA+eX)), and the final rounding
    (plus the reference's own)."""
    out = np.zeros((len(rows), nrhs))
    acc_terms = (16.0 / 31.0) ** 2
    for k, r in enumerate(rows):
        i = r // b
        sc = np.zeros(nrhs)
        for J in range(T):
            sc += np.ldexp(1.0, eA[i, J] + eX[J, :nrhs])
        out[k] = sc * b * (term_error() + acc_terms * gamma(2 * T)) + 3.0 * U64 * np.abs(Rex[k])
    return out


def row_exps(M):
    return np.array([scale_exp(float(np.max(np.abs(M[r])))) for r in range(M.shape[0])], dtype=np.int64)


def col_exps(M):
    return row_exps(M.T)


def trmm_sliced(W32, U):
    """L = fp64(W) U the sliced way (B3T_TRMM_SL): W rows with their own
    exponents, U columns with theirs; one rounding per element.  Returns
    (L, eW, eU)."""
    Wd = np.asarray(W32, dtype=np.float64)
    eW, eU = row_exps(Wd), col_exps(U)
    G = group_sums(digits(to_int(Wd, eW[:, None])), digits(to_int(U, eU[None, :])))
    H = np.zeros(G.shape[1:], dtype=np.int64)
    L = np.zeros(G.shape[1:], dtype=np.int64)
    for m in range(DIGITS):
        if m < 6:
            H += G[m] << (5 * (5 - m))
        else:
            L += G[m] << (5 * (11 - m))
    sc = eW[:, None] + eU[None, :]
    return np.ldexp(H.astype(np.float64), sc - 35) + np.ldexp(L.astype(np.float64), sc - 65), eW, eU


def exact_product_entries(A, B, entries):
    """(A B)[r, c], correctly rounded, for the given (r, c) pairs."""
    out = []
    for r, c in entries:
        a, x = A[r], B[:, c]
        ah, al = _split(a)
        xh, xl = _split(x)
        p = a * x
        e = ((ah * xh - p) + ah * xl + al * xh) + al * xl
        out.append(math.fsum(list(p) + list(e)))
    return np.array(out)
