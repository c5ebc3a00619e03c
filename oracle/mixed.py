"""Oracle for the mixed-precision tiled Cholesky and iterative refinement.

TEST INFRASTRUCTURE ONLY.  The paper has no numerics of its own; this
follows the workload definition of the precision form: trailing-matrix
updates (SYRK, GEMM) take low-precision operands (bfloat16, or FP8 E4M3 with
a power-of-two scale per tile) with binary32 accumulation, while the
diagonal factorisation (POTRF), the panel solve (TRSM) and the refinement
residual stay in FP64.

Data per lower tile (i, j): W_ij binary32 working tile (initialised to
fl32(A_ij)), L_ij FP64 factor tile, and for panel tiles Q_ij the quantised
copy of L_ij with its scale exponent.  Submission order is right-looking:

    for k:
        POTRF_MX(W_kk: R, L_kk: W)        L_kk = chol(fp64(W_kk))
        for i > k:  TRSM_MX(L_kk: R, W_ik: R, L_ik: W, Q_ik: W)
                    L_ik = fp64(W_ik) L_kk^{-T};  Q_ik = quantise(L_ik)
        for i > k:
            SYRK_MX(Q_ik: R, W_ii: RW)     W_ii -= s_ik^2 Q_ik Q_ik^T  (lower)
            for k < j < i:  GEMM_MX(Q_ik: R, Q_jk: R, W_ij: RW)
                           W_ij -= s_ik s_jk Q_ik Q_jk^T
"""
import numpy as np

from . import tiles as _t
from .cholesky import tile_index, ntiles
from .dag import R, W, RW

POTRF_MX, TRSM_MX, SYRK_MX, GEMM_MX = "POTRF_MX", "TRSM_MX", "SYRK_MX", "GEMM_MX"


def task_list(T):
    """(kind, [((buffer, i, j), mode), ...]) in right-looking order; buffer is
    'W', 'L' or 'Q'."""
    out = []
    for k in range(T):
        out.append((POTRF_MX, [(("W", k, k), R), (("L", k, k), W)]))
        for i in range(k + 1, T):
            out.append((TRSM_MX, [(("L", k, k), R), (("W", i, k), R),
                                  (("L", i, k), W), (("Q", i, k), W)]))
        for i in range(k + 1, T):
            out.append((SYRK_MX, [(("Q", i, k), R), (("W", i, i), RW)]))
            for j in range(k + 1, i):
                out.append((GEMM_MX, [(("Q", i, k), R), (("Q", j, k), R),
                                      (("W", i, j), RW)]))
    return out


def factor(A_tiles, T, b, fmt, state=False):
    """Run the mixed task list in submission order on packed FP64 tiles of A
    (unchanged).  Returns (L tiles FP64, info); L tiles use the packed
    layout of cholesky.to_tiles.  state=True also returns the updated
    binary32 tiles W and the quantised panels {(i, k): (Q, e)}."""
    Wt = A_tiles.astype(np.float32)
    Lt = np.zeros_like(A_tiles)
    Q = {}
    for kind, acc in task_list(T):
        if kind == POTRF_MX:
            k = acc[0][0][1]
            t = tile_index(k, k, T)
            Lt[t] = np.tril(Wt[t].T.astype(np.float64)).T   # lower part only
            info = _t.potrf(Lt[t].T)
            if info:
                return (Lt, k * b + info, Wt, Q) if state else (Lt, k * b + info)
        elif kind == TRSM_MX:
            _, i, k = acc[1][0]
            t = tile_index(i, k, T)
            Lt[t] = Wt[t].astype(np.float64)
            _t.trsm(Lt[tile_index(k, k, T)].T, Lt[t].T)
            Q[(i, k)] = _t.quantise(Lt[t].T, fmt)
        elif kind == SYRK_MX:
            _, i, k = acc[0][0]
            qa, ea = Q[(i, k)]
            C = Wt[tile_index(i, i, T)].T
            _t.gemm_lowp(qa, qa, 2.0 ** (2 * ea), C, lower=True)
        else:
            _, i, k = acc[0][0]
            _, j, _ = acc[1][0]
            qa, ea = Q[(i, k)]
            qb, eb = Q[(j, k)]
            C = Wt[tile_index(i, j, T)].T
            _t.gemm_lowp(qa, qb, 2.0 ** (ea + eb), C)
    return (Lt, 0, Wt, Q) if state else (Lt, 0)
