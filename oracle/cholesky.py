"""Oracle for the tiled Cholesky workload: task list, tile layout, checks.

TEST INFRASTRUCTURE ONLY.

The matrix is split into b x b tiles, each registered as a buffer of its own:
the workaround Section 5.1 of the paper gives for partitioned matrices
("registering various parts of the data separately"), used there for
Cholesky.  Only lower tiles (i >= j) exist.  Submission is right-looking:

    for k in 0..T-1:
        POTRF(A_kk: RW)
        for i in k+1..T-1:  TRSM(A_kk: R, A_ik: RW)
        for i in k+1..T-1:
            SYRK(A_ik: R, A_ii: RW)
            for j in k+1..i-1:  GEMM(A_ik: R, A_jk: R, A_ij: RW)

Packed tile order: column by column, t(i, j) = j*T - j*(j-1)/2 + (i - j) for
i >= j.  Each tile is column-major; as a numpy array ``tiles[t]`` has shape
(b, b) with ``tiles[t][c, r]`` = A[i*b + r, j*b + c] (C order of A_ij^T).
"""
import numpy as np

from . import tiles as _t
from .dag import R, RW

POTRF, TRSM, SYRK, GEMM = "POTRF", "TRSM", "SYRK", "GEMM"


def ntiles(T):
    return T * (T + 1) // 2


def tile_index(i, j, T):
    assert 0 <= j <= i < T
    return j * T - j * (j - 1) // 2 + (i - j)


def task_list(T):
    """Right-looking submission order: list of (kind, [(tile, mode), ...])
    with tiles as (i, j) pairs."""
    out = []
    for k in range(T):
        out.append((POTRF, [((k, k), RW)]))
        for i in range(k + 1, T):
            out.append((TRSM, [((k, k), R), ((i, k), RW)]))
        for i in range(k + 1, T):
            out.append((SYRK, [((i, k), R), ((i, i), RW)]))
            for j in range(k + 1, i):
                out.append((GEMM, [((i, k), R), ((j, k), R), ((i, j), RW)]))
    return out


def accesses(T):
    """task_list(T) with tiles replaced by packed tile indices."""
    return [[(tile_index(i, j, T), m) for (i, j), m in acc] for _, acc in task_list(T)]


def to_tiles(A, b):
    """Dense N x N (lower triangle used) -> packed lower tiles, shape
    (T(T+1)/2, b, b), tiles[t][c, r] = A[i*b + r, j*b + c]."""
    N = A.shape[0]
    assert N % b == 0
    T = N // b
    out = np.empty((ntiles(T), b, b), dtype=A.dtype)
    for j in range(T):
        for i in range(j, T):
            out[tile_index(i, j, T)] = A[i * b:(i + 1) * b, j * b:(j + 1) * b].T
    return out


def from_tiles(tl, N, b, fill_upper=0.0):
    """Packed lower tiles -> dense N x N; tile contents are copied verbatim,
    blocks above the diagonal get fill_upper."""
    T = N // b
    A = np.full((N, N), fill_upper, dtype=tl.dtype)
    for j in range(T):
        for i in range(j, T):
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = tl[tile_index(i, j, T)].T
    return A


def _F(tile):
    """Column-major view of one packed tile: F[r, c] = element (r, c)."""
    v = tile.T
    assert v.flags.f_contiguous
    return v


def run(tl, T, b, stop_on_info=True):
    """Execute task_list(T) on packed tiles `tl` (float64), in submission
    order, each task at once (the sequential reading of Section 3).
    Returns info: 0, or the 1-based global column of the first non-positive
    pivot (the factor is undefined past it)."""
    for kind, acc in task_list(T):
        v = [_F(tl[tile_index(i, j, T)]) for (i, j), _ in acc]
        if kind == POTRF:
            k = acc[0][0][0]
            info = _t.potrf(v[0])
            if info:
                if stop_on_info:
                    return k * b + info
        elif kind == TRSM:
            _t.trsm(v[0], v[1])
        elif kind == SYRK:
            _t.syrk(v[0], v[1])
        else:
            _t.gemm(v[0], v[1], v[2])
    return 0


def dense_potrf(A):
    """Unblocked Cholesky-Crout of a dense matrix (lower triangle of the
    result holds L; the strict upper triangle is left as given)."""
    F = np.asfortranarray(A, dtype=np.float64).copy(order="F")
    info = _t.potrf(F)
    return np.ascontiguousarray(F), info


def rel_residual(L, A):
    """||L L^T - A||_F / ||A||_F over the lower triangle, FP64 (L is taken
    as tril(L))."""
    Lt = np.tril(L)
    D = np.tril(Lt @ Lt.T - A)
    return float(np.linalg.norm(D) / np.linalg.norm(np.tril(A)))


def flops(N):
    """N^3/3 + N^2/2 + N/6 = N(N+1)(2N+1)/6: the operation count of Cholesky."""
    return float(N * (N + 1) * (2 * N + 1) // 6)


def task_flops(kind, b):
    """Flops of one tile task: POTRF b^3/3 (+ lower order), TRSM b^3,
    SYRK b^2 (b + 1), GEMM 2 b^3."""
    return {POTRF: flops(b), TRSM: float(b) ** 3, SYRK: float(b) ** 2 * (b + 1),
            GEMM: 2.0 * b ** 3}[kind]


def run_prefix(get_tile, T, b, budget_s):
    """Run task_list(T) in submission order, each task at once, until
    budget_s seconds have passed (a bounded sample of a factorisation too
    large to run whole).  get_tile(i, j) returns the packed tile (b, b)
    float64 array for (i, j), fetched lazily and then reused.  Returns
    (tasks done, flops done, seconds)."""
    import time
    cache = {}

    def tile(i, j):
        if (i, j) not in cache:
            cache[(i, j)] = np.ascontiguousarray(get_tile(i, j), dtype=np.float64)
        return _F(cache[(i, j)])

    done, fl = 0, 0.0
    t0 = time.perf_counter()
    for kind, acc in task_list(T):
        v = [tile(i, j) for (i, j), _ in acc]
        if kind == POTRF:
            _t.potrf(v[0])
        elif kind == TRSM:
            _t.trsm(v[0], v[1])
        elif kind == SYRK:
            _t.syrk(v[0], v[1])
        else:
            _t.gemm(v[0], v[1], v[2])
        done += 1
        fl += task_flops(kind, b)
        if time.perf_counter() - t0 > budget_s:
            break
    return done, fl, time.perf_counter() - t0
