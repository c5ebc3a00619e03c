"""Oracle solutions of served requests (test helper, run in spawned worker
processes): the request's padded matrix diag(A, I) from the client's packed
lower tiles, factored by the oracle's sequential tiled Cholesky, then the
oracle's forward and back substitution on the right-hand sides."""
import numpy as np


def dense_rhs(parts):
    """T parts of b x nrhs (part k: [j, r] = B(k*b + r, j)) -> Np x nrhs."""
    T, nrhs, b = parts.shape
    return np.ascontiguousarray(parts.transpose(0, 2, 1).reshape(T * b, nrhs))


def solve(args):
    """(packed tiles, rhs parts, Np, b) -> (X, A symmetric, B), all dense."""
    from oracle import cholesky as och, ir as oir
    tiles, parts, Np, b = args
    T = Np // b
    A = oir.symmetric_from_lower(och.from_tiles(tiles, Np, b))
    Bm = dense_rhs(parts)
    Lt = tiles.copy()
    info = och.run(Lt, T, b)
    assert info == 0, info
    L = np.tril(och.from_tiles(Lt, Np, b))
    return oir.chol_solve(L, Bm), A, Bm
